"""The adversarial-spectrum pages (synth/spectra.py): their premises, and the
oracle on them pinned to a 50-digit solution of the same problem.

Section 2 of the paper forms the within- and between-class scatter of the
training pixels and takes the eigenvectors of their eigenanalysis; Section 4
solves it as the generalized symmetric-definite problem Sb v = lambda Sw v.
Here Sw and Sb are formed EXACTLY (Python fractions of the integer class
moments) and the problem is solved by Cholesky reduction and a symmetric
eigensolver in 50-digit arithmetic (mpmath), independently of the oracle's C
code.  On these pages the oracle's FP64 results are then held to 1e-7
relative per eigenvalue and 1e-7 per canonical vector in the Sw norm (inside
a degenerate pair: the pair's subspace; on the near-singular page, where the
oracle's FP64 scatter sums meet cond(Sw) ~ 1e11, 2e-6), so that the GPU
tests, which compare against the oracle at 1e-6 / 1e-5, compare against
values known to be right.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth.spectra import degenerate_pair_page, near_singular_page, wide_spread_page

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _exact_scatter(w):
    """Sw and Sb as exact fractions from the integer moments of the training
    pixels (the definitions: Sw = sum_c sum_p (x - mu_c)(x - mu_c)^T,
    Sb = sum_c n_c (mu_c - mu)(mu_c - mu)^T)."""
    B, K = w.B, w.K
    X = w.cube.reshape(B, -1).T.astype(np.int64)
    lab = w.labels.reshape(-1)
    n, s, M = [], [], []
    for c in range(K):
        Xc = X[lab == c + 1]
        n.append(int(Xc.shape[0]))
        s.append([int(v) for v in Xc.sum(axis=0)])
        Mc = Xc.T @ Xc
        M.append([[int(Mc[i, j]) for j in range(B)] for i in range(B)])
    N = sum(n)
    S = [sum(s[c][b] for c in range(K)) for b in range(B)]
    Sw = [[sum(Fraction(n[c] * M[c][i][j] - s[c][i] * s[c][j], n[c]) for c in range(K)) for j in range(B)]
          for i in range(B)]
    Sb = [[sum(Fraction((N * s[c][i] - n[c] * S[i]) * (N * s[c][j] - n[c] * S[j]), n[c] * N * N)
               for c in range(K)) for j in range(B)] for i in range(B)]
    return Sw, Sb


def _mp(F):
    return mp.matrix([[mp.mpf(x.numerator) / x.denominator for x in row] for row in F])


def _mp_solution(Sw, Sb, dps=50):
    """Descending eigenvalues and Sw-orthonormal eigenvectors (columns, as
    float64) of Sb v = lambda Sw v in `dps`-digit arithmetic."""
    mp.dps = dps
    A, Bm = _mp(Sw), _mp(Sb)
    L = mp.cholesky(A)
    Li = L ** -1
    C = Li * Bm * Li.T
    C = (C + C.T) / 2
    ev, Q = mp.eigsy(C)
    V = Li.T * Q
    n = len(Sw)
    order = sorted(range(n), key=lambda i: -ev[i])
    lam = np.array([float(ev[i]) for i in order])
    Vf = np.array([[float(V[b, i]) for i in order] for b in range(n)])
    return lam, Vf


def _sw_dist(u, v, Sw):
    d = u - v
    return float(np.sqrt(max(d @ Sw @ d, 0.0)))


def _signed(v):
    return v if v[np.argmax(np.abs(v))] > 0 else -v


def test_wide_spread_premise_and_oracle_pin():
    w = wide_spread_page()
    Sw, Sb = _exact_scatter(w)
    lam_mp, V_mp = _mp_solution(Sw, Sb)
    r = w.K - 1
    assert lam_mp[0] / lam_mp[r - 1] >= 1e8          # the page's premise
    f = oracle.fit(w.cube, w.labels, w.K)
    assert np.all(np.abs(f["lam"][:r] - lam_mp[:r]) / lam_mp[:r] <= 1e-7)
    Swf = np.array([[float(x) for x in row] for row in Sw])
    for j in range(r):
        assert _sw_dist(f["V"][:, j], _signed(V_mp[:, j]), Swf) <= 1e-7


def test_near_singular_premise_and_oracle_pin():
    w = near_singular_page()
    Sw, Sb = _exact_scatter(w)
    Swf = np.array([[float(x) for x in row] for row in Sw])
    assert np.linalg.cond(Swf) >= 1e10                # the page's premise
    f = oracle.fit(w.cube, w.labels, w.K)             # positive definite: no NOT_SPD
    lam_mp, V_mp = _mp_solution(Sw, Sb)
    r = w.K - 1
    assert np.all(np.abs(f["lam"][:r] - lam_mp[:r]) / lam_mp[:r] <= 1e-7)
    for j in range(r):
        assert _sw_dist(f["V"][:, j], _signed(V_mp[:, j]), Swf) <= 2e-6


def _rot(F):
    """R F R^T for R the band map of the degenerate page (a quarter turn of
    bands 0 and 1, sign change of band 2), on a matrix of fractions."""
    B = len(F)
    R = [[0] * B for _ in range(B)]
    R[0][1], R[1][0], R[2][2] = -1, 1, -1
    for b in range(3, B):
        R[b][b] = 1
    RF = [[sum(R[i][k] * F[k][j] for k in range(B)) for j in range(B)] for i in range(B)]
    return [[sum(RF[i][k] * R[j][k] for k in range(B)) for j in range(B)] for i in range(B)]


@pytest.mark.parametrize("split", [0, 20, 40])
def test_degenerate_pair_premise_and_oracle_pin(split):
    w = degenerate_pair_page(perturb=split)
    Sw, Sb = _exact_scatter(w)
    if split == 0:  # both scatter matrices commute with R exactly
        assert _rot(Sw) == Sw and _rot(Sb) == Sb
    lam_mp, V_mp = _mp_solution(Sw, Sb)
    gap = (lam_mp[0] - lam_mp[1]) / lam_mp[0]
    assert gap <= 1e-6                                 # the page's premise
    if split == 0:
        assert gap <= 1e-30
    f = oracle.fit(w.cube, w.labels, w.K)
    r = w.K - 1
    assert np.all(np.abs(f["lam"][:r] - lam_mp[:r]) / lam_mp[:r] <= 1e-7)
    Swf = np.array([[float(x) for x in row] for row in Sw])
    # the pair: the oracle's two vectors span the 50-digit pair's subspace
    P = V_mp[:, :2]
    Vo = f["V"][:, :2]
    resid = Vo - P @ (P.T @ Swf @ Vo)
    assert max(_sw_dist(resid[:, j], 0 * resid[:, j], Swf) for j in range(2)) <= 1e-7
    assert _sw_dist(f["V"][:, 2], _signed(V_mp[:, 2]), Swf) <= 1e-7
