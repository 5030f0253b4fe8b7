"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a hand-solved example, a closed form, a library routine, an
invariant of the mathematics, exact rational arithmetic or brute force.

Section 2 of the paper defines the method (class scatter matrices, their
eigenanalysis, projection and the 0..255 rescale); Section 4 names the
generalized symmetric-definite eigenproblem and notes the sign ambiguity.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
from synth import make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(seed=7, B=5, H=40, W=48, K=3, n=(150, 120, 100), sep=None, both=False):
    return make_workload(seed, B, H, W, K, n, K - 1, separation=sep, both=both)


def _train_matrix(w):
    X = w.cube.reshape(w.B, -1).T.astype(np.float64)
    lab = w.labels.reshape(-1)
    return X, lab


# --------------------------------------------------------------------------
# hand-solved example (tests/golden/two_class_two_band.json)
# --------------------------------------------------------------------------

def _golden_cube():
    g = json.load(open(os.path.join(GOLDEN, "two_class_two_band.json")))
    cube = np.stack([np.array(g["band0"]), np.array(g["band1"])]).astype(np.uint16)
    labels = np.array(g["labels"], np.uint8)
    return g, cube, labels


def test_golden_two_class_two_band_fit():
    g, cube, labels = _golden_cube()
    f = oracle.fit(cube, labels, g["K"])
    np.testing.assert_allclose(f["Sw"], g["Sw"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(f["Sb"], g["Sb"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(f["mu"], g["mean"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(f["lam"], g["lambda"], rtol=1e-14, atol=1e-13)
    np.testing.assert_allclose(f["V"] * np.sqrt(136.0), g["V_times_sqrt136"], rtol=0, atol=1e-12)


def test_golden_two_class_two_band_projection_and_u8():
    g, cube, labels = _golden_cube()
    f = oracle.fit(cube, labels, g["K"])
    y = oracle.project(cube, f["V"], f["mu"], 2)
    np.testing.assert_allclose(y * np.sqrt(136.0), g["scores_times_sqrt136"], rtol=0, atol=1e-12)
    for rng in (oracle.range_global(y), oracle.range_training(y, labels)):
        u = oracle.to_u8(y, rng)
        np.testing.assert_array_equal(u, np.array(g["u8"], np.uint8))


# --------------------------------------------------------------------------
# scatter matrices
# --------------------------------------------------------------------------

def test_scatter_matches_numpy_covariance_and_total_decomposition():
    """Sw = sum_c n_c cov_c (numpy.cov, population form); Sb is pinned by the
    decomposition total scatter = within + between, with the total scatter
    taken from numpy.cov over all training pixels."""
    w = _small(seed=11, B=6, K=4, n=(300, 200, 150, 90), both=True)
    X, lab = _train_matrix(w)
    f = oracle.scatter(w.cube, w.labels, w.K)
    Sw = np.zeros((w.B, w.B))
    for c in range(w.K):
        Xc = X[lab == c + 1]
        assert f["n"][c] == len(Xc)
        Sw += len(Xc) * np.cov(Xc.T, bias=True)
        np.testing.assert_allclose(f["mu_c"][c], Xc.mean(axis=0), rtol=1e-14)
    Xt = X[lab > 0]
    St = len(Xt) * np.cov(Xt.T, bias=True)
    np.testing.assert_allclose(f["Sw"], Sw, rtol=1e-11, atol=1e-9 * np.abs(Sw).max())
    np.testing.assert_allclose(f["Sb"], St - Sw, rtol=1e-8, atol=1e-9 * np.abs(St).max())
    np.testing.assert_allclose(f["mu"], Xt.mean(axis=0), rtol=1e-14)


def test_scatter_exact_rationals_tiny():
    """Exact rational Sw and Sb of a tiny cube (Python fractions) against the
    oracle's FP64 values."""
    rng = np.random.default_rng(3)
    B, H, W, K = 3, 6, 7, 3
    cube = rng.integers(0, 4096, size=(B, H, W)).astype(np.uint16)
    labels = rng.integers(0, K + 1, size=(H, W)).astype(np.uint8)
    for c in range(1, K + 1):
        labels.flat[c * 5] = c  # every class present
    X = cube.reshape(B, -1).T.tolist()
    lab = labels.reshape(-1).tolist()
    groups = {c: [X[p] for p in range(len(lab)) if lab[p] == c + 1] for c in range(K)}
    N = sum(len(v) for v in groups.values())
    mu_c = {c: [Fraction(sum(x[b] for x in v), len(v)) for b in range(B)] for c, v in groups.items()}
    mu = [sum(Fraction(len(groups[c])) * mu_c[c][b] for c in range(K)) / N for b in range(B)]
    Sw = [[Fraction(0)] * B for _ in range(B)]
    Sb = [[Fraction(0)] * B for _ in range(B)]
    for c, v in groups.items():
        for x in v:
            d = [x[b] - mu_c[c][b] for b in range(B)]
            for i in range(B):
                for j in range(B):
                    Sw[i][j] += d[i] * d[j]
        e = [mu_c[c][b] - mu[b] for b in range(B)]
        for i in range(B):
            for j in range(B):
                Sb[i][j] += len(v) * e[i] * e[j]
    f = oracle.scatter(cube, labels, K)
    np.testing.assert_allclose(f["Sw"], np.array(Sw, dtype=float), rtol=1e-13)
    np.testing.assert_allclose(f["Sb"], np.array(Sb, dtype=float), rtol=1e-12, atol=1e-9)


# --------------------------------------------------------------------------
# generalized eigenproblem
# --------------------------------------------------------------------------

def _sign_fix(V):
    V = V.copy()
    for j in range(V.shape[1]):
        a = np.abs(V[:, j])
        i = int(np.flatnonzero(a >= a.max() * (1 - 1e-12))[0])
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V


def test_two_class_fisher_closed_form():
    """K = 2 (LDA, Section 2): v1 is parallel to Sw^-1 (mu_1 - mu_2),
    lambda_1 = (n1 n2 / N) d^T Sw^-1 d, every other eigenvalue is zero."""
    w = make_workload(21, 7, 48, 40, 2, (400, 260), 1, separation=(2.0, 3.0))
    f = oracle.fit(w.cube, w.labels, 2)
    n1, n2 = f["n"]
    d = f["mu_c"][0] - f["mu_c"][1]
    z = np.linalg.solve(f["Sw"], d)
    lam1 = n1 * n2 / (n1 + n2) * float(d @ z)
    assert abs(f["lam"][0] - lam1) <= 1e-11 * lam1
    v = f["V"][:, 0]
    cos = abs(v @ z) / (np.linalg.norm(v) * np.linalg.norm(z))
    assert cos > 1 - 1e-13
    assert np.all(np.abs(f["lam"][1:]) <= 1e-12 * lam1)


def test_geneig_matches_scipy_eigh():
    """scipy.linalg.eigh(Sb, Sw) solves the same generalized
    symmetric-definite problem (LAPACK) with the same V^T Sw V = I scaling."""
    w = _small(seed=5, B=8, K=4, n=(300, 250, 200, 150), sep=(1.0, 4.0), both=True)
    f = oracle.fit(w.cube, w.labels, w.K)
    lam, V = scipy.linalg.eigh(f["Sb"], f["Sw"])
    lam, V = lam[::-1], _sign_fix(V[:, ::-1])
    r = w.K - 1
    np.testing.assert_allclose(f["lam"][:r], lam[:r], rtol=1e-10)
    np.testing.assert_allclose(f["V"][:, :r], V[:, :r], rtol=0, atol=1e-9 * np.abs(V[:, :r]).max())
    assert np.all(np.abs(f["lam"][r:]) <= 1e-12 * f["lam"][0])


def test_within_scatter_identity_reduces_to_symmetric_eigh():
    """With Sw = c I the problem is the ordinary symmetric eigenproblem of
    Sb / c (numpy.linalg.eigh)."""
    rng = np.random.default_rng(2)
    B, c = 9, 3.5
    A = rng.standard_normal((B, B))
    Sb = A @ A.T
    lam, V, _ = oracle.gen_eig(c * np.eye(B), Sb)
    ref_l, ref_v = np.linalg.eigh(Sb / c)
    np.testing.assert_allclose(lam, ref_l[::-1], rtol=1e-12, atol=1e-13 * ref_l.max())
    np.testing.assert_allclose(V, _sign_fix(ref_v[:, ::-1]) / np.sqrt(c), atol=1e-10)


def test_invariants_and_trace_identity():
    """V^T Sw V = I, V^T Sb V = diag(lambda), small residual
    ||Sb v - lambda Sw v||, and sum(lambda) = trace(Sw^-1 Sb)."""
    w = _small(seed=9, B=12, K=5, H=64, W=64, n=(500, 300, 200, 150, 100), sep=(1.0, 4.0), both=True)
    f = oracle.fit(w.cube, w.labels, w.K)
    V, lam, Sw, Sb = f["V"], f["lam"], f["Sw"], f["Sb"]
    np.testing.assert_allclose(V.T @ Sw @ V, np.eye(w.B), atol=1e-10)
    np.testing.assert_allclose(V.T @ Sb @ V, np.diag(lam), atol=1e-10 * lam[0])
    res = np.linalg.norm(Sb @ V - Sw @ V * lam[None, :], axis=0)
    assert res.max() <= 1e-10 * np.linalg.norm(Sb) * np.linalg.norm(V, axis=0).max()
    assert abs(lam.sum() - np.trace(np.linalg.solve(Sw, Sb))) <= 1e-10 * lam.sum()
    assert np.all(np.diff(lam) <= 0)


def test_brute_force_rayleigh_two_bands():
    """B = 2: lambda_1 is the maximum over directions of the Rayleigh
    quotient w^T Sb w / w^T Sw w (dense sweep of 10^6 angles)."""
    w = make_workload(31, 2, 40, 40, 3, (200, 150, 120), 1)
    f = oracle.fit(w.cube, w.labels, 3)
    th = np.linspace(0, np.pi, 1_000_000, endpoint=False)
    W2 = np.stack([np.cos(th), np.sin(th)])
    q = np.einsum("in,ij,jn->n", W2, f["Sb"], W2) / np.einsum("in,ij,jn->n", W2, f["Sw"], W2)
    assert abs(q.max() - f["lam"][0]) <= 1e-9 * f["lam"][0]
    assert abs(q.min() - f["lam"][1]) <= 1e-9 * f["lam"][0]
    best = W2[:, q.argmax()]
    v = f["V"][:, 0] / np.linalg.norm(f["V"][:, 0])
    assert abs(abs(best @ v) - 1) < 1e-9


def test_brute_force_rayleigh_three_bands_sphere():
    """B = 3: a dense sphere grid plus local refinement of the Rayleigh
    quotient reaches lambda_1 from below and never exceeds it."""
    w = make_workload(33, 3, 40, 40, 3, (200, 150, 120), 2)
    f = oracle.fit(w.cube, w.labels, 3)
    th = np.linspace(0, np.pi, 700)
    ph = np.linspace(0, 2 * np.pi, 1400, endpoint=False)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    D = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)]).reshape(3, -1)
    q = np.einsum("in,ij,jn->n", D, f["Sb"], D) / np.einsum("in,ij,jn->n", D, f["Sw"], D)
    assert q.max() <= f["lam"][0] * (1 + 1e-12)
    x = D[:, q.argmax()]
    for _ in range(200):  # power-style refinement on Sw^-1 Sb from the best grid point
        x = np.linalg.solve(f["Sw"], f["Sb"] @ x)
        x /= np.linalg.norm(x)
    qx = x @ f["Sb"] @ x / (x @ f["Sw"] @ x)
    assert abs(qx - f["lam"][0]) <= 1e-10 * f["lam"][0]


def test_sign_convention_tie_goes_to_lowest_band():
    """Section 4: solvers disagree on eigenvector signs.  The convention makes
    the largest-magnitude component positive; with a tie the lowest band wins."""
    Sw = np.eye(2)
    Sb = np.array([[1.0, -1.0], [-1.0, 1.0]])  # top vector (1, -1) / sqrt 2
    lam, V, _ = oracle.gen_eig(Sw, Sb)
    assert lam[0] == pytest.approx(2.0, rel=1e-14)
    assert V[0, 0] > 0 and V[1, 0] < 0
    np.testing.assert_allclose(np.abs(V[:, 0]), [2 ** -0.5] * 2, rtol=1e-14)
    Sb2 = np.array([[1.0, 2.0], [2.0, 4.0]])  # top vector (1, 2) / sqrt 5
    lam, V, _ = oracle.gen_eig(Sw, Sb2)
    assert V[1, 0] > 0 and V[0, 0] > 0
    lam, V, _ = oracle.gen_eig(Sw, -Sb2 + 10 * np.eye(2))
    for j in range(2):
        a = np.abs(V[:, j])
        assert V[np.argmax(a), j] > 0


# --------------------------------------------------------------------------
# invariance properties of the method
# --------------------------------------------------------------------------

def test_affine_band_transform_invariance():
    """x -> A x + b (integer band mixing, gains, offsets, a permutation) leaves
    the eigenvalues and the centred projections unchanged."""
    w = _small(seed=13, B=4, K=3, n=(200, 180, 150), sep=(1.5, 3.0))
    f = oracle.fit(w.cube, w.labels, w.K)
    A = np.array([[2, 1, 0, 0], [0, 1, 0, 0], [0, 0, 0, 3], [1, 0, 1, 0]], dtype=np.int64)
    off = np.array([100, 7, 0, 31], dtype=np.int64)
    X = w.cube.reshape(w.B, -1).astype(np.int64)
    Y = (A @ X + off[:, None])
    assert Y.max() < 65536
    cube2 = Y.astype(np.uint16).reshape(w.cube.shape)
    g = oracle.fit(cube2, w.labels, w.K)
    r = w.K - 1
    np.testing.assert_allclose(g["lam"][:r], f["lam"][:r], rtol=1e-9)
    y1 = oracle.project(w.cube, f["V"], f["mu"], r)
    y2 = oracle.project(cube2, g["V"], g["mu"], r)
    for j in range(r):
        s = np.sign(y1[j] @ y2[j])
        np.testing.assert_allclose(s * y2[j], y1[j], atol=1e-8 * np.abs(y1[j]).max())


def test_replicated_training_set():
    """Duplicating every training pixel doubles Sw and Sb and leaves the
    eigenvalues and canonical directions unchanged."""
    w = _small(seed=17, B=5, K=3, n=(200, 150, 100), sep=(1.0, 3.0))
    f = oracle.fit(w.cube, w.labels, w.K)
    cube2 = np.concatenate([w.cube, w.cube], axis=2)
    lab2 = np.concatenate([w.labels, w.labels], axis=1)
    g = oracle.fit(cube2, lab2, w.K)
    np.testing.assert_allclose(g["Sw"], 2 * f["Sw"], rtol=1e-11)
    np.testing.assert_allclose(g["Sb"], 2 * f["Sb"], rtol=1e-11, atol=1e-9)
    r = w.K - 1
    np.testing.assert_allclose(g["lam"][:r], f["lam"][:r], rtol=1e-10)
    np.testing.assert_allclose(g["V"][:, :r] * np.sqrt(2.0), f["V"][:, :r], rtol=1e-8, atol=1e-12)


# --------------------------------------------------------------------------
# projection, ranges and the 8-bit rescale
# --------------------------------------------------------------------------

def test_projection_direct_definition():
    """y_j[p] = sum_b V[b, j] (x_b[p] - mu_b), by Python loops on a tiny cube."""
    rng = np.random.default_rng(4)
    B, H, W, k = 3, 5, 6, 2
    cube = rng.integers(0, 4096, size=(B, H, W)).astype(np.uint16)
    V = rng.standard_normal((B, B))
    mu = rng.uniform(0, 4000, size=B)
    y = oracle.project(cube, V, mu, k)
    for j in range(k):
        for p in range(H * W):
            ref = 0.0
            for b in range(B):
                ref += V[b, j] * (float(cube.reshape(B, -1)[b, p]) - mu[b])
            assert abs(y[j, p] - ref) <= 1e-9 * (1 + abs(ref))
    ys = oracle.project(cube, V, mu, k, 7, 19)
    np.testing.assert_array_equal(ys, y[:, 7:19])


def test_to_u8_end_points_rounding_and_clamp():
    y = np.array([[0.0, 1.0, 2.0, 0.5 / 255.0 * 2.0, 3.0, -1.0, 1.0 - 1e-12]])
    rng = np.array([0.0, 2.0])
    u = oracle.to_u8(y, rng)[0]
    assert u[0] == 0 and u[2] == 255          # range ends map to 0 and 255
    assert u[1] == 128                         # 127.5 rounds half up
    assert u[3] == 1                           # 0.5 rounds up to 1
    assert u[4] == 255 and u[5] == 0           # clamped outside the range
    assert u[6] == 127                         # just below the half point
    assert np.all(oracle.to_u8(y, np.array([1.0, 1.0])) == 0)  # empty range


def test_ranges_global_and_training():
    y = np.array([[5.0, -2.0, 7.0, 1.0], [0.0, 3.0, -4.0, 9.0]])
    labels = np.array([0, 1, 0, 2], np.uint8)
    np.testing.assert_array_equal(oracle.range_global(y), [-2, 7, -4, 9])
    np.testing.assert_array_equal(oracle.range_training(y, labels), [-2, 1, 3, 9])


def test_to_u16_end_points_rounding_and_clamp():
    y = np.array([[0.0, 1.0, 2.0, 3.0, -1.0, 1.0 - 1e-9, 2.0 / 65535.0]])
    rng = np.array([0.0, 2.0])
    u = oracle.to_u16(y, rng)[0]
    assert u.dtype == np.uint16
    assert u[0] == 0 and u[2] == 65535        # range ends map to 0 and 65535
    assert u[1] == 32768                       # 32767.5 rounds half up
    assert u[3] == 65535 and u[4] == 0         # clamped outside the range
    assert u[5] == 32767                       # just below the half point
    assert u[6] == 1                           # one step of the 16-bit scale
    assert np.all(oracle.to_u16(y, np.array([1.0, 1.0])) == 0)  # empty range


def _order_stat_by_counting(vals, m, largest):
    """The (m+1)-th smallest (or largest) value of vals, by counting: the v
    with at most m values strictly beyond it and more than m at or beyond it."""
    for v in vals:
        beyond = sum(1 for x in vals if (x > v if largest else x < v))
        at_or_beyond = sum(1 for x in vals if (x >= v if largest else x <= v))
        if beyond <= m < at_or_beyond:
            return v
    raise AssertionError("no order statistic")


@pytest.mark.parametrize("P", [1, 2, 7, 100, 401])
@pytest.mark.parametrize("percent", [0.0, 0.01, 0.1, 1.0, 5.0, 12.34, 49.99])
def test_percentile_range_by_counting(P, percent):
    """Third rescale of Section 2: p percent out of each tail.  Brute force by
    counting on small arrays with ties (integers), against the oracle's sort."""
    rng = np.random.default_rng(P * 7 + int(percent * 100))
    y = rng.integers(-20, 20, size=(2, P)).astype(np.float64)
    got = oracle.percentile_range(y, percent)
    m = int(round(percent * 100)) * P // 10000
    for j in range(2):
        vals = list(y[j])
        assert got[2 * j] == _order_stat_by_counting(vals, m, largest=False)
        assert got[2 * j + 1] == _order_stat_by_counting(vals, m, largest=True)


def test_percentile_range_special_cases():
    y = np.random.default_rng(5).normal(size=(3, 1000))
    # nothing taken out: the global range of the first rescale
    np.testing.assert_array_equal(oracle.percentile_range(y, 0.0), oracle.range_global(y))
    # 1 % of 1000 values out of each tail: 10 values gone at each end
    s = np.sort(y, axis=1)
    r = oracle.percentile_range(y, 1.0)
    np.testing.assert_array_equal(r[0::2], s[:, 10])
    np.testing.assert_array_equal(r[1::2], s[:, 989])
    # 0.01 % of 1000 values is 0.1 of a value: nothing taken out
    np.testing.assert_array_equal(oracle.percentile_range(y, 0.01), oracle.range_global(y))
    with pytest.raises(ValueError):
        oracle.percentile_range(y, 0.005)
    with pytest.raises(ValueError):
        oracle.percentile_range(y, 50.0)


# --------------------------------------------------------------------------
# principal components (Section 2: unsupervised PCA of the page)
# --------------------------------------------------------------------------

def _pca_cube(seed=31, B=6, H=20, W=30):
    w = make_workload(seed, B, H, W, 3, (60, 60, 60), 2, separation=(1.0, 3.0))
    return w


def test_pca_matches_numpy_cov_and_eigh():
    w = _pca_cube()
    X = w.cube.reshape(w.B, -1).astype(np.float64)
    r = oracle.pca(w.cube)
    np.testing.assert_allclose(r["mu"], X.mean(axis=1), rtol=1e-13)
    np.testing.assert_allclose(r["C"], np.cov(X), rtol=1e-11, atol=1e-9 * np.abs(np.cov(X)).max())
    lam, U = np.linalg.eigh(np.cov(X))
    lam, U = lam[::-1], U[:, ::-1]
    np.testing.assert_allclose(r["lam"], lam, rtol=1e-10, atol=1e-10 * lam[0])
    for j in range(w.B):  # distinct eigenvalues: vectors equal up to sign
        assert abs(abs(r["V"][:, j] @ U[:, j]) - 1.0) <= 1e-9


def test_pca_invariants():
    w = _pca_cube(seed=32, B=9)
    r = oracle.pca(w.cube)
    V, lam, C = r["V"], r["lam"], r["C"]
    np.testing.assert_allclose(V.T @ V, np.eye(w.B), atol=1e-12)
    np.testing.assert_allclose(C @ V, V * lam, atol=1e-10 * lam[0])
    assert abs(lam.sum() - np.trace(C)) <= 1e-12 * np.trace(C)  # total variance
    assert np.all(np.diff(lam) <= 0)
    for j in range(w.B):  # sign convention: largest-magnitude component positive
        v = V[:, j]
        assert v[np.argmax(np.abs(v))] > 0


def test_pca_mask_selects_pixels():
    w = _pca_cube(seed=33)
    mask = (np.arange(w.P) % 3 == 0).astype(np.uint8).reshape(w.H, w.W)
    r = oracle.pca(w.cube, mask)
    sub = w.cube.reshape(w.B, -1)[:, mask.reshape(-1) > 0]
    r2 = oracle.pca(sub.reshape(w.B, 1, -1))
    assert r["N"] == sub.shape[1]
    np.testing.assert_array_equal(r["mu"], r2["mu"])
    np.testing.assert_array_equal(r["C"], r2["C"])


def test_pca_band_permutation():
    w = _pca_cube(seed=34, B=7)
    perm = np.array([3, 0, 6, 1, 5, 2, 4])
    r = oracle.pca(w.cube)
    rp = oracle.pca(w.cube[perm])
    np.testing.assert_allclose(rp["lam"], r["lam"], rtol=1e-11)
    np.testing.assert_allclose(rp["V"], r["V"][perm], atol=1e-9)


def test_pca_rank_one_closed_form():
    """Pixels on a line x = a + t d: one component, lambda = var(t) |d|^2."""
    rng = np.random.default_rng(35)
    t = rng.integers(0, 40, size=500)
    d = np.array([3, -1, 2, 5])
    a = np.array([1000, 2000, 1500, 500])
    cube = (a[:, None] + t[None, :] * d[:, None]).astype(np.uint16).reshape(4, 20, 25)
    r = oracle.pca(cube)
    lam1 = np.var(t, ddof=1) * float(d @ d)
    assert abs(r["lam"][0] - lam1) <= 1e-11 * lam1
    np.testing.assert_allclose(r["V"][:, 0], d / np.linalg.norm(d), atol=1e-12)
    assert np.all(np.abs(r["lam"][1:]) <= 1e-9 * lam1)


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def test_error_cases():
    w = _small(seed=19, B=4, K=3, n=(100, 100, 100))
    lab = w.labels.copy()
    lab[lab == 3] = 0
    with pytest.raises(oracle.OracleError) as e:
        oracle.fit(w.cube, lab, 3)
    assert e.value.code == oracle.ERR_EMPTY_CLASS
    lab = w.labels.copy()
    lab[0, 0] = 4
    with pytest.raises(oracle.OracleError) as e:
        oracle.fit(w.cube, lab, 3)
    assert e.value.code == oracle.ERR_LABEL
    cube = w.cube.copy()
    cube[2] = 1234  # a dead band: Sw is singular
    with pytest.raises(oracle.OracleError) as e:
        oracle.fit(cube, w.labels, 3)
    assert e.value.code == oracle.ERR_NOT_SPD


# --------------------------------------------------------------------------
# quality sanity (Section 3, Davies-Bouldin index, eqs. 1-3)
# --------------------------------------------------------------------------

def _dbi(a, b):
    """Eq. 3 for two one-dimensional clusters, through the oracle."""
    y = np.concatenate([a, b])[None, :]
    labels = np.concatenate([np.ones(a.size), 2 * np.ones(b.size)]).astype(np.uint8)
    return oracle.cluster_indices(y, labels, 2)["R"][0, 1]


def test_cluster_indices_hand_solved_one_band():
    """Class 1 = {0, 2}: centroid 1, scatter 1.  Class 2 = {10, 14}: centroid
    12, scatter 2.  M = 11, R = 3/11 (eq. 3), DI = (11 - 3)/2 = 4 (eq. 5)."""
    y = np.array([[0.0, 10.0, 2.0, 14.0, 99.0]])
    labels = np.array([1, 2, 1, 2, 0], np.uint8)
    r = oracle.cluster_indices(y, labels, 2)
    np.testing.assert_array_equal(r["T"], [2, 2])
    np.testing.assert_array_equal(r["A"][:, 0], [1.0, 12.0])
    np.testing.assert_array_equal(r["S"], [1.0, 2.0])
    assert r["M"][0, 1] == 11.0 and r["M"][1, 0] == 11.0
    assert r["R"][0, 1] == pytest.approx(3.0 / 11.0, rel=1e-15)
    assert r["DI"][0, 1] == 4.0
    assert r["R"][0, 0] == 0.0 and r["DI"][1, 1] == 0.0


def test_cluster_indices_hand_solved_two_bands():
    """{(0,0), (0,2)}: centroid (0,1), scatter 1; {(3,1), (5,1)}: centroid
    (4,1), scatter 1; M = 4, R = 1/2, DI = (4 - 2)/1 = 2; a third class
    {(0,1)} has scatter 0 and the same centroid as the first: R = inf."""
    y = np.array([[0.0, 0.0, 3.0, 5.0, 0.0], [0.0, 2.0, 1.0, 1.0, 1.0]])
    labels = np.array([1, 1, 2, 2, 3], np.uint8)
    r = oracle.cluster_indices(y, labels, 3)
    np.testing.assert_array_equal(r["A"], [[0.0, 1.0], [4.0, 1.0], [0.0, 1.0]])
    np.testing.assert_array_equal(r["S"], [1.0, 1.0, 0.0])
    assert r["R"][0, 1] == 0.5 and r["DI"][0, 1] == 2.0
    assert np.isinf(r["R"][0, 2])


def test_cluster_indices_invariances():
    rng = np.random.default_rng(44)
    y = rng.normal(size=(3, 400))
    labels = rng.integers(0, 4, size=400).astype(np.uint8)
    r = oracle.cluster_indices(y, labels, 3)
    rs = oracle.cluster_indices(7.5 * y + 3.0, labels, 3)      # scale and shift of the image
    np.testing.assert_allclose(rs["R"], r["R"], rtol=1e-12)
    np.testing.assert_allclose(rs["DI"], r["DI"], rtol=1e-12, atol=1e-12)
    rp = oracle.cluster_indices(y[[2, 0, 1]], labels, 3)       # band order
    np.testing.assert_allclose(rp["R"], r["R"], rtol=1e-12)
    perm = np.array([0, 3, 1, 2], np.uint8)                     # class order: 1->3, 2->1, 3->2
    rc = oracle.cluster_indices(y, perm[labels], 3)
    np.testing.assert_allclose(rc["R"][np.ix_([2, 0, 1], [2, 0, 1])], r["R"], rtol=1e-12)
    with pytest.raises(oracle.OracleError):
        oracle.cluster_indices(y, np.zeros(400, np.uint8), 2)   # empty classes


def test_rgb_composite_hand_example():
    planes = np.array([[[10, 20]], [[30, 40]], [[50, 60]]], np.uint8)  # 3 planes of 1 x 2
    rgb = oracle.rgb_composite(planes, (2, 0, 1))
    assert rgb.tolist() == [[[50, 10, 30], [60, 20, 40]]]
    rgb = oracle.rgb_composite(planes, (0, 0, 2), invert=(True, False, True))
    assert rgb.tolist() == [[[245, 10, 205], [235, 20, 195]]]


def test_cva_image_separates_undertext_better_than_any_band():
    """Section 3 / Section 4: the best CVA grayscale image separates 200
    undertext points from 200 parchment points better (lower Davies-Bouldin
    index) than any single band normalised to 0..255."""
    w = make_workload(41, 12, 256, 256, 3, (2000, 2000, 2000), 2, separation=(1.5, 2.5), both=False)
    f = oracle.fit(w.cube, w.labels, w.K)
    y = oracle.project(w.cube, f["V"], f["mu"], 2)
    u = oracle.to_u8(y, oracle.range_global(y)).astype(np.float64)
    cm = w.classmap.reshape(-1)
    rng = np.random.default_rng(0)
    und = rng.choice(np.flatnonzero(cm == 2), 200, replace=False)
    par = rng.choice(np.flatnonzero(cm == 0), 200, replace=False)
    cva = min(_dbi(u[j, und], u[j, par]) for j in range(2))
    X = w.cube.reshape(w.B, -1).astype(np.float64)
    bands = []
    for b in range(w.B):
        xb = 255.0 * (X[b] - X[b].min()) / (X[b].max() - X[b].min())
        bands.append(_dbi(xb[und], xb[par]))
    assert cva < min(bands)
