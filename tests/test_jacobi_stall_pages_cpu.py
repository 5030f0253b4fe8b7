"""CPU check of the premise of the GPU stall-rule test (test_gpu_parity's
EARLY_STALL pages): on each page the reduced K x K problem T = G^T G
(G = L^-1 Mb, S_w = L L^T, S_b = Mb Mb^T, T scaled by a power of two to about
unit norm, as the finalize kernel scales it) makes a cyclic Jacobi in FP32
that declares itself stalled once a sweep shrinks the off-diagonal norm by
less than 4x stop after one sweep, far from diagonal; with the stall test
applied only once off/total < 1e-9 the same model diagonalizes T.  The
matrices come from the FP64 oracle; the Jacobi here is a plain model of the
rotation formulas (Golub & Van Loan's symmetric Schur rotation), not the
kernel."""
import numpy as np
import pytest

import oracle
from synth import make_workload

F = np.float32
PAGES = [(9089, 8, 5, "cyclic"), (9094, 8, 5, "cyclic"), (9405, 8, 4, "round-robin"),
         (9298, 8, 6, "round-robin"), (9526, 12, 10, "round-robin")]


def _reduced(seed, B, K):
    w = make_workload(seed, B, 64, 64, K, (150,) * K, min(K - 1, 3), separation=(1.0, 4.0), both=False)
    r = oracle.fit(w.cube, w.labels, w.K)
    Mb = np.sqrt(r["n"].astype(np.float64))[None, :] * (r["mu_c"].T - r["mu"][:, None])
    np.testing.assert_allclose(Mb @ Mb.T, r["Sb"], rtol=1e-9, atol=1e-9 * np.abs(r["Sb"]).max())
    G = np.linalg.solve(np.linalg.cholesky(r["Sw"]), Mb)
    T = G.T @ G
    ex = np.frexp(np.sqrt((T * T).sum()))[1]
    return T * 2.0 ** (-int(ex))


def _rotate(a, w, p, q):
    apq = a[p, q]
    if apq == 0:
        return
    tau = (a[q, q] - a[p, p]) / (F(2) * apq)
    u = tau * tau + F(1)
    t = np.copysign(F(1) / (abs(tau) + np.sqrt(u)), tau)
    cs = F(1) / np.sqrt(t * t + F(1))
    sn = t * cs
    for m in (a, w):
        x, y = m[:, p].copy(), m[:, q].copy()
        m[:, p], m[:, q] = cs * x - sn * y, sn * x + cs * y
    x, y = a[p, :].copy(), a[q, :].copy()
    a[p, :], a[q, :] = cs * x - sn * y, sn * x + cs * y


def _pairs(n, order):
    if order == "cyclic":
        return [[(p, q) for p in range(n - 1) for q in range(p + 1, n)]]
    m = n + (n & 1)
    seat = lambda i, rnd: 0 if i == 0 else 1 + (i - 1 + rnd) % (m - 1)
    rounds = []
    for rnd in range(m - 1):
        prs = [tuple(sorted((seat(i, rnd), seat(m - 1 - i, rnd)))) for i in range(m // 2)]
        rounds.append([pq for pq in prs if pq[1] < n])
    return rounds


def _jacobi(T, order, gate):
    n = T.shape[0]
    a, w = T.astype(F), np.eye(n, dtype=F)
    tot, prev = F((a * a).sum()), F(3e38)
    for sweep in range(40):
        off = F((a * a).sum() - (np.diag(a) ** 2).sum())
        stalled = off >= F(0.25) * prev and (gate is None or off <= F(gate) * tot)
        if off <= F(1e-11) * tot or stalled:
            return sweep, float(off / tot)
        prev = off
        for rnd in _pairs(n, order):
            for p, q in rnd:
                _rotate(a, w, p, q)
    return 40, float(off / tot)


@pytest.mark.parametrize("page", PAGES, ids=[f"seed{p[0]}_K{p[2]}_{p[3]}" for p in PAGES])
def test_old_rule_stops_after_one_sweep_and_the_gated_rule_converges(page):
    seed, B, K, order = page
    T = _reduced(seed, B, K)
    sweeps, rel = _jacobi(T, order, gate=None)
    assert sweeps == 1 and rel > 0.05, (sweeps, rel)
    sweeps, rel = _jacobi(T, order, gate=1e-9)
    assert rel <= 1e-9, (sweeps, rel)
