"""The page-split protocol (paper_1612_06457_gb300/split.py) on CPU: two gloo
ranks, each holding one band of rows of a page, run run_split with stand-in
parts whose phases use exact integer sums and the FP64 oracle (test
infrastructure, no GPU).  Section 2's scatter matrices are sums over the
training pixels, so the merged moments must equal the whole page's exactly,
and with the merged training-score range every band's 8-bit image must be
the whole page's image band by band.  The CUDA parts are checked the same
way on one GPU in test_gpu_split.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1612_06457_gb300.split import merge_ranges, row_band, run_split


def _moments(cube, labels, K):
    """Exact class moments in the layout of cva_model_moments: class c, then
    the upper triangle of sum x'_a x'_b with x' = (x, 1), row-major."""
    B = cube.shape[0]
    X = cube.reshape(B, -1).T.astype(np.int64)
    lab = labels.reshape(-1)
    out = []
    iu = np.triu_indices(B + 1)
    for c in range(K):
        Xa = np.hstack([X[lab == c + 1], np.ones((int((lab == c + 1).sum()), 1), np.int64)])
        out.append((Xa.T @ Xa)[iu])
    return np.concatenate(out)


class OraclePart:
    """A part whose phases are exact integer sums and the FP64 oracle."""

    def __init__(self, cube, labels, K, k):
        self.cube, self.labels, self.K, self.k = cube, labels, K, k
        self.B = cube.shape[0]

    def moments(self):
        return torch.from_numpy(_moments(self.cube, self.labels, self.K)), 0

    def fit(self, total):
        import oracle

        B, K = self.B, self.K
        iu = np.triu_indices(B + 1)
        t = total.numpy().reshape(K, -1)
        n, s, M = [], [], []
        for c in range(K):
            A = np.zeros((B + 1, B + 1), np.int64)
            A[iu] = t[c]
            A = A + np.triu(A, 1).T
            n.append(A[B, B])
            s.append(A[:B, B])
            M.append(A[:B, :B])
        N = sum(n)
        mu_c = [s[c] / n[c] for c in range(K)]
        mu = sum(s) / N
        Sw = sum(M[c] - np.outer(s[c], s[c]) / n[c] for c in range(K))
        Sb = sum(n[c] * np.outer(mu_c[c] - mu, mu_c[c] - mu) for c in range(K))
        lam, V, _ = oracle.gen_eig(Sw, Sb)
        self.V, self.mu = V, mu
        tr = np.flatnonzero(self.labels.reshape(-1))
        sub = self.cube.reshape(B, -1)[:, tr].reshape(B, 1, -1)
        rng = oracle.range_global(oracle.project(sub, V, mu, self.k)) if tr.size else \
            np.array([np.inf, -np.inf] * self.k)
        self.lam = lam
        return torch.from_numpy(rng.astype(np.float64)), 0

    def project(self, rng, out):
        import oracle

        y = oracle.project(self.cube, self.V, self.mu, self.k)
        out.copy_(torch.from_numpy(oracle.to_u8(y, rng.numpy()).reshape(out.shape)))


def _page():
    from synth import make_workload

    return make_workload(6100, 12, 120, 96, 3, (900, 700, 600), 2, separation=(1.0, 4.0), both=False)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    try:
        _rank_body(rank, world, port, q)
    except Exception as exc:  # noqa: BLE001 - reported to the parent
        q.put((rank, "error", repr(exc)))
        raise


def _rank_body(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _page()
    r0, r1 = row_band(w.H, world, rank)
    part = OraclePart(np.ascontiguousarray(w.cube[:, r0:r1]), np.ascontiguousarray(w.labels[r0:r1]), w.K, w.k)
    out = torch.empty((w.k, r1 - r0, w.W), dtype=torch.uint8)
    seen = {}
    inner = part.fit

    def fit(total):  # keep what the part saw of the exchange
        seen["total"] = total.clone()
        return inner(total)

    part.fit = fit
    run_split(part, out)
    q.put((rank, r0, r1, out.numpy(), seen["total"].numpy(), part.lam))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_page():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=180) for _ in range(2)], key=lambda t: t[0])
    for g in got:
        assert g[1] != "error", g
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _page()
    whole = OraclePart(w.cube, w.labels, w.K, w.k)
    mom, _ = whole.moments()
    rng, _ = whole.fit(mom)
    img = torch.empty((w.k, w.H, w.W), dtype=torch.uint8)
    whole.project(rng, img)
    for rank, r0, r1, band, total, lam in got:
        np.testing.assert_array_equal(total, mom.numpy())          # exact merge
        np.testing.assert_array_equal(lam, whole.lam)
        np.testing.assert_array_equal(band, img.numpy()[:, r0:r1])  # the page's image, band by band
    assert got[0][2] == got[1][1] and got[0][1] == 0 and got[1][2] == w.H


def test_row_bands_cover_the_page():
    for H in (1, 2, 7, 4096):
        for parts in (1, 2, 3, 8):
            if parts > H:
                continue
            bands = [row_band(H, parts, i) for i in range(parts)]
            assert bands[0][0] == 0 and bands[-1][1] == H
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [b - a for a, b in bands]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        row_band(10, 2, 2)


def test_merge_ranges_interleaves():
    lo = torch.tensor([1.0, 2.0])
    hi = torch.tensor([5.0, 6.0])
    assert merge_ranges(lo, hi).tolist() == [1.0, 5.0, 2.0, 6.0]
