"""Batched form (cva_fit_project_batched) against the single-page path and the
oracle, through the C ABI.

Each page of a batch is its own Section 2 problem.  The batched kernels run
the same arithmetic as the single-page ones (exact integer moments, the same
eigensolve, the same FP32 projection), so every page's eigenvalues and 8-bit
image must be bit-identical to cva_fit + cva_project_u8 on that page alone;
against the FP64 oracle the usual tolerance holds (within one level on
>= 99.9 % of pixels, eigenvalues to 1e-6).
"""
import os

import numpy as np
import pytest
import torch

import oracle
from synth import batch_workloads, make_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _skip_without_gpu():
    if DEV is None:
        pytest.skip("no CUDA device")


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _pages(ws):
    out = []
    for w in ws:
        out.append((_to_dev(w.cube), _to_dev(w.labels), w.K, w.k,
                    torch.full((w.k, w.H, w.W), 7, dtype=torch.uint8, device=DEV),
                    torch.zeros(w.B, dtype=torch.float64, device=DEV)))
    return out


def _single(w, cube, labels):
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    o = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, o)
    lam, V, mu, _ = cva.cva_model_get(m)
    m.close()
    return o.cpu().numpy(), lam, V, mu


def _uneven_batch():
    ws = batch_workloads(count=9, seed0=7100, sizes=[128, 256, 384, 512])
    # ragged pages: pixel counts that are not multiples of 8 take the single-page kernels
    ws.append(make_workload(7201, 13, 129, 131, 3, (900, 700, 500), 2, separation=(1.0, 4.0), both=False))
    ws.append(make_workload(7202, 32, 64, 200, 6, (300, 300, 250, 200, 150, 120), 5, separation=(1.0, 4.0)))
    ws.append(make_workload(7203, 1, 97, 64, 2, (400, 300), 1, separation=(1.0, 4.0), both=False))
    return ws


def test_batch_matches_single_page_path_and_oracle():
    _skip_without_gpu()
    ws = _uneven_batch()
    pages = _pages(ws)
    total_px = sum(w.P for w in ws)
    b = cva.Batch(len(ws), total_px, 2_000_000)
    for call in range(2):  # the workspace keeps no state that changes a second call
        for p in pages:
            p[4].fill_(7)
        cva.cva_fit_project_batched(b, pages)
        st = cva.cva_batch_status(b, len(ws))
        assert (st == cva.CVA_OK).all(), st
        for i, (w, p) in enumerate(zip(ws, pages)):
            u_ref, lam_ref, V, mu = _single(w, p[0], p[1])
            np.testing.assert_array_equal(p[4].cpu().numpy(), u_ref, err_msg=f"page {i}")
            np.testing.assert_array_equal(p[5].cpu().numpy(), lam_ref, err_msg=f"page {i}")
    # two pages against the oracle as well
    for i in (0, len(ws) - 3):
        w = ws[i]
        ref = oracle.fit(w.cube, w.labels, w.K)
        r = w.K - 1
        lam = pages[i][5].cpu().numpy()
        assert (np.abs(lam[:r] - ref["lam"][:r]) / ref["lam"][:r]).max() <= 1e-6
        y = oracle.project(w.cube, ref["V"], ref["mu"], w.k)
        u_ref = oracle.to_u8(y, oracle.range_training(y, w.labels))
        d = np.abs(pages[i][4].cpu().numpy().reshape(w.k, -1).astype(np.int32) - u_ref.astype(np.int32))
        assert (d[:r] <= 1).mean() >= 0.999
    b.close()


def test_failed_pages_fail_alone():
    """A page with a label above K and a page that overflows the pooled
    training storage report their errors and leave their images untouched;
    the other pages are unaffected."""
    _skip_without_gpu()
    ws = [make_workload(7300 + i, 12, 256, 256, 3, (800, 600, 400), 2, separation=(1.0, 4.0), both=False)
          for i in range(4)]
    bad = ws[1].labels.copy()
    bad[5, 7] = 9
    pages = _pages(ws)
    pages[1] = (pages[1][0], _to_dev(bad)) + pages[1][2:]
    # room for the training pixels of pages 0-2 (page 1 takes none), not of page 3
    cap = 2 * 1800 + 100
    b = cva.Batch(4, sum(w.P for w in ws), cap)
    cva.cva_fit_project_batched(b, pages)
    st = cva.cva_batch_status(b, 4)
    assert list(st) == [cva.CVA_OK, cva.CVA_ERR_LABEL_RANGE, cva.CVA_OK, cva.CVA_ERR_CAPACITY]
    for i in (1, 3):
        assert int((pages[i][4] != 7).sum().item()) == 0
    for i in (0, 2):
        u_ref, _, _, _ = _single(ws[i], pages[i][0], pages[i][1])
        np.testing.assert_array_equal(pages[i][4].cpu().numpy(), u_ref)
    b.close()


def test_batch_in_a_cuda_graph_and_autotuner():
    _skip_without_gpu()
    ws = batch_workloads(count=6, seed0=7400, sizes=[256, 384, 512])
    pages = _pages(ws)
    b = cva.Batch(len(ws), sum(w.P for w in ws), 1_000_000)
    gpi, per_sm = cva.cva_batch_tune(b, pages)
    assert gpi in (1, 2, 4, 8, 16, 32) and per_sm in (0, 2)
    refs = [_single(w, p[0], p[1])[0] for w, p in zip(ws, pages)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        cva.cva_fit_project_batched(b, pages, stream=s)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cva.cva_fit_project_batched(b, pages, stream=s)
    for p in pages:
        p[4].fill_(7)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert (cva.cva_batch_status(b, len(ws)) == cva.CVA_OK).all()
    for p, u_ref in zip(pages, refs):
        np.testing.assert_array_equal(p[4].cpu().numpy(), u_ref)
    # the projection pass alone, with the models of that batch
    for p in pages:
        p[4].fill_(7)
    cva.cva_project_batched(b, pages)
    torch.cuda.synchronize()
    for p, u_ref in zip(pages, refs):
        np.testing.assert_array_equal(p[4].cpu().numpy(), u_ref)
    b.close()


def test_batch_argument_errors():
    _skip_without_gpu()
    w = make_workload(7500, 12, 64, 64, 3, (200, 200, 200), 2, separation=(1.0, 4.0), both=False)
    b = cva.Batch(2, 2 * w.P, 10_000)
    cube, labels = _to_dev(w.cube), _to_dev(w.labels)
    out = torch.empty((2, 64, 64), dtype=torch.uint8, device=DEV)
    with pytest.raises(cva.CvaError):   # more pages than the workspace holds
        cva.cva_fit_project_batched(b, [(cube, labels, 3, 2, out)] * 3)
    with pytest.raises(cva.CvaError):   # k above the batched limit
        cva.cva_fit_project_batched(b, [(cube, labels, 3, 9, torch.empty((9, 64, 64), dtype=torch.uint8, device=DEV))])
    with pytest.raises(cva.CvaError):   # pixels above the workspace's tile capacity
        big = make_workload(7501, 12, 512, 512, 3, (200, 200, 200), 2, separation=(1.0, 4.0), both=False)
        small = cva.Batch(1, 64 * 64, 10_000)
        cva.cva_fit_project_batched(small, [(_to_dev(big.cube), _to_dev(big.labels), 3, 2,
                                             torch.empty((2, 512, 512), dtype=torch.uint8, device=DEV))])
    b.close()


def test_batch64_at_full_size_against_oracle_and_single_page_path():
    """The 64-page uneven batch as benchmarked (sides 512-3072, 12-23 bands,
    2-6 classes, 1k-100k training pixels a class, 169.5 M pixels): every page
    bit-identical to cva_fit + cva_project_u8 on it alone, and against the
    FP64 oracle its full fit (eigenvalues 1e-6 relative, canonical vectors
    1e-5 in the Sw norm) and its 8-bit images on a sampled band of 24 rows
    (within one level on >= 99.9 % of pixels)."""
    _skip_without_gpu()
    ws = batch_workloads(64, workers=os.cpu_count() or 1)
    pages = _pages(ws)
    ntrain = sum(sum(w.n_train) for w in ws)
    b = cva.Batch(len(ws), sum(w.P for w in ws), int(ntrain) + 1024)
    cva.cva_fit_project_batched(b, pages)
    st = cva.cva_batch_status(b, len(ws))
    assert (st == cva.CVA_OK).all(), st
    rs = np.random.default_rng(64)
    for i, (w, p) in enumerate(zip(ws, pages)):
        u_single, lam_single, V, _ = _single(w, p[0], p[1])
        u = p[4].cpu().numpy()
        lam = p[5].cpu().numpy()
        np.testing.assert_array_equal(u, u_single, err_msg=f"page {i}")
        np.testing.assert_array_equal(lam, lam_single, err_msg=f"page {i}")
        ref = oracle.fit(w.cube, w.labels, w.K)
        r = w.K - 1
        assert (np.abs(lam[:r] - ref["lam"][:r]) / ref["lam"][:r]).max() <= 1e-6, i
        Sw = ref["Sw"]
        for j in range(r):
            d = V[:, j] - ref["V"][:, j]
            assert np.sqrt(max(d @ Sw @ d, 0.0)) <= 1e-5, (i, j)
        tr = np.flatnonzero(w.labels.reshape(-1))
        sub = w.cube.reshape(w.B, -1)[:, tr].reshape(w.B, 1, -1)
        rng_tr = oracle.range_global(oracle.project(sub, ref["V"], ref["mu"], w.k))
        rows = 24
        r0 = int(rs.integers(0, w.H - rows + 1))
        p0, p1 = r0 * w.W, (r0 + rows) * w.W
        u_ref = oracle.to_u8(oracle.project(w.cube, ref["V"], ref["mu"], w.k, p0, p1), rng_tr)
        d = np.abs(u.reshape(w.k, -1)[:, p0:p1].astype(np.int32) - u_ref.astype(np.int32))
        assert (d <= 1).mean() >= 0.999, i
    b.close()



def test_fit_alone_then_projection_equals_the_whole_batch_call():
    """cva_fit_batched (every page's fit, no projection) followed by
    cva_project_batched gives the images of cva_fit_project_batched."""
    _skip_without_gpu()
    ws = batch_workloads(count=5, seed0=7600, sizes=[256, 384])
    pages = _pages(ws)
    b = cva.Batch(len(ws), sum(w.P for w in ws), 500_000)
    cva.cva_fit_project_batched(b, pages)
    ref = [p[4].cpu().numpy() for p in pages]
    lam_ref = [p[5].cpu().numpy() for p in pages]
    for p in pages:
        p[4].fill_(7)
        p[5].fill_(0.0)
    cva.cva_fit_batched(b, pages)
    torch.cuda.synchronize()
    assert all(int((p[4] != 7).sum().item()) == 0 for p in pages)   # nothing projected yet
    assert (cva.cva_batch_status(b, len(ws)) == cva.CVA_OK).all()
    cva.cva_project_batched(b, pages)
    torch.cuda.synchronize()
    for p, u, lam in zip(pages, ref, lam_ref):
        np.testing.assert_array_equal(p[4].cpu().numpy(), u)
        np.testing.assert_array_equal(p[5].cpu().numpy(), lam)
    b.close()


def test_densely_labelled_pages_in_sixteen_classes():
    """Pages labelled everywhere (each pixel with its class, up to 16 classes;
    the batch projects at most 8 variates a page) beside a sparsely labelled one: the batched label passes then stage full
    512-label chunks in every class, and each chunk reserves its rows of the
    tile's share.  Every page bit-identical to the single-page path."""
    _skip_without_gpu()
    import dataclasses

    ws = []
    for i, (B, H, W, K) in enumerate(((20, 160, 208, 16), (9, 128, 96, 5))):
        w = make_workload(7700 + i, B, H, W, K, tuple([150] * K), min(K - 1, 5), separation=(1.0, 4.0))
        lab = (w.classmap + 1).astype(np.uint8)
        ws.append(dataclasses.replace(w, labels=lab, n_train=tuple(int((lab == c + 1).sum()) for c in range(K))))
    ws.append(make_workload(7702, 12, 256, 256, 3, (800, 600, 400), 2, separation=(1.0, 4.0), both=False))
    assert all(min(w.n_train) > w.B for w in ws)
    pages = _pages(ws)
    b = cva.Batch(len(ws), sum(w.P for w in ws), sum(sum(w.n_train) for w in ws) + 1024)
    cva.cva_fit_project_batched(b, pages)
    st = cva.cva_batch_status(b, len(ws))
    assert (st == cva.CVA_OK).all(), st
    for i, (w, p) in enumerate(zip(ws, pages)):
        u_ref, lam_ref, _, _ = _single(w, p[0], p[1])
        np.testing.assert_array_equal(p[4].cpu().numpy(), u_ref, err_msg=f"page {i}")
        np.testing.assert_array_equal(p[5].cpu().numpy(), lam_ref, err_msg=f"page {i}")
    b.close()
