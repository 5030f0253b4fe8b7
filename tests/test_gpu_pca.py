"""Principal components (cva_pca_fit) against the oracle's FP64 PCA, through
the C ABI.

Tolerances: mean within 1e-12 relative; covariance within 1e-10 of its
largest entry; eigenvalues within 1e-6 relative, each to itself (all B of
them); unit
eigenvectors within 1e-6 componentwise after the sign convention (the
synthetic covariances have well separated eigenvalues); FP32 projections
within 1e-4 normwise per component; 8-bit images within one level on
>= 99.9 % of pixels.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import make_workload, named_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _skip_without_gpu():
    if DEV is None:
        pytest.skip("no CUDA device")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _check(w, m, cube, ref, k):
    lam, V, mu, _ = cva.cva_model_get(m)
    n, mc, C, Sb = cva.cva_model_get_scatter(m)
    assert n[0] == ref["N"]
    np.testing.assert_allclose(mu, ref["mu"], rtol=1e-12)
    assert np.abs(C - ref["C"]).max() <= 1e-10 * np.abs(ref["C"]).max()
    assert np.all(Sb == 0.0)
    rel = np.abs(lam - ref["lam"]) / np.abs(ref["lam"])  # every eigenvalue relative to itself
    assert rel.max() <= 1e-6, rel
    assert np.abs(V[:, :k] - ref["V"][:, :k]).max() <= 1e-6
    np.testing.assert_allclose(V[:, :k].T @ V[:, :k], np.eye(k), atol=1e-9)
    y = torch.empty((k, w.H, w.W), dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, k, out_f32=y)
    y_ref = oracle.project(w.cube, ref["V"], ref["mu"], k)
    yg = y.cpu().numpy().reshape(k, -1)
    assert (np.abs(yg - y_ref).max(axis=1) / np.abs(y_ref).max(axis=1)).max() <= 1e-4
    out = torch.empty((k, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, k, cva.CVA_RANGE_GLOBAL, out)
    u_ref = oracle.to_u8(y_ref, oracle.range_global(y_ref))
    d = np.abs(out.cpu().numpy().reshape(k, -1).astype(np.int32) - u_ref.astype(np.int32))
    assert (d <= 1).mean() >= 0.999


CASES = [
    # seed, B, H, W, masked
    (501, 23, 256, 320, False),
    (502, 16, 257, 301, False),   # P not a multiple of 8: per-pixel staging
    (503, 32, 128, 160, False),
    (504, 1, 64, 64, False),
    (505, 12, 200, 200, True),
]


@pytest.mark.parametrize("case", CASES, ids=[f"B{c[1]}_{c[2]}x{c[3]}{'_mask' if c[4] else ''}" for c in CASES])
def test_pca_matches_oracle(case):
    _skip_without_gpu()
    seed, B, H, W, masked = case
    w = make_workload(seed, B, H, W, 3, (300, 300, 300), 2, separation=(1.0, 4.0), both=False)
    cube = _dev(w.cube)
    mask = None
    if masked:  # a cropped "folio": a rectangle and a few scattered pixels
        mask = np.zeros((H, W), np.uint8)
        mask[20:170, 30:185] = 1
        mask.reshape(-1)[::97] = 3
    m = cva.Model(B, 2)
    cva.cva_pca_fit(cube, m, mask=_dev(mask) if masked else None)
    assert cva.cva_status(m) == cva.CVA_OK
    _check(w, m, cube, oracle.pca(w.cube, mask), B)
    m.close()


def test_pca_unaligned_mask_and_refusals():
    _skip_without_gpu()
    w = make_workload(506, 10, 96, 128, 3, (300, 300, 300), 2, separation=(1.0, 4.0), both=False)
    cube = _dev(w.cube)
    mask = np.zeros((w.H, w.W), np.uint8)
    mask[10:80, 5:120] = 1
    base = torch.zeros(w.P + 8, dtype=torch.uint8, device=DEV)
    md = base[3:3 + w.P].view(w.H, w.W)   # 1-byte aligned: per-pixel staging
    md.copy_(_dev(mask))
    m = cva.Model(w.B, 2)
    cva.cva_pca_fit(cube, m, mask=md)
    _check(w, m, cube, oracle.pca(w.cube, mask), 4)
    out = torch.empty((2, w.H, w.W), dtype=torch.uint8, device=DEV)
    with pytest.raises(cva.CvaError):  # no training pixels after a PCA fit
        cva.cva_project_u8(cube, m, 2, cva.CVA_RANGE_TRAINING, out)
    one = np.zeros((w.H, w.W), np.uint8)
    one[5, 5] = 1
    cva.cva_pca_fit(cube, m, mask=_dev(one))
    assert cva.cva_status(m) == cva.CVA_ERR_EMPTY_CLASS
    m.close()


def test_pca_then_cva_on_one_model():
    _skip_without_gpu()
    w = make_workload(507, 14, 128, 128, 2, (500, 400), 1, separation=(1.0, 4.0), both=False)
    cube, labels = _dev(w.cube), _dev(w.labels)
    m = cva.Model(w.B, w.K)
    cva.cva_pca_fit(cube, m)
    cva.cva_fit(cube, labels, w.K, m)
    assert cva.cva_status(m) == cva.CVA_OK
    ref = oracle.fit(w.cube, w.labels, w.K)
    lam, V, mu, tr = cva.cva_model_get(m)
    assert abs(lam[0] - ref["lam"][0]) <= 1e-6 * ref["lam"][0]
    out = torch.empty((1, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, 1, cva.CVA_RANGE_TRAINING, out)  # allowed again
    m.close()


def test_pca_of_the_23_band_4096x4096_page():
    """The whole 16.8 M-pixel page, as Section 2's unsupervised PCA takes it."""
    _skip_without_gpu()
    w = named_workload("cube23b_4096x4096_K4")
    cube = _dev(w.cube)
    m = cva.Model(w.B, 2)
    cva.cva_set_variates(m, 5)
    cva.cva_pca_fit(cube, m)
    ref = oracle.pca(w.cube)
    lam, V, mu, _ = cva.cva_model_get(m)
    np.testing.assert_allclose(mu, ref["mu"], rtol=1e-12)
    assert (np.abs(lam - ref["lam"]) / ref["lam"]).max() <= 1e-6
    assert np.abs(V[:, :5] - ref["V"][:, :5]).max() <= 1e-6
    out = torch.empty((5, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, 5, cva.CVA_RANGE_GLOBAL, out)
    y = torch.empty((5, w.H, w.W), dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, 5, out_f32=y)
    y_ref = oracle.project(w.cube, ref["V"], ref["mu"], 5)
    yg = y.reshape(5, -1).cpu().numpy()
    assert (np.abs(yg - y_ref).max(axis=1) / np.abs(y_ref).max(axis=1)).max() <= 1e-4
    u_ref = oracle.to_u8(y_ref, oracle.range_global(y_ref))
    d = np.abs(out.reshape(5, -1).cpu().numpy().astype(np.int32) - u_ref.astype(np.int32))
    assert (d <= 1).mean() >= 0.999
    m.close()
