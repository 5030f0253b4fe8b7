"""Projection of ragged cubes through the C ABI: pixel counts that are not a
multiple of 8, cubes that do not start on 16 bytes, and unaligned output
planes, against the oracle and against the other output paths.

Section 2 of the paper projects every pixel of the page; real page scans have
any width and height.  Such cubes take the two-chunk streaming kernel; its
results must meet the same bars as the aligned kernel's: FP32 projections
within 1e-4 normwise of the oracle, 8-bit images within one level on
>= 99.9 % of pixels, the fused 8-bit path bit-identical to FP32 projection +
cva_to_u8, and the global range bit-exact against the FP32 projections.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _skip_without_gpu():
    if DEV is None:
        pytest.skip("no CUDA device")


def _view(a, dtype, offset):
    """A device copy of numpy array `a` that starts `offset` elements into
    its allocation (an unaligned view)."""
    flat = torch.empty(a.size + offset + 16, dtype=dtype, device=DEV)
    v = flat[offset:offset + a.size].view(a.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return v


def _empty(shape, dtype, offset):
    n = int(np.prod(shape))
    flat = torch.empty(n + offset + 16, dtype=dtype, device=DEV)
    return flat[offset:offset + n].view(shape)


def _fit(w, cube, labels):
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    assert cva.cva_status(m) == cva.CVA_OK
    return m


CASES = [
    # seed, B, H, W, K, k, cube offset (values), output offset (bytes / floats)
    (801, 13, 97, 89, 4, 3, 0, 0),     # P % 8 = 1
    (802, 23, 61, 107, 5, 4, 3, 1),    # P % 8 = 7, cube 6 bytes off, outputs off
    (803, 7, 98, 83, 3, 2, 1, 2),      # P % 8 = 6
    (804, 32, 67, 61, 4, 9, 5, 3),     # two passes of variates (8 + 1), P % 8 = 7
    (805, 16, 64, 64, 6, 5, 2, 0),     # P % 8 == 0 but the cube starts 4 bytes off
    (806, 12, 64, 64, 3, 2, 0, 5),     # aligned cube, unaligned outputs
    (807, 2, 5, 6, 2, 1, 1, 1),        # below 32 pixels: the scalar kernel
]


@pytest.mark.parametrize("case", CASES, ids=[f"B{c[1]}_{c[2]}x{c[3]}_k{c[5]}_o{c[6]}{c[7]}" for c in CASES])
def test_ragged_cube_projection(case):
    _skip_without_gpu()
    seed, B, H, W, K, k, co, oo = case
    n = tuple([max(8, H * W // (4 * K))] * K)
    w = make_workload(seed, B, H, W, K, n, k, separation=(1.0, 4.0), both=False, cap_frac=0.9)
    if w.P < 64:  # a page this small is all strokes: label every other pixel of each class by hand
        w.labels[...] = 0
        w.labels.reshape(-1)[0::2] = 1
        w.labels.reshape(-1)[1::2] = 2
    cube = _view(w.cube, torch.uint16, co)
    labels = torch.from_numpy(w.labels).to(DEV)
    m = _fit(w, cube, labels)
    lam, V, mu, tr = cva.cva_model_get(m)
    y = _empty((k, H, W), torch.float32, oo)
    rg = torch.empty(2 * k, dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, k, out_f32=y, range_out=rg)
    yg = y.cpu().numpy().reshape(k, -1)
    y_ref = oracle.project(w.cube, V, mu, k)  # the oracle's projection with the fitted vectors
    assert (np.abs(yg - y_ref).max(axis=1) / np.abs(y_ref).max(axis=1)).max() <= 1e-4
    np.testing.assert_array_equal(rg.cpu().numpy()[0::2], yg.min(axis=1))
    np.testing.assert_array_equal(rg.cpu().numpy()[1::2], yg.max(axis=1))
    for mode in (cva.CVA_RANGE_TRAINING, cva.CVA_RANGE_GLOBAL):
        fused = _empty((k, H, W), torch.uint8, oo)
        fused.fill_(7)
        cva.cva_project_u8(cube, m, k, mode, fused)
        two = torch.empty((k, H, W), dtype=torch.uint8, device=DEV)
        cva.cva_to_u8(y, mode, two, m=m)
        np.testing.assert_array_equal(fused.cpu().numpy(), two.cpu().numpy())
        rng = oracle.range_training(y_ref, w.labels) if mode == cva.CVA_RANGE_TRAINING else oracle.range_global(y_ref)
        u_ref = oracle.to_u8(y_ref, rng)
        d = np.abs(fused.cpu().numpy().reshape(k, -1).astype(np.int32) - u_ref.astype(np.int32))
        assert (d <= 1).mean() >= 0.999
    m.close()


def test_ragged_page_23b_4093x4099():
    """A page the size of the benchmark page with odd sides (4093 x 4099,
    P % 8 = 7): the fit and the fused 8-bit projection against the oracle,
    FP32 projections and codes on sampled row bands."""
    _skip_without_gpu()
    w = make_workload(1009, 23, 4093, 4099, 4, (50000,) * 4, 3, separation=(1.0, 4.0), both=True)
    assert w.P % 8 == 7
    cube = torch.from_numpy(w.cube).to(DEV)
    labels = torch.from_numpy(w.labels).to(DEV)
    m = _fit(w, cube, labels)
    ref = oracle.fit(w.cube, w.labels, w.K)
    lam, V, mu, _ = cva.cva_model_get(m)
    r = w.K - 1
    assert (np.abs(lam[:r] - ref["lam"][:r]) / ref["lam"][:r]).max() <= 1e-6
    out = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out)
    y = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, w.k, out_f32=y)
    tr = np.flatnonzero(w.labels.reshape(-1))
    sub = w.cube.reshape(w.B, -1)[:, tr].reshape(w.B, 1, -1)
    rng_tr = oracle.range_global(oracle.project(sub, ref["V"], ref["mu"], w.k))
    u = out.reshape(w.k, -1).cpu().numpy()
    yg = y.reshape(w.k, -1).cpu().numpy()
    for r0 in (0, 1777, w.H - 32):   # first rows, middle, last rows (the scalar head and tail)
        p0, p1 = r0 * w.W, (r0 + 32) * w.W
        y_ref = oracle.project(w.cube, ref["V"], ref["mu"], w.k, p0, p1)
        assert (np.abs(yg[:, p0:p1] - y_ref).max(axis=1) / np.abs(y_ref).max(axis=1)).max() <= 1e-4
        d = np.abs(u[:, p0:p1].astype(np.int32) - oracle.to_u8(y_ref, rng_tr).astype(np.int32))
        assert (d <= 1).mean() >= 0.999
    m.close()
