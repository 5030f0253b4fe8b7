"""The FP64 form (CVA_PRECISION_FP64) against the FP64 oracle, and the mixed
form against the FP64 form, through the C ABI.

Tolerances:
  * FP64 projections, stored as float32: max |y - y_ref| / max |y_ref| <= 2e-7
    per variate (one float rounding of an FP64 result);
  * FP64-form 8-bit images: identical to the oracle's at every pixel whose
    oracle score is not within 1e-9 (of a bin) of a bin edge, and within one
    level at those (a code can differ only where an FP64 score sits within
    rounding of an edge; with one band and integer data whole groups of
    pixels sit exactly on edges);
  * mixed (FP32) projections against the FP64 form: relative 1e-4, the bound
    the mixed form is held to.
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


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _normwise(y, yref):
    return (np.abs(y - yref).max(axis=1) / np.abs(yref).max(axis=1)).max()


def _codes_match(u, uref, y=None, rng=None):
    d = np.abs(u.astype(np.int32) - uref.astype(np.int32))
    assert d.max() <= 1
    if y is None:
        assert (d == 0).mean() >= 0.99999
        return
    # the oracle's unrounded code position 255 (y - lo) / (hi - lo) + 1/2
    lo, hi = rng[0::2][:, None], rng[1::2][:, None]
    t = 255.0 * (y - lo) / (hi - lo) + 0.5
    edge = np.abs(t - np.rint(t)) <= 1e-9
    assert (d[~edge] == 0).all()


CASES = [
    # seed, B, H, W, K, n per class, nvec (= k projected)
    (201, 16, 200, 264, 3, (2000, 1500, 1200), 2),
    (202, 23, 257, 301, 4, (3000, 2000, 1500, 900), 3),   # P not a multiple of 8
    (203, 32, 96, 128, 5, (900, 800, 700, 600, 500), 12),  # two passes of 8 and 4 variates
    (204, 1, 64, 96, 2, (500, 400), 1),
]


@pytest.mark.parametrize("case", CASES, ids=[f"B{c[1]}_{c[2]}x{c[3]}_K{c[4]}_k{c[6]}" for c in CASES])
def test_fp64_form_matches_oracle(case):
    _skip_without_gpu()
    seed, B, H, W, K, n, k = case
    w = make_workload(seed, B, H, W, K, n, k, separation=(1.0, 4.0), both=K >= 4)
    cube, labels = _to_dev(w.cube), _to_dev(w.labels)
    m = cva.Model(B, K)
    cva.cva_set_variates(m, k)
    cva.cva_set_precision(m, cva.CVA_PRECISION_FP64)
    cva.cva_fit(cube, labels, K, m)
    assert cva.cva_status(m) == cva.CVA_OK
    lam, V, mu, tr = cva.cva_model_get(m)
    y_own = oracle.project(w.cube, V, mu, k)

    y = torch.empty((k, H, W), dtype=torch.float32, device=DEV)
    rg = torch.empty(2 * k, dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, k, out_f32=y, range_out=rg)
    yg = y.cpu().numpy().reshape(k, w.P)
    assert _normwise(yg, y_own) <= 2e-7
    r_glob = oracle.range_global(y_own)
    r_tr = oracle.range_training(y_own, w.labels)
    np.testing.assert_array_equal(rg.cpu().numpy(), r_glob.astype(np.float32))
    np.testing.assert_array_equal(tr[: 2 * k], r_tr.astype(np.float32))

    out = torch.empty((k, H, W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, k, cva.CVA_RANGE_TRAINING, out)
    _codes_match(out.cpu().numpy().reshape(k, w.P), oracle.to_u8(y_own, r_tr), y_own, r_tr)
    cva.cva_project_u8(cube, m, k, cva.CVA_RANGE_GLOBAL, out)
    _codes_match(out.cpu().numpy().reshape(k, w.P), oracle.to_u8(y_own, r_glob), y_own, r_glob)
    given = np.empty(2 * k, np.float32)
    given[0::2] = np.percentile(y_own, 2, axis=1)
    given[1::2] = np.percentile(y_own, 97, axis=1)
    cva.cva_project_u8(cube, m, k, cva.CVA_RANGE_GIVEN, out, range=_to_dev(given))
    _codes_match(out.cpu().numpy().reshape(k, w.P), oracle.to_u8(y_own, given.astype(np.float64)), y_own,
                 given.astype(np.float64))
    m.close()


def test_precision_can_change_after_the_fit():
    _skip_without_gpu()
    w = make_workload(205, 23, 256, 256, 4, (3000, 2000, 1500, 900), 3, separation=(1.0, 4.0), both=True)
    cube, labels = _to_dev(w.cube), _to_dev(w.labels)
    outs = []
    for fit_mode in (cva.CVA_PRECISION_MIXED, cva.CVA_PRECISION_FP64):
        m = cva.Model(w.B, w.K)
        cva.cva_set_precision(m, fit_mode)
        cva.cva_fit(cube, labels, w.K, m)
        cva.cva_set_precision(m, cva.CVA_PRECISION_FP64)
        o = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=DEV)
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, o)
        _, _, _, tr = cva.cva_model_get(m)
        outs.append((o.cpu().numpy(), tr[: 2 * w.k].copy()))
        # and back: the mixed training range is still the fit's own
        cva.cva_set_precision(m, cva.CVA_PRECISION_MIXED)
        o2 = torch.empty_like(o)
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, o2)
        y = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=DEV)
        cva.cva_project(cube, m, w.k, out_f32=y)
        yn = y.cpu().numpy().reshape(w.k, w.P)
        lab = w.labels.reshape(-1) > 0
        _, _, _, tr_m = cva.cva_model_get(m)
        np.testing.assert_array_equal(tr_m[0 : 2 * w.k : 2], yn[:, lab].min(axis=1))
        np.testing.assert_array_equal(tr_m[1 : 2 * w.k : 2], yn[:, lab].max(axis=1))
        m.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def test_mixed_form_within_1e4_of_fp64_form_on_the_23_band_cube():
    """4096 x 4096, 23 bands, 4 classes of 50,000 training pixels: the mixed
    FP32 projection against the FP64 form over every pixel."""
    _skip_without_gpu()
    w = make_workload(1001, 23, 4096, 4096, 4, (50000,) * 4, 3, separation=(1.0, 4.0), both=True)
    cube, labels = _to_dev(w.cube), _to_dev(w.labels)
    m = cva.Model(w.B, w.K)
    cva.cva_fit(cube, labels, w.K, m)
    ys = []
    for mode in (cva.CVA_PRECISION_MIXED, cva.CVA_PRECISION_FP64):
        cva.cva_set_precision(m, mode)
        y = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=DEV)
        cva.cva_project(cube, m, w.k, out_f32=y)
        ys.append(y.reshape(w.k, -1))
    err = ((ys[0] - ys[1]).abs().amax(dim=1) / ys[1].abs().amax(dim=1)).max().item()
    assert err <= 1e-4, err
    m.close()
