"""Third rescale (p percent out of each tail) and the 16-bit image, through the
C ABI, against the oracle.

Tolerances:
  * the trimmed range is a pair of exact order statistics of the float32
    values it is given: bit-identical to the oracle's on the same values;
  * 16-bit codes from float32 values: within one level everywhere (the FP32
    rescale against the FP64 one, 65535 levels);
  * end to end from a cube (FP32 projection against the FP64 oracle): 8-bit
    within one level on >= 99.9 % of pixels; 16-bit within one level on
    >= 99.9 % and two everywhere.
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


def _values(seed, k, P):
    """Seeded float32 'projections': a Gaussian body, heavy tails and ties."""
    rng = np.random.default_rng(seed)
    y = rng.normal(0.0, 40.0, size=(k, P))
    y[:, ::7] = np.round(y[:, ::7])                  # ties
    y[:, ::97] *= 50.0                               # outliers in both tails
    return y.astype(np.float32)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 7), (3, 1003, 997), (3, 2048, 2048)],
                         ids=["1px", "7px", "ragged_1003x997", "2048x2048"])
@pytest.mark.parametrize("percent", [0.0, 0.01, 0.1, 1.0, 5.0, 49.99])
def test_percentile_range_is_exact(shape, percent):
    _skip_without_gpu()
    k, H, W = shape
    y = _values(int(percent * 100) + H, k, H * W)
    m = cva.Model(4, 2)
    r = torch.empty(2 * k, dtype=torch.float32, device=DEV)
    cva.cva_percentile_range(torch.from_numpy(y.reshape(k, H, W)).to(DEV), percent, m, r)
    ref = oracle.percentile_range(y.astype(np.float64), percent).astype(np.float32)
    np.testing.assert_array_equal(r.cpu().numpy(), ref)
    m.close()


def test_percentile_range_scratch_is_reusable():
    """Consecutive calls on one model (different k, percent) stay exact."""
    _skip_without_gpu()
    m = cva.Model(4, 2)
    for i, (k, P, pc) in enumerate([(5, 4096, 1.0), (2, 999, 5.0), (32, 512, 0.1)]):
        y = _values(50 + i, k, P)
        r = torch.empty(2 * k, dtype=torch.float32, device=DEV)
        cva.cva_percentile_range(torch.from_numpy(y.reshape(k, 1, P)).to(DEV), pc, m, r)
        ref = oracle.percentile_range(y.astype(np.float64), pc).astype(np.float32)
        np.testing.assert_array_equal(r.cpu().numpy(), ref)
    m.close()


def test_percentile_argument_errors():
    _skip_without_gpu()
    m = cva.Model(4, 2)
    y = torch.zeros((1, 4, 4), dtype=torch.float32, device=DEV)
    r = torch.empty(2, dtype=torch.float32, device=DEV)
    for bad in (0.005, 50.0, -1.0):
        with pytest.raises(cva.CvaError):
            cva.cva_percentile_range(y, bad, m, r)
    m.close()


@pytest.mark.parametrize("shape", [(2, 64, 96), (3, 101, 77)], ids=["aligned", "ragged"])
def test_to_u16_given_and_global(shape):
    _skip_without_gpu()
    k, H, W = shape
    y = _values(7, k, H * W)
    yd = torch.from_numpy(y.reshape(k, H, W)).to(DEV)
    given = np.array([v for j in range(k) for v in (np.percentile(y[j], 3), np.percentile(y[j], 96))], np.float32)
    m = cva.Model(4, 2)
    out = torch.empty((k, H, W), dtype=torch.uint16, device=DEV)
    cva.cva_to_u16(yd, cva.CVA_RANGE_GIVEN, out, range=torch.from_numpy(given).to(DEV))
    ref = oracle.to_u16(y.astype(np.float64), given.astype(np.float64))
    d = np.abs(out.cpu().numpy().reshape(k, -1).astype(np.int64) - ref.astype(np.int64))
    assert d.max() <= 1
    cva.cva_to_u16(yd, cva.CVA_RANGE_GLOBAL, out, m=m)
    ref = oracle.to_u16(y.astype(np.float64), oracle.range_global(y.astype(np.float64)))
    u = out.cpu().numpy().reshape(k, -1)
    d = np.abs(u.astype(np.int64) - ref.astype(np.int64))
    assert d.max() <= 1
    assert (u.min(axis=1) == 0).all() and (u.max(axis=1) == 65535).all()
    m.close()


def test_third_rescale_and_16_bit_end_to_end():
    """A cube through fit, FP32 projection, the 1 % trimmed range and both
    rescales, against the oracle's FP64 pipeline."""
    _skip_without_gpu()
    w = make_workload(401, 23, 512, 640, 4, (4000, 3000, 2000, 1500), 3, separation=(1.0, 4.0), both=True)
    cube, labels = torch.from_numpy(w.cube).to(DEV), torch.from_numpy(w.labels).to(DEV)
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    y = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=DEV)
    cva.cva_project(cube, m, w.k, out_f32=y)
    r = torch.empty(2 * w.k, dtype=torch.float32, device=DEV)
    cva.cva_percentile_range(y, 1.0, m, r)
    u8 = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_to_u8(y, cva.CVA_RANGE_GIVEN, u8, range=r)
    u16 = torch.empty((w.k, w.H, w.W), dtype=torch.uint16, device=DEV)
    cva.cva_to_u16(y, cva.CVA_RANGE_GIVEN, u16, range=r)
    ref = oracle.fit(w.cube, w.labels, w.K)
    y_ref = oracle.project(w.cube, ref["V"], ref["mu"], w.k)
    r_ref = oracle.percentile_range(y_ref, 1.0)
    d8 = np.abs(u8.cpu().numpy().reshape(w.k, -1).astype(np.int64) - oracle.to_u8(y_ref, r_ref).astype(np.int64))
    assert (d8 <= 1).mean() >= 0.999
    d16 = np.abs(u16.cpu().numpy().reshape(w.k, -1).astype(np.int64) - oracle.to_u16(y_ref, r_ref).astype(np.int64))
    assert (d16 <= 1).mean() >= 0.999 and d16.max() <= 2
    # 16-bit with the training range
    cva.cva_to_u16(y, cva.CVA_RANGE_TRAINING, u16, m=m)
    d16 = np.abs(u16.cpu().numpy().reshape(w.k, -1).astype(np.int64) -
                 oracle.to_u16(y_ref, oracle.range_training(y_ref, w.labels)).astype(np.int64))
    assert (d16 <= 1).mean() >= 0.999 and d16.max() <= 2
    m.close()
