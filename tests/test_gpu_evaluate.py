"""Section 3's cluster-separation indices and the colour composite on the
device, through the C ABI, against the oracle.

Tolerances: 8-bit inputs -- class sums are exact, the rest FP64: 1e-12
relative; float32 inputs: 1e-9 relative; the colour image is bit-exact.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _compare(g, r, rtol):
    np.testing.assert_array_equal(g["T"], r["T"])
    for key in ("A", "S", "M", "R", "DI"):
        np.testing.assert_allclose(g[key], r[key], rtol=rtol, atol=0, err_msg=key)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("shape", [(1, 64, 64, 2), (3, 301, 257, 4), (8, 512, 512, 16)],
                         ids=["k1_K2", "k3_K4_ragged", "k8_K16"])
def test_cluster_indices_match_oracle(dtype, shape):
    _skip_without_gpu()
    k, H, W, K = shape
    rng = np.random.default_rng(k * 100 + K)
    labels = rng.integers(0, K + 1, size=(H, W)).astype(np.uint8)
    labels[0, :K] = np.arange(1, K + 1)  # every class present
    if dtype == "u8":
        img = rng.integers(0, 256, size=(k, H, W)).astype(np.uint8)
        rtol = 1e-12
    else:
        img = (rng.normal(size=(k, H, W)) * 50.0).astype(np.float32)
        rtol = 1e-9
    m = cva.Model(4, 2)
    g = cva.cva_cluster_indices(_dev(img), _dev(labels), K, m)
    r = oracle.cluster_indices(img.reshape(k, -1).astype(np.float64), labels, K)
    _compare(g, r, rtol)
    m.close()


def test_cluster_indices_errors():
    _skip_without_gpu()
    m = cva.Model(4, 2)
    img = torch.zeros((2, 8, 8), dtype=torch.uint8, device=DEV)
    lab = np.zeros((8, 8), np.uint8)
    lab[0, 0] = 1
    with pytest.raises(cva.CvaError) as e:  # class 2 has no pixels
        cva.cva_cluster_indices(img, _dev(lab), 2, m)
    assert e.value.code == cva.CVA_ERR_EMPTY_CLASS
    lab[1, 1] = 2
    lab[2, 2] = 5
    with pytest.raises(cva.CvaError) as e:  # label above K
        cva.cva_cluster_indices(img, _dev(lab), 2, m)
    assert e.value.code == cva.CVA_ERR_LABEL_RANGE
    m.close()


@pytest.mark.parametrize("hw", [(64, 96), (33, 35)], ids=["aligned", "ragged"])
@pytest.mark.parametrize("invert", [(False, False, False), (True, True, False), (False, True, True)])
def test_rgb_composite_matches_oracle(hw, invert):
    _skip_without_gpu()
    H, W = hw
    planes = np.random.default_rng(H).integers(0, 256, size=(5, H, W)).astype(np.uint8)
    out = torch.empty((H, W, 3), dtype=torch.uint8, device=DEV)
    cva.cva_rgb_composite(_dev(planes), (3, 0, 4), out, invert=invert)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.rgb_composite(planes, (3, 0, 4), invert))


def test_cva_image_separates_undertext_better_than_bands():
    """Section 3's use of the indices: on the CVA 8-bit image the undertext
    and parchment training points are better separated (lower R, higher DI)
    than on any single band; the device indices of the device image agree
    with the oracle's indices of the oracle's image."""
    _skip_without_gpu()
    w = make_workload(601, 12, 256, 256, 3, (2000, 2000, 2000), 2, separation=(1.5, 2.5), both=False)
    cube, labels = _dev(w.cube), _dev(w.labels)
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, 2)
    cva.cva_fit(cube, labels, w.K, m)
    u = torch.empty((2, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, 2, cva.CVA_RANGE_GLOBAL, u)
    # class 3 = undertext (c = 2), class 1 = parchment (c = 0)
    g = cva.cva_cluster_indices(u[:1].contiguous(), labels, w.K, m)
    ref = oracle.fit(w.cube, w.labels, w.K)
    y = oracle.project(w.cube, ref["V"], ref["mu"], 2)
    uo = oracle.to_u8(y, oracle.range_global(y))
    r = oracle.cluster_indices(uo[:1].astype(np.float64), w.labels, w.K)
    np.testing.assert_allclose(g["R"], r["R"], rtol=1e-2)
    X = w.cube.reshape(w.B, -1).astype(np.float64)
    band_R = []
    for b in range(w.B):
        xb = 255.0 * (X[b] - X[b].min()) / (X[b].max() - X[b].min())
        band_R.append(oracle.cluster_indices(xb[None, :], w.labels, w.K)["R"][2, 0])
    assert g["R"][2, 0] < min(band_R)
    m.close()
