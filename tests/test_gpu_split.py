"""One page split into bands of rows (paper_1612_06457_gb300/split.py)
through the C ABI, the parts driven one after another on one GPU: the
phases of the protocol are the ones run_split runs on one GPU per part, and
the exchanges (an int64 sum of the class moments, a min / max merge of the
training-score ranges) are done here on the device.  Section 2's scatter
matrices are sums over the training pixels and the moments are exact
integers, so the merged moments, eigenvalues, canonical vectors and every
band of the 8-bit image must be bit-identical to cva_fit + cva_project_u8 on
the whole page."""
import numpy as np
import pytest
import torch

from synth import make_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")
split = pytest.importorskip("paper_1612_06457_gb300.split")

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _whole(w, cube, labels):
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    assert cva.cva_status(m) == cva.CVA_OK
    out = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=DEV)
    cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out)
    lam, V, mu, rng = cva.cva_model_get(m)
    mom = torch.empty(cva.moment_words(w.B, w.K), dtype=torch.int64, device=DEV)
    cva.cva_model_moments(m, mom)
    m.close()
    return out.cpu().numpy(), lam, V, rng[: 2 * w.k], mom.cpu().numpy()


def _parts(w, n, labels=None):
    lab = w.labels if labels is None else labels
    out = []
    for i in range(n):
        r0, r1 = split.row_band(w.H, n, i)
        cube = torch.from_numpy(np.ascontiguousarray(w.cube[:, r0:r1])).to(DEV)
        lb = torch.from_numpy(np.ascontiguousarray(lab[r0:r1])).to(DEV)
        out.append((r0, r1, split.PagePart(cube, lb, w.K, w.k)))
    return out


@pytest.mark.parametrize("n", [2, 3])
def test_split_page_is_bit_identical_to_the_whole_page(n):
    if DEV is None:
        pytest.skip("no CUDA device")
    w = make_workload(6200 + n, 23, 515, 389, 4, (6000, 5000, 4000, 3000), 3, separation=(1.0, 4.0), both=True)
    u_ref, lam_ref, V_ref, rng_ref, mom_ref = _whole(w, torch.from_numpy(w.cube).to(DEV),
                                                     torch.from_numpy(w.labels).to(DEV))
    parts = _parts(w, n)
    moms = []
    for _, _, p in parts:
        mom, st = p.moments()
        assert st == cva.CVA_OK
        moms.append(mom)
    total = torch.stack(moms).sum(dim=0)                      # the all-reduce
    np.testing.assert_array_equal(total.cpu().numpy(), mom_ref)
    rngs = []
    for _, _, p in parts:
        r, st = p.fit(total)
        assert st == cva.CVA_OK
        rngs.append(r)
    R = torch.stack(rngs)
    merged = split.merge_ranges(R[:, 0::2].amin(dim=0), R[:, 1::2].amax(dim=0))
    np.testing.assert_array_equal(merged.cpu().numpy(), rng_ref)
    for r0, r1, p in parts:
        lam, V, _, _ = cva.cva_model_get(p.model)
        np.testing.assert_array_equal(lam, lam_ref)
        np.testing.assert_array_equal(V[:, : w.k], V_ref[:, : w.k])
        out = torch.full((w.k, r1 - r0, w.W), 7, dtype=torch.uint8, device=DEV)
        p.project(merged, out)
        np.testing.assert_array_equal(out.cpu().numpy(), u_ref[:, r0:r1])
        p.close()


def test_a_part_with_a_bad_label_fails_the_page():
    """The parts' statuses are reduced by min before the moments are summed,
    so a label above K in one part fails every part."""
    if DEV is None:
        pytest.skip("no CUDA device")
    w = make_workload(6210, 12, 200, 160, 3, (1500, 1200, 900), 2, separation=(1.0, 4.0), both=False)
    bad = w.labels.copy()
    bad[150, 10] = 9   # in the second part
    parts = _parts(w, 2, labels=bad)
    sts = [p.moments()[1] for _, _, p in parts]
    assert sts[0] == cva.CVA_OK and sts[1] == cva.CVA_ERR_LABEL_RANGE
    assert min(sts) == cva.CVA_ERR_LABEL_RANGE
    for _, _, p in parts:
        p.close()
