"""The allocation-free entry point against the model-based one.

cva_fit_project_u8_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory budget, plug-ins that forbid device
allocations after start-up, loops that must stay out of the allocator); it
keeps its scratch in one array of the library's device data.  It runs the
same kernels on the same inputs as cva_fit + cva_project_u8 with the
training-score range, so its images and eigenvalues must be bit-identical to
theirs; the calls share the one array, so a call must not see anything of
the previous one: pages alternate here between two band counts, class
counts and training sets, and a call that fails (too many training pixels)
sits between two that succeed.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")

NOALLOC_MAX_TRAIN = 1 << 18


def _model_path(w, cube, labels):
    """cva_fit + cva_project_u8 (training-score range) on a model."""
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    ref = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=cube.device)
    cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, ref)
    lam, _, _, _ = cva.cva_model_get(m)
    m.close()
    return ref.cpu().numpy(), lam


class _Page:
    def __init__(self, w, dev):
        self.w = w
        self.cube = torch.from_numpy(w.cube).to(dev)
        self.labels = torch.from_numpy(w.labels).to(dev)
        self.out = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=dev)
        self.lam = torch.empty(w.B, dtype=torch.float64, device=dev)
        self.status = torch.empty(1, dtype=torch.int32, device=dev)

    def call(self):
        self.out.fill_(7)
        self.lam.fill_(-1.0)
        self.status.fill_(-99)
        cva.cva_fit_project_u8_noalloc(self.cube, self.labels, self.w.K, self.w.k, self.out,
                                       eigvals=self.lam, status=self.status)


def test_noalloc_matches_model_path_bit_for_bit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    wa = make_workload(301, 23, 384, 512, 4, (3000, 2500, 2000, 1500), 3, separation=(1.0, 4.0), both=True)
    wb = make_workload(302, 12, 257, 301, 3, (900, 1200, 700), 2, separation=(1.0, 4.0), both=False)
    pa, pb = _Page(wa, dev), _Page(wb, dev)
    refs = {id(pa): _model_path(wa, pa.cube, pa.labels), id(pb): _model_path(wb, pb.cube, pb.labels)}

    # a page with more training pixels than the array holds: refused on the
    # device (CVA_ERR_CAPACITY in status), its image left as it was
    wc = make_workload(303, 4, 768, 768, 2, (300000, 20000), 1, separation=(1.0, 4.0), both=False, cap_frac=0.9)
    assert sum(wc.n_train) > NOALLOC_MAX_TRAIN
    pc = _Page(wc, dev)
    torch.cuda.synchronize()

    # device memory is sampled once every page has been called once (by then
    # the driver has loaded the array and the kernels each page launches);
    # the comparisons run on host copies so that the test allocates nothing
    # on the device either
    mem = None
    for i, p in enumerate([pa, pb, pc, pa, pa, pb, pc, pa, pb, pb]):
        p.call()
        torch.cuda.synchronize()
        if i == 2:
            mem = torch.cuda.mem_get_info()[0]
        st = int(p.status.item())
        if p is pc:
            assert st == cva.CVA_ERR_CAPACITY, i
            assert (p.out.cpu().numpy() == 7).all(), i
            continue
        assert st == cva.CVA_OK, i
        u_ref, lam_ref = refs[id(p)]
        np.testing.assert_array_equal(p.out.cpu().numpy(), u_ref, err_msg=f"call {i}")
        np.testing.assert_array_equal(p.lam.cpu().numpy(), lam_ref, err_msg=f"call {i}")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == mem  # nothing allocated on the device since

    # and against the FP64 oracle, at the library's tolerances
    for p in (pa, pb):
        w = p.w
        ref = oracle.fit(w.cube, w.labels, w.K)
        r = w.K - 1
        lam = p.lam.cpu().numpy()
        assert (np.abs(lam[:r] - ref["lam"][:r]) / ref["lam"][:r]).max() <= 1e-6
        y = oracle.project(w.cube, ref["V"], ref["mu"], w.k)
        u_ref = oracle.to_u8(y, oracle.range_training(y, w.labels))
        d = np.abs(p.out.cpu().numpy().reshape(w.k, -1).astype(np.int32) - u_ref.astype(np.int32))
        assert (d <= 1).mean() >= 0.999


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    cube = torch.zeros((2, 4, 4), dtype=torch.uint16, device=dev)
    labels = torch.zeros((4, 4), dtype=torch.uint8, device=dev)
    out = torch.zeros((1, 4, 4), dtype=torch.uint8, device=dev)
    lib = cva.load()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 8193 x 8193 pixels is above the 2^26 limit: refused on the host, nothing launched
    rc = lib.cva_fit_project_u8_noalloc(ctypes.c_void_p(cube.data_ptr()), 2, 8193, 8193,
                                        ctypes.c_void_p(labels.data_ptr()), 2, 1,
                                        ctypes.c_void_p(out.data_ptr()), None, None, s)
    assert rc == cva.CVA_ERR_INVALID_ARG
    # the binding checks the output shapes before the call
    with pytest.raises(ValueError):
        cva.cva_fit_project_u8_noalloc(cube, labels, 2, 1, torch.zeros((2, 4, 4), dtype=torch.uint8, device=dev))
    with pytest.raises(ValueError):
        cva.cva_fit_project_u8_noalloc(cube, labels, 2, 1, out, eigvals=torch.zeros(1, dtype=torch.float64,
                                                                                     device=dev))
