"""The allocation-free entry point against the model-based one.

cva_fit_project_u8_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory budget, plug-ins that forbid device
allocations after start-up, loops that must stay out of the allocator); it
keeps its scratch in one array of the library's device data.  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from synth import make_workload

pytestmark = pytest.mark.gpu

cva = pytest.importorskip("paper_1612_06457_gb300")


def test_noalloc_matches_model_path_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    w = make_workload(301, 23, 384, 512, 4, (3000, 2500, 2000, 1500), 3, separation=(1.0, 4.0), both=True)
    cube = torch.from_numpy(w.cube).to(dev)
    labels = torch.from_numpy(w.labels).to(dev)

    # the existing entry points: a model, cva_fit, cva_project_u8
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    cva.cva_fit(cube, labels, w.K, m)
    ref = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=dev)
    cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, ref)
    lam_ref, _, _, _ = cva.cva_model_get(m)
    m.close()
    ref = ref.cpu().numpy()

    r = w.K - 1
    for _ in range(2):
        out = torch.full((w.k, w.H, w.W), 7, dtype=torch.uint8, device=dev)
        lam = torch.zeros(w.B, dtype=torch.float64, device=dev)
        status = torch.full((1,), -99, dtype=torch.int32, device=dev)
        cva.cva_fit_project_u8_noalloc(cube, labels, w.K, w.k, out, eigvals=lam, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == cva.CVA_OK
        got = out.cpu().numpy()
        close = np.abs(got.astype(np.int32) - ref.astype(np.int32)) <= 1
        assert close.mean() >= 0.999
        lam = lam.cpu().numpy()
        np.testing.assert_allclose(lam[:r], lam_ref[:r], rtol=1e-6)


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
