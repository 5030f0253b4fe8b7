"""ctypes binding of the C ABI in include/cva.h.

Argument marshalling only: every computation runs in the CUDA kernels of
``libcva.so``.  Functions keep the C names; where the C call takes a device
pointer plus its sizes, the binding takes a CUDA tensor and reads the sizes
from its shape.  A missing library raises ImportError on first use; nothing
ever falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

from . import _build

CVA_OK = 0
CVA_ERR_INVALID_ARG = -1
CVA_ERR_EMPTY_CLASS = -2
CVA_ERR_NOT_SPD = -3
CVA_ERR_NO_CONVERGENCE = -4
CVA_ERR_TIMEOUT = -5
CVA_ERR_CUDA = -6
CVA_ERR_LABEL_RANGE = -7
CVA_ERR_NOT_FITTED = -8
CVA_ERR_CAPACITY = -9

CVA_RANGE_GLOBAL = 0
CVA_RANGE_TRAINING = 1
CVA_RANGE_GIVEN = 2

CVA_PRECISION_MIXED = 0
CVA_PRECISION_FP64 = 1

CVA_MAX_BANDS = 32
CVA_MAX_CLASSES = 16

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "cva_model_create": (_I, [_I, _I, ctypes.POINTER(_P)]),
    "cva_model_destroy": (None, [_P]),
    "cva_model_reserve": (_I, [_P, ctypes.c_int64]),
    "cva_set_precision": (_I, [_P, _I]),
    "cva_set_variates": (_I, [_P, _I]),
    "cva_fit": (_I, [_P, _I, _I, _I, _P, _I, _P, _P]),
    "cva_fit_moments": (_I, [_P, _I, _I, _I, _P, _I, _P, _P]),
    "cva_model_moments": (_I, [_P, _P, _P]),
    "cva_fit_from_moments": (_I, [_P, _P, _P]),
    "cva_model_training_range": (_I, [_P, _P, _P]),
    "cva_set_training_range": (_I, [_P, _P, _P]),
    "cva_status": (_I, [_P, _P]),
    "cva_model_get": (_I, [_P, _P, _P, _P, _P, _P]),
    "cva_model_get_scatter": (_I, [_P, _P, _P, _P, _P, _P]),
    "cva_project": (_I, [_P, _I, _I, _I, _P, _I, _P, _P, _P]),
    "cva_to_u8": (_I, [_P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "cva_project_u8": (_I, [_P, _I, _I, _I, _P, _I, _I, _P, _P, _P]),
    "cva_pca_fit": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "cva_cluster_indices": (_I, [_P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cva_rgb_composite": (_I, [_P, _I, _I, _I, _P, _I, _P, _P]),
    "cva_percentile_range": (_I, [_P, _I, _I, _I, ctypes.c_double, _P, _P, _P]),
    "cva_to_u16": (_I, [_P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "cva_fit_project_u8_noalloc": (_I, [_P, _I, _I, _I, _P, _I, _I, _P, _P, _P, _P]),
    "cva_batch_create": (_I, [_I, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)]),
    "cva_batch_destroy": (None, [_P]),
    "cva_fit_project_batched": (_I, [_P, _P, _I, _P]),
    "cva_batch_status": (_I, [_P, _I, _P, _P]),
    "cva_project_batched": (_I, [_P, _P, _I, _P]),
    "cva_fit_batched": (_I, [_P, _P, _I, _P]),
    "cva_batch_tune": (_I, [_P, _P, _I, _P, _P]),
    "cva_strerror": (ctypes.c_char_p, [_I]),
}

_lib = None


class CvaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {cva_strerror(code)} ({code})")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcva.so (building it first if it is missing or stale and
    ``build_if_missing`` is set)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run paper_1612_06457_gb300.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str) -> None:
    if code != CVA_OK:
        raise CvaError(code, where)


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: Optional[torch.Tensor], dtype: torch.dtype, name: str):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def cva_strerror(code: int) -> str:
    return load().cva_strerror(code).decode()


class Model:
    """Owner of one ``cva_model`` handle."""

    def __init__(self, B: int, K: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.cva_model_create(B, K, ctypes.byref(h)), "cva_model_create")
        self.handle = h
        self.B = B
        self.K = K
        self.nvec = B

    def close(self) -> None:
        if self.handle:
            load().cva_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cva_model_create(B: int, K: int) -> Model:
    return Model(B, K)


def cva_model_destroy(m: Model) -> None:
    m.close()


def cva_model_reserve(m: Model, max_train: int) -> None:
    _check(load().cva_model_reserve(m.handle, max_train), "cva_model_reserve")


def cva_set_precision(m: Model, mode: int) -> None:
    _check(load().cva_set_precision(m.handle, mode), "cva_set_precision")


def cva_set_variates(m: Model, nvec: int) -> None:
    _check(load().cva_set_variates(m.handle, nvec), "cva_set_variates")
    m.nvec = nvec


def cva_fit(cube: torch.Tensor, labels: torch.Tensor, K: int, m: Model, stream=None) -> None:
    B, H, W = cube.shape
    if tuple(labels.shape) != (H, W):
        raise ValueError("labels must be H x W")
    rc = load().cva_fit(_dptr(cube, torch.uint16, "cube"), B, H, W, _dptr(labels, torch.uint8, "labels"),
                        K, m.handle, _stream_ptr(stream))
    _check(rc, "cva_fit")


def moment_words(B: int, K: int) -> int:
    """Words of a class-moment array (CVA_MOMENT_WORDS in cva.h)."""
    return K * (B + 1) * (B + 2) // 2


def cva_fit_moments(cube: torch.Tensor, labels: torch.Tensor, K: int, m: Model, stream=None) -> None:
    B, H, W = cube.shape
    if tuple(labels.shape) != (H, W):
        raise ValueError("labels must be H x W")
    rc = load().cva_fit_moments(_dptr(cube, torch.uint16, "cube"), B, H, W, _dptr(labels, torch.uint8, "labels"),
                                K, m.handle, _stream_ptr(stream))
    _check(rc, "cva_fit_moments")


def cva_model_moments(m: Model, moments: torch.Tensor, stream=None) -> None:
    """Copy the model's class moments into ``moments`` (int64, moment_words(B, K), device)."""
    if moments.numel() < moment_words(m.B, m.K):
        raise ValueError("moments must hold moment_words(B, K) int64")
    _check(load().cva_model_moments(m.handle, _dptr(moments, torch.int64, "moments"), _stream_ptr(stream)),
           "cva_model_moments")


def cva_fit_from_moments(m: Model, moments: torch.Tensor, stream=None) -> None:
    if moments.numel() < moment_words(m.B, m.K):
        raise ValueError("moments must hold moment_words(B, K) int64")
    _check(load().cva_fit_from_moments(m.handle, _dptr(moments, torch.int64, "moments"), _stream_ptr(stream)),
           "cva_fit_from_moments")


def cva_model_training_range(m: Model, range: torch.Tensor, stream=None) -> None:
    if range.numel() < 2 * m.nvec:
        raise ValueError("range must hold 2 nvec float32")
    _check(load().cva_model_training_range(m.handle, _dptr(range, torch.float32, "range"), _stream_ptr(stream)),
           "cva_model_training_range")


def cva_set_training_range(m: Model, range: torch.Tensor, stream=None) -> None:
    if range.numel() < 2 * m.nvec:
        raise ValueError("range must hold 2 nvec float32")
    _check(load().cva_set_training_range(m.handle, _dptr(range, torch.float32, "range"), _stream_ptr(stream)),
           "cva_set_training_range")


def cva_status(m: Model, stream=None) -> int:
    return load().cva_status(m.handle, _stream_ptr(stream))


def cva_model_get(m: Model, stream=None):
    """Returns (eigvals [B], V [B, B], mean [B], train_range [2B]) as numpy."""
    import numpy as np

    B = m.B
    lam = np.zeros(B)
    V = np.zeros((B, B))
    mean = np.zeros(B)
    rng = np.zeros(2 * B, np.float32)
    _check(load().cva_model_get(m.handle, _hptr(lam), _hptr(V), _hptr(mean), _hptr(rng), _stream_ptr(stream)),
           "cva_model_get")
    return lam, V, mean, rng


def cva_model_get_scatter(m: Model, stream=None):
    """Returns (counts [K], class_means [K, B], Sw [B, B], Sb [B, B]) as numpy."""
    import numpy as np

    B, K = m.B, m.K
    n = np.zeros(K, np.int64)
    mc = np.zeros((K, B))
    Sw = np.zeros((B, B))
    Sb = np.zeros((B, B))
    _check(load().cva_model_get_scatter(m.handle, _hptr(n), _hptr(mc), _hptr(Sw), _hptr(Sb), _stream_ptr(stream)),
           "cva_model_get_scatter")
    return n, mc, Sw, Sb


def cva_project(cube: torch.Tensor, m: Model, k: int, out_f32: Optional[torch.Tensor] = None,
                range_out: Optional[torch.Tensor] = None, stream=None) -> None:
    B, H, W = cube.shape
    rc = load().cva_project(_dptr(cube, torch.uint16, "cube"), B, H, W, m.handle, k,
                            _dptr(out_f32, torch.float32, "out_f32"), _dptr(range_out, torch.float32, "range_out"),
                            _stream_ptr(stream))
    _check(rc, "cva_project")


def cva_to_u8(proj: torch.Tensor, mode: int, out: torch.Tensor, m: Optional[Model] = None,
              range: Optional[torch.Tensor] = None, stream=None) -> None:
    k, H, W = proj.shape
    rc = load().cva_to_u8(_dptr(proj, torch.float32, "proj"), k, H, W, mode, _dptr(range, torch.float32, "range"),
                          m.handle if m is not None else None, _dptr(out, torch.uint8, "out"), _stream_ptr(stream))
    _check(rc, "cva_to_u8")


def cva_project_u8(cube: torch.Tensor, m: Model, k: int, mode: int, out: torch.Tensor,
                   range: Optional[torch.Tensor] = None, stream=None) -> None:
    B, H, W = cube.shape
    rc = load().cva_project_u8(_dptr(cube, torch.uint16, "cube"), B, H, W, m.handle, k, mode,
                               _dptr(range, torch.float32, "range"), _dptr(out, torch.uint8, "out"),
                               _stream_ptr(stream))
    _check(rc, "cva_project_u8")


def cva_fit_project_u8_noalloc(cube: torch.Tensor, labels: torch.Tensor, K: int, k: int, out: torch.Tensor,
                               eigvals: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
                               stream=None) -> None:
    """Fit and fused 8-bit projection without device allocations (see cva.h).
    ``eigvals`` (float64, B) and ``status`` (int32, 1) are optional device
    outputs."""
    B, H, W = cube.shape
    if tuple(labels.shape) != (H, W):
        raise ValueError("labels must be H x W")
    if tuple(out.shape) != (k, H, W):
        raise ValueError("out must be k x H x W")
    if eigvals is not None and eigvals.numel() < B:
        raise ValueError("eigvals must hold B doubles")
    if status is not None and status.numel() < 1:
        raise ValueError("status must hold one int")
    rc = load().cva_fit_project_u8_noalloc(_dptr(cube, torch.uint16, "cube"), B, H, W,
                                           _dptr(labels, torch.uint8, "labels"), K, k,
                                           _dptr(out, torch.uint8, "out"),
                                           _dptr(eigvals, torch.float64, "eigvals"),
                                           _dptr(status, torch.int32, "status"), _stream_ptr(stream))
    _check(rc, "cva_fit_project_u8_noalloc")


CVA_MAX_BATCH_PAGES = 4096
CVA_MAX_BATCH_VARIATES = 8


class cva_page(ctypes.Structure):
    """One page of a batch (layout of ``cva_page`` in cva.h)."""
    _fields_ = [("cube", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("eigvals", ctypes.c_void_p), ("B", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("K", ctypes.c_int), ("k", ctypes.c_int)]


class Batch:
    """Owner of one ``cva_batch`` workspace."""

    def __init__(self, max_pages: int, max_pixels: int, max_train: int):
        h = ctypes.c_void_p()
        _check(load().cva_batch_create(max_pages, max_pixels, max_train, ctypes.byref(h)), "cva_batch_create")
        self.handle = h
        self.max_pages = max_pages

    def close(self) -> None:
        if self.handle:
            load().cva_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cva_batch_create(max_pages: int, max_pixels: int, max_train: int) -> Batch:
    return Batch(max_pages, max_pixels, max_train)


def cva_batch_destroy(b: Batch) -> None:
    b.close()


def _pages(items):
    """(cube, labels, K, k, out[, eigvals]) tuples -> ctypes array of cva_page."""
    arr = (cva_page * len(items))()
    for i, it in enumerate(items):
        cube, labels, K, k, out = it[:5]
        eig = it[5] if len(it) > 5 else None
        B, H, W = cube.shape
        if tuple(labels.shape) != (H, W) or tuple(out.shape) != (k, H, W):
            raise ValueError(f"page {i}: labels must be H x W and out k x H x W")
        arr[i] = cva_page(_dptr(cube, torch.uint16, "cube"), _dptr(labels, torch.uint8, "labels"),
                          _dptr(out, torch.uint8, "out"), _dptr(eig, torch.float64, "eigvals"), B, H, W, K, k)
    return arr


def cva_fit_project_batched(b: Batch, pages, stream=None) -> None:
    """Fit + fused 8-bit projection (training-score range) of every page.
    ``pages``: sequence of (cube, labels, K, k, out[, eigvals]) device tensors."""
    arr = _pages(pages)
    _check(load().cva_fit_project_batched(b.handle, arr, len(pages), _stream_ptr(stream)), "cva_fit_project_batched")


def cva_fit_batched(b: Batch, pages, stream=None) -> None:
    """Every page's fit alone (no projection); cva_project_batched projects."""
    arr = _pages(pages)
    _check(load().cva_fit_batched(b.handle, arr, len(pages), _stream_ptr(stream)), "cva_fit_batched")


def cva_project_batched(b: Batch, pages, stream=None) -> None:
    """The projection pass alone, with the models of the last batch on ``b``."""
    arr = _pages(pages)
    _check(load().cva_project_batched(b.handle, arr, len(pages), _stream_ptr(stream)), "cva_project_batched")


def cva_batch_status(b: Batch, n: int, stream=None):
    """Per-page status codes of the last batch (numpy int32 array)."""
    import numpy as np

    st = np.zeros(n, np.int32)
    load().cva_batch_status(b.handle, n, ctypes.c_void_p(st.ctypes.data), _stream_ptr(stream))
    return st


def cva_batch_tune(b: Batch, pages, stream=None):
    """Autotune the batched projection on ``pages``; returns (groups per item, CTAs per SM)."""
    arr = _pages(pages)
    chosen = (ctypes.c_int * 2)()
    _check(load().cva_batch_tune(b.handle, arr, len(pages), _stream_ptr(stream), chosen), "cva_batch_tune")
    return int(chosen[0]), int(chosen[1])


def cva_percentile_range(proj: torch.Tensor, percent: float, m: Model, range_out: torch.Tensor, stream=None) -> None:
    """(lo, hi) of each projection with ``percent`` of the pixels taken out of
    each tail (see cva.h) into the device float32 tensor ``range_out`` (2 k)."""
    k, H, W = proj.shape
    _check(load().cva_percentile_range(_dptr(proj, torch.float32, "proj"), k, H, W, float(percent), m.handle,
                                       _dptr(range_out, torch.float32, "range_out"), _stream_ptr(stream)),
           "cva_percentile_range")


def cva_to_u16(proj: torch.Tensor, mode: int, out: torch.Tensor, m: Optional[Model] = None,
               range: Optional[torch.Tensor] = None, stream=None) -> None:
    """16-bit image of the linear rescale (see cva.h)."""
    k, H, W = proj.shape
    _check(load().cva_to_u16(_dptr(proj, torch.float32, "proj"), k, H, W, mode,
                             _dptr(range, torch.float32, "range"), m.handle if m is not None else None,
                             _dptr(out, torch.uint16, "out"), _stream_ptr(stream)), "cva_to_u16")


def cva_pca_fit(cube: torch.Tensor, m: Model, mask: Optional[torch.Tensor] = None, stream=None) -> None:
    """Principal components of the page (or of the masked pixels) into ``m``."""
    B, H, W = cube.shape
    if mask is not None and tuple(mask.shape) != (H, W):
        raise ValueError("mask must be H x W")
    _check(load().cva_pca_fit(_dptr(cube, torch.uint16, "cube"), B, H, W, _dptr(mask, torch.uint8, "mask"),
                              m.handle, _stream_ptr(stream)), "cva_pca_fit")


CVA_IMAGE_U8 = 0
CVA_IMAGE_F32 = 1


def cva_cluster_indices(image: torch.Tensor, labels: torch.Tensor, K: int, m: Model, stream=None):
    """Section 3's indices of the labelled classes in ``image`` (k x H x W,
    uint8 or float32).  Returns a dict of numpy arrays T, A, S, M, R, DI."""
    import numpy as np

    k, H, W = image.shape
    if image.dtype == torch.uint8:
        dtype, ptr = CVA_IMAGE_U8, _dptr(image, torch.uint8, "image")
    else:
        dtype, ptr = CVA_IMAGE_F32, _dptr(image, torch.float32, "image")
    T = np.zeros(K, np.int64)
    A = np.zeros((K, k))
    S = np.zeros(K)
    M = np.zeros((K, K))
    R = np.zeros((K, K))
    DI = np.zeros((K, K))
    _check(load().cva_cluster_indices(ptr, dtype, k, H, W, _dptr(labels, torch.uint8, "labels"), K, m.handle,
                                      _hptr(T), _hptr(A), _hptr(S), _hptr(M), _hptr(R), _hptr(DI),
                                      _stream_ptr(stream)), "cva_cluster_indices")
    return {"T": T, "A": A, "S": S, "M": M, "R": R, "DI": DI}


def cva_rgb_composite(planes: torch.Tensor, src, out: torch.Tensor, invert=(False, False, False), stream=None) -> None:
    """Interleaved H x W x 3 colour image from planes[src[0..2]] (see cva.h)."""
    k, H, W = planes.shape
    s3 = (ctypes.c_int * 3)(*[int(x) for x in src])
    inv = sum(1 << c for c in range(3) if invert[c])
    _check(load().cva_rgb_composite(_dptr(planes, torch.uint8, "planes"), k, H, W, s3, inv,
                                    _dptr(out, torch.uint8, "out"), _stream_ptr(stream)), "cva_rgb_composite")
