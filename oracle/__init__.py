"""FP64 CPU oracle for Canonical Variates Analysis image enhancement.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code, header or table with the CUDA path.

The arithmetic lives in ``cva_oracle.c`` (plain scalar C, compiled here with
gcc on first use); this module only marshals numpy arrays into it.  Each
function cites the part of the paper it restates; the readings taken where
the paper is silent are listed at the top of ``cva_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cva_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None        # the library the functions below call (plain or threaded)
_libs = {}         # path -> loaded library

OK = 0
ERR_ARG = -1
ERR_EMPTY_CLASS = -2
ERR_NOT_SPD = -3
ERR_NO_CONVERGENCE = -4
ERR_LABEL = -7


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where} failed with code {code}")
        self.code = code


def build(force: bool = False, threaded: bool = False) -> str:
    """Compile ``cva_oracle.c`` into ``_build/liboracle.so`` (plain gcc -O2,
    no fast-math, no FMA contraction, so x86 and Arm round alike); with
    ``threaded``, the same source with -fopenmp into ``liboracle_omp.so``
    (identical results, used to time the oracle on every host core)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _OMP_PATH if threaded else _LIB_PATH
    stale = (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math"] + (["-fopenmp"] if threaded else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def use_threads(n: int) -> int:
    """Route the following oracle calls to the plain library (n <= 1) or to
    the OpenMP build with n threads; returns the threads in effect."""
    global _lib
    lib = _open(build(threaded=n > 1))
    with _lock:
        _lib = lib
    return int(lib.orc_threads(int(n) if n > 1 else 0))


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = _open(build())
    with _lock:
        if _lib is None:
            _lib = lib
        return _lib


def _open(path):
    with _lock:
        if path in _libs:
            return _libs[path]
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_class_sums.argtypes = [P, I64, I64, P, I64, P, P]
        lib.orc_scatter.argtypes = [P, I64, I64, P, I64, P, P, P, P, P]
        lib.orc_gen_eig.argtypes = [I64, P, P, P, P, P]
        lib.orc_project.argtypes = [P, I64, I64, I64, I64, P, I64, P, I64, P]
        lib.orc_range_global.argtypes = [P, I64, I64, P]
        lib.orc_range_training.argtypes = [P, I64, I64, P, P]
        lib.orc_to_u8.argtypes = [P, I64, I64, P, P]
        lib.orc_to_u16.argtypes = [P, I64, I64, P, P]
        lib.orc_to_u16.restype = None
        lib.orc_percentile_range.argtypes = [P, I64, I64, I64, P]
        lib.orc_pca_cov.argtypes = [P, I64, I64, P, P, P, P]
        lib.orc_cluster_indices.argtypes = [P, I64, I64, P, I64, P, P, P, P, P, P]
        lib.orc_cluster_indices.restype = ctypes.c_int
        lib.orc_pca_cov.restype = ctypes.c_int
        lib.orc_percentile_range.restype = ctypes.c_int
        for name in ("orc_class_sums", "orc_scatter", "orc_gen_eig", "orc_project"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("orc_range_global", "orc_range_training", "orc_to_u8"):
            getattr(lib, name).restype = None
        lib.orc_threads.argtypes = [ctypes.c_int]
        lib.orc_threads.restype = ctypes.c_int
        _libs[path] = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _planar(cube: np.ndarray):
    cube = np.ascontiguousarray(cube, dtype=np.uint16)
    B = cube.shape[0]
    return cube, B, int(np.prod(cube.shape[1:]))


def class_sums(cube: np.ndarray, labels: np.ndarray, K: int):
    """Counts ``n[c]`` and exact band sums ``s[c, b]`` of the training pixels
    of each class (Section 2: the points picked for each class)."""
    lib = _load()
    cube, B, P = _planar(cube)
    labels = np.ascontiguousarray(labels, dtype=np.uint8).reshape(-1)
    if labels.size != P:
        raise ValueError("labels must have one entry per pixel")
    n = np.zeros(K, np.int64)
    s = np.zeros((K, B), np.int64)
    rc = lib.orc_class_sums(_ptr(cube), B, P, _ptr(labels), K, _ptr(n), _ptr(s))
    if rc != OK:
        raise OracleError(rc, "class_sums")
    return n, s


def scatter(cube: np.ndarray, labels: np.ndarray, K: int) -> Dict[str, np.ndarray]:
    """Class means, total mean, within-class scatter Sw and between-class
    scatter Sb (Section 2: the covariance matrices within and between the
    classes), as unnormalised sums of squares and cross-products."""
    lib = _load()
    cube, B, P = _planar(cube)
    labels = np.ascontiguousarray(labels, dtype=np.uint8).reshape(-1)
    if labels.size != P:
        raise ValueError("labels must have one entry per pixel")
    n = np.zeros(K, np.int64)
    mu_c = np.zeros((K, B))
    mu = np.zeros(B)
    Sw = np.zeros((B, B))
    Sb = np.zeros((B, B))
    rc = lib.orc_scatter(_ptr(cube), B, P, _ptr(labels), K, _ptr(n), _ptr(mu_c), _ptr(mu), _ptr(Sw), _ptr(Sb))
    if rc != OK:
        raise OracleError(rc, "scatter")
    return {"n": n, "mu_c": mu_c, "mu": mu, "Sw": Sw, "Sb": Sb}


def gen_eig(Sw: np.ndarray, Sb: np.ndarray):
    """Solve Sb v = lambda Sw v (Section 4: the generalized symmetric-definite
    eigenproblem) by Cholesky reduction and cyclic Jacobi.  Returns
    (lambda descending, V with column j = vector j, Jacobi sweeps)."""
    lib = _load()
    Sw = np.ascontiguousarray(Sw, dtype=np.float64)
    Sb = np.ascontiguousarray(Sb, dtype=np.float64)
    B = Sw.shape[0]
    lam = np.zeros(B)
    V = np.zeros((B, B))
    sweeps = ctypes.c_int(0)
    rc = lib.orc_gen_eig(B, _ptr(Sw), _ptr(Sb), _ptr(lam), _ptr(V), ctypes.addressof(sweeps))
    if rc != OK:
        raise OracleError(rc, "gen_eig")
    return lam, V, int(sweeps.value)


def fit(cube: np.ndarray, labels: np.ndarray, K: int) -> Dict[str, np.ndarray]:
    """Scatter matrices followed by the eigenanalysis (Section 2)."""
    out = scatter(cube, labels, K)
    lam, V, sweeps = gen_eig(out["Sw"], out["Sb"])
    out.update({"lam": lam, "V": V, "sweeps": sweeps})
    return out


def project(cube: np.ndarray, V: np.ndarray, mu: np.ndarray, k: int,
            p0: int = 0, p1: Optional[int] = None) -> np.ndarray:
    """y_j = v_j^T (x - mu) for every pixel in [p0, p1) (Section 2: the
    coefficients multiplied with the band images).  Returns k x (p1 - p0)."""
    lib = _load()
    cube, B, P = _planar(cube)
    if p1 is None:
        p1 = P
    V = np.ascontiguousarray(V, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    y = np.zeros((k, p1 - p0))
    rc = lib.orc_project(_ptr(cube), B, P, p0, p1, _ptr(V), V.shape[1], _ptr(mu), k, _ptr(y))
    if rc != OK:
        raise OracleError(rc, "project")
    return y


def range_global(y: np.ndarray) -> np.ndarray:
    """(lo_j, hi_j) over every pixel: the first rescale of Section 2."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    k, P = y.shape
    r = np.zeros(2 * k)
    lib.orc_range_global(_ptr(y), k, P, _ptr(r))
    return r


def range_training(y: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """(lo_j, hi_j) over the training pixels: the second rescale of Section 2."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    k, P = y.shape
    labels = np.ascontiguousarray(labels, dtype=np.uint8).reshape(-1)
    r = np.zeros(2 * k)
    lib.orc_range_training(_ptr(y), k, P, _ptr(labels), _ptr(r))
    return r


def to_u8(y: np.ndarray, rng: np.ndarray) -> np.ndarray:
    """floor(255 (y - lo) / (hi - lo) + 1/2) clamped to 0..255 (Section 2)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    k, P = y.shape
    rng = np.ascontiguousarray(rng, dtype=np.float64)
    out = np.zeros((k, P), np.uint8)
    lib.orc_to_u8(_ptr(y), k, P, _ptr(rng), _ptr(out))
    return out


def to_u16(y: np.ndarray, rng: np.ndarray) -> np.ndarray:
    """floor(65535 (y - lo) / (hi - lo) + 1/2) clamped to 0..65535: the 16-bit
    image of the same rescale (Section 2's CVA-GSL tool writes 8- and 16-bit
    images)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    k, P = y.shape
    rng = np.ascontiguousarray(rng, dtype=np.float64)
    out = np.zeros((k, P), np.uint16)
    lib.orc_to_u16(_ptr(y), k, P, _ptr(rng), _ptr(out))
    return out


def percentile_basis_points(percent: float) -> int:
    """p percent as an integer number of 0.01 % steps (0 .. 4999)."""
    bp = int(round(percent * 100.0))
    if abs(bp - percent * 100.0) > 1e-6 or not 0 <= bp <= 4999:
        raise ValueError("percent must be a multiple of 0.01 in [0, 50)")
    return bp


def percentile_range(y: np.ndarray, percent: float) -> np.ndarray:
    """The third rescale of Section 2: (lo_j, hi_j) with `percent` of the
    pixels taken out of each tail -- m = floor(p P / 100) values at each end,
    lo the (m+1)-th smallest, hi the (m+1)-th largest.  Values are elements of
    y (float32 input gives float32-representable results)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    k, P = y.shape
    r = np.zeros(2 * k)
    rc = lib.orc_percentile_range(_ptr(y), k, P, percentile_basis_points(percent), _ptr(r))
    if rc != 0:
        raise OracleError(rc, "orc_percentile_range")
    return r


def pca(cube: np.ndarray, mask: Optional[np.ndarray] = None) -> Dict[str, np.ndarray]:
    """Principal components of the pixels selected by `mask` (all pixels when
    None): Section 2's PCA -- subtract the mean, form the covariance matrix
    (sample covariance, divided by N - 1), take its eigenvectors,
    orthonormal.  The eigenproblem is the same solver with Sw = I, so the
    order (descending) and the sign convention match the CVA vectors."""
    lib = _load()
    cube, B, P = _planar(cube)
    mp = None
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        if mask.size != P:
            raise ValueError("mask must have one entry per pixel")
        mp = _ptr(mask)
    mu = np.zeros(B)
    C = np.zeros((B, B))
    N = ctypes.c_int64(0)
    rc = lib.orc_pca_cov(_ptr(cube), B, P, mp, _ptr(mu), _ptr(C), ctypes.addressof(N))
    if rc != OK:
        raise OracleError(rc, "pca_cov")
    lam, V, sweeps = gen_eig(np.eye(B), C)
    return {"N": int(N.value), "mu": mu, "C": C, "lam": lam, "V": V, "sweeps": sweeps}


def cluster_indices(y: np.ndarray, labels: np.ndarray, K: int) -> Dict[str, np.ndarray]:
    """Section 3's cluster-separation indices of the labelled classes in a
    k-band image y (k x P): counts T, centroids A (K x k), scatters S (eq. 1),
    centroid distances M (eq. 2), Davies-Bouldin ratios R (eq. 3) and Dunn
    indices DI (eq. 5), the last three K x K."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    if y.ndim == 1:
        y = y[None, :]
    k, P = y.shape
    labels = np.ascontiguousarray(labels, dtype=np.uint8).reshape(-1)
    if labels.size != P:
        raise ValueError("labels must have one entry per pixel")
    T = np.zeros(K, np.int64)
    A = np.zeros((K, k))
    S = np.zeros(K)
    M = np.zeros((K, K))
    R = np.zeros((K, K))
    DI = np.zeros((K, K))
    rc = lib.orc_cluster_indices(_ptr(y), k, P, _ptr(labels), K, _ptr(T), _ptr(A), _ptr(S), _ptr(M), _ptr(R),
                                 _ptr(DI))
    if rc != OK:
        raise OracleError(rc, "cluster_indices")
    return {"T": T, "A": A, "S": S, "M": M, "R": R, "DI": DI}


def rgb_composite(planes: np.ndarray, src, invert=(False, False, False)) -> np.ndarray:
    """The colour image of Section 2 / Figure 5: three 8-bit images as the
    red, green and blue channels (planes[src[c]] for channel c, optionally
    inverted as 255 - v), interleaved H x W x 3."""
    planes = np.asarray(planes, dtype=np.uint8)
    k = planes.shape[0]
    out = np.zeros(planes.shape[1:] + (3,), np.uint8)
    for c in range(3):
        if not 0 <= src[c] < k:
            raise ValueError("channel source out of range")
        v = planes[src[c]]
        out[..., c] = (255 - v) if invert[c] else v
    return out
