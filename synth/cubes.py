"""Seeded synthetic stand-ins for multispectral manuscript cubes.

The paper's images (the Galen palimpsest folios and John Rylands Latin MS 18,
Section 2 and Section 4) are not available, so every input here is drawn from
a fixed recipe with a numpy PCG64 generator:

* the cube is ``B x H x W`` uint16 (band-sequential, 12-bit values), band 0
  being the shortest wavelength (UV) and band B-1 the longest (IR), like the
  23 LED bands of Section 2;
* every pixel belongs to one ground-truth class: class 0 is parchment (the
  background), class 1 overtext ink, class 2 undertext ink, class 3 the
  overlap of both ("Class Both" of Section 2) and classes 4.. further stroke
  classes (the "Class Outside"-style extras the paper allows);
* each class is Gaussian in band space with a smooth mean spectrum and a
  random SPD covariance that shares a rank-1 "illumination" term;
* overtext and undertext are random quadratic Bezier strokes 2-6 px wide;
* training labels are taken from random axis-aligned rectangles (8-64 px a
  side) placed on pixels of the class, pixels of that class inside a rectangle
  being taken in raster order until the class has its requested count.

The label map uses 0 for "not a training pixel" and c+1 for class c.

Nothing in this module computes any part of Canonical Variates Analysis.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

_MAX_DN = 4095  # 12-bit sensor values stored in uint16


@dataclasses.dataclass
class Workload:
    """One synthetic cube with its label map and the projection width ``k``."""

    name: str
    cube: np.ndarray  # (B, H, W) uint16, band-sequential
    labels: np.ndarray  # (H, W) uint8, 0 = unlabelled, c + 1 = class c
    classmap: np.ndarray  # (H, W) uint8 ground-truth class of every pixel
    K: int
    k: int
    n_train: Tuple[int, ...]
    seed: int
    means: np.ndarray  # (K, B) population mean spectra (DN)
    covs: np.ndarray  # (K, B, B) population covariances (DN^2)

    @property
    def B(self) -> int:
        return int(self.cube.shape[0])

    @property
    def H(self) -> int:
        return int(self.cube.shape[1])

    @property
    def W(self) -> int:
        return int(self.cube.shape[2])

    @property
    def P(self) -> int:
        return self.H * self.W


# ----------------------------------------------------------------------------
# class spectra and covariances
# ----------------------------------------------------------------------------

def _bumps(rng: np.random.Generator, B: int, n: int, amp: Tuple[float, float]) -> np.ndarray:
    """Sum of ``n`` Gaussian bumps over the band index (sigma 2-5 bands)."""
    b = np.arange(B, dtype=np.float64)
    out = np.zeros(B)
    for _ in range(n):
        centre = rng.uniform(0, B - 1)
        sigma = rng.uniform(2.0, 5.0)
        a = rng.uniform(*amp) * rng.choice([-1.0, 1.0])
        out += a * np.exp(-0.5 * ((b - centre) / sigma) ** 2)
    return out


def _mean_spectra(rng: np.random.Generator, B: int, K: int) -> np.ndarray:
    """Smooth mean spectra: bright parchment rising to the IR, darker inks."""
    t = np.arange(B, dtype=np.float64) / max(B - 1, 1)  # 0 = UV, 1 = IR
    means = np.zeros((K, B))
    base = rng.uniform(2500.0, 2900.0)
    rise = rng.uniform(300.0, 700.0)
    parch = base + rise * t + _bumps(rng, B, 3, (30.0, 120.0))
    means[0] = parch
    for c in range(1, K):
        if c == 1:  # overtext: dark iron-gall-like ink, fading toward the IR
            lvl = rng.uniform(600.0, 1200.0)
            m = lvl + (parch - lvl) * 0.35 * t ** 2 + _bumps(rng, B, 3, (30.0, 150.0))
        elif c == 2:  # undertext: differs from parchment mostly in UV / blue
            depth = rng.uniform(900.0, 1400.0)
            tau = rng.uniform(0.15, 0.35)
            m = parch - depth * np.exp(-t / tau) - 150.0 + _bumps(rng, B, 3, (30.0, 100.0))
        elif c == 3:  # both inks on top of each other: darker than overtext
            m = 0.5 * (means[1] + means[2]) - rng.uniform(150.0, 400.0) + _bumps(rng, B, 3, (20.0, 80.0))
        else:  # further stroke classes (stains, rubrics, margins)
            lvl = rng.uniform(1000.0, 2000.0)
            m = lvl + rng.uniform(-300.0, 300.0) * t + _bumps(rng, B, 3, (50.0, 200.0))
        means[c] = m
    return np.clip(means, 200.0, 3900.0)


def _haar_orthogonal(rng: np.random.Generator, B: int) -> np.ndarray:
    z = rng.standard_normal((B, B))
    q, r = np.linalg.qr(z)
    return q * np.sign(np.diag(r))[None, :]


def _covariances(rng: np.random.Generator, B: int, K: int) -> np.ndarray:
    """Random SPD covariances Q diag(s^2) Q^T + 40^2 11^T, stds s in [8, 60]."""
    ones = np.ones((B, 1))
    covs = np.zeros((K, B, B))
    for c in range(K):
        q = _haar_orthogonal(rng, B)
        s = np.exp(rng.uniform(math.log(8.0), math.log(60.0), size=B))
        cov = (q * s ** 2) @ q.T + 40.0 ** 2 * (ones @ ones.T)
        covs[c] = 0.5 * (cov + cov.T)
    return covs


def _set_separation(rng: np.random.Generator, means: np.ndarray, covs: np.ndarray,
                    sep: Tuple[float, float]) -> np.ndarray:
    """Pull every class mean toward the parchment mean so that its Mahalanobis
    distance (pooled population covariance) to parchment is uniform in ``sep``:
    classes then overlap partially instead of being trivially separable."""
    pooled = covs.mean(axis=0)
    chol = np.linalg.cholesky(pooled)
    out = means.copy()
    for c in range(1, means.shape[0]):
        d = means[c] - means[0]
        z = np.linalg.solve(chol, d)
        dist = float(np.sqrt(z @ z))
        target = rng.uniform(*sep)
        out[c] = means[0] + d * (target / dist)
    return out


# ----------------------------------------------------------------------------
# class layout: strokes on a parchment background
# ----------------------------------------------------------------------------

def _stroke_mask(rng: np.random.Generator, H: int, W: int, frac: float) -> np.ndarray:
    """Random quadratic Bezier strokes, 2-6 px wide, until ``frac`` of the
    page is covered."""
    mask = np.zeros((H, W), dtype=bool)
    target = frac * H * W
    if target <= 0:
        return mask
    scale = max(8.0, min(H, W) / 8.0)
    discs = {}
    while mask.sum() < target:
        for _ in range(64):
            p0 = np.array([rng.uniform(0, H), rng.uniform(0, W)])
            p1 = p0 + rng.normal(0.0, scale * 0.5, size=2)
            p2 = p0 + rng.normal(0.0, scale * 0.7, size=2)
            length = np.linalg.norm(p1 - p0) + np.linalg.norm(p2 - p1) + 1.0
            t = np.linspace(0.0, 1.0, int(2 * length) + 2)[:, None]
            pts = (1 - t) ** 2 * p0 + 2 * (1 - t) * t * p1 + t ** 2 * p2
            width = int(rng.integers(2, 7))
            if width not in discs:
                r = width / 2.0
                rr = int(math.ceil(r))
                dy, dx = np.mgrid[-rr:rr + 1, -rr:rr + 1]
                keep = (dy + 0.5) ** 2 + (dx + 0.5) ** 2 <= r * r + 0.5
                discs[width] = (dy[keep].ravel(), dx[keep].ravel())
            dy, dx = discs[width]
            ys = np.rint(pts[:, 0])[:, None].astype(np.int64) + dy[None, :]
            xs = np.rint(pts[:, 1])[:, None].astype(np.int64) + dx[None, :]
            ok = (ys >= 0) & (ys < H) & (xs >= 0) & (xs < W)
            mask[ys[ok], xs[ok]] = True
    return mask


def _class_map(rng: np.random.Generator, H: int, W: int, K: int, both: bool) -> np.ndarray:
    """Parchment background, overtext (~8 %) and undertext (~6 %) strokes, the
    overlap as "both" when ``both`` is set, further classes as ~2 % strokes."""
    cmap = np.zeros((H, W), dtype=np.uint8)
    if K == 1:
        return cmap
    over = _stroke_mask(rng, H, W, 0.08)
    under = _stroke_mask(rng, H, W, 0.06) if K >= 3 else np.zeros_like(over)
    cmap[under] = 2
    cmap[over] = 1
    if both and K >= 4:
        cmap[over & under] = 3
    first_extra = 4 if (both and K >= 4) else 3
    for c in range(first_extra, K):
        cmap[_stroke_mask(rng, H, W, 0.02)] = c
    return cmap


# ----------------------------------------------------------------------------
# pixels and training labels
# ----------------------------------------------------------------------------

def _draw_pixels(rng: np.random.Generator, cmap: np.ndarray, means: np.ndarray,
                 covs: np.ndarray, chunk: int = 1 << 20, max_dn: int = _MAX_DN) -> np.ndarray:
    """Gaussian pixels per class, rounded and clipped to 0..max_dn (12 bits
    by default), planar.

    Pixels are drawn in raster-order chunks: one standard normal vector per
    pixel, coloured by the Cholesky factor of its class covariance."""
    K, B = means.shape
    H, W = cmap.shape
    P = H * W
    cube = np.empty((B, P), dtype=np.uint16)
    flat = cmap.ravel()
    chols = [np.linalg.cholesky(covs[c]).astype(np.float32) for c in range(K)]
    mus = [means[c].astype(np.float32)[:, None] for c in range(K)]
    for s in range(0, P, chunk):
        e = min(P, s + chunk)
        z = rng.standard_normal((B, e - s), dtype=np.float32)
        x = chols[0] @ z
        x += mus[0]
        cls = flat[s:e]
        for c in range(1, K):
            idx = np.flatnonzero(cls == c)
            if idx.size:
                x[:, idx] = chols[c] @ z[:, idx] + mus[c]
        np.rint(x, out=x)
        np.clip(x, 0, max_dn, out=x)
        cube[:, s:e] = x
    return cube.reshape(B, H, W)


def _training_labels(rng: np.random.Generator, cmap: np.ndarray, n_train: Sequence[int],
                     cap_frac: float) -> Tuple[np.ndarray, Tuple[int, ...]]:
    """Drop 8-64 px rectangles on pixels of each class; inside a rectangle the
    still-unlabelled pixels of that class are taken in raster order."""
    H, W = cmap.shape
    labels = np.zeros((H, W), dtype=np.uint8)
    counts = np.bincount(cmap.ravel(), minlength=len(n_train))
    got_all = []
    for c, want in enumerate(n_train):
        need = int(min(want, math.floor(cap_frac * counts[c])))
        got = 0
        rounds = 0
        while got < need:
            rounds += 1
            ys = rng.integers(0, H, size=4096)
            xs = rng.integers(0, W, size=4096)
            hit = cmap[ys, xs] == c
            for y, x in zip(ys[hit], xs[hit]):
                h = int(rng.integers(8, 65))
                w = int(rng.integers(8, 65))
                h = min(h, H)
                w = min(w, W)
                y0 = min(max(int(y) - h // 2, 0), H - h)
                x0 = min(max(int(x) - w // 2, 0), W - w)
                sub_c = cmap[y0:y0 + h, x0:x0 + w]
                sub_l = labels[y0:y0 + h, x0:x0 + w]
                flat = np.flatnonzero((sub_c == c) & (sub_l == 0))[: need - got]
                if flat.size:
                    ry, rx = np.divmod(flat, w)
                    labels[y0 + ry, x0 + rx] = c + 1
                    got += int(flat.size)
                if got >= need:
                    break
            if rounds > 4000 and got < need:
                # rectangles stopped finding pixels: take the rest in raster order
                rest = np.flatnonzero((cmap.ravel() == c) & (labels.ravel() == 0))[: need - got]
                labels.ravel()[rest] = c + 1
                got += int(rest.size)
        got_all.append(got)
    return labels, tuple(got_all)


def make_workload(seed: int, B: int, H: int, W: int, K: int, n_train: Sequence[int], k: int,
                  separation: Optional[Tuple[float, float]] = None, both: bool = True,
                  cap_frac: float = 0.8, name: str = "custom", means: Optional[np.ndarray] = None,
                  covs: Optional[np.ndarray] = None, max_dn: int = _MAX_DN) -> Workload:
    """Draw one cube, its class map and its training label map.  ``means``
    (K x B) and ``covs`` (K x B x B), when given, replace the drawn class
    spectra and covariances (and ``separation`` is not applied); ``max_dn``
    is the largest pixel value (4095: 12-bit data)."""
    if len(n_train) != K:
        raise ValueError("n_train must give one count per class")
    rng = np.random.Generator(np.random.PCG64(seed))
    if means is None or covs is None:
        means = _mean_spectra(rng, B, K)
        covs = _covariances(rng, B, K)
        if separation is not None:
            means = _set_separation(rng, means, covs, separation)
    cmap = _class_map(rng, H, W, K, both)
    cube = _draw_pixels(rng, cmap, means, covs, max_dn=max_dn)
    labels, got = _training_labels(rng, cmap, n_train, cap_frac)
    return Workload(name=name, cube=cube, labels=labels, classmap=cmap, K=K, k=k,
                    n_train=got, seed=seed, means=means, covs=covs)


# ----------------------------------------------------------------------------
# the named workloads (shapes of the paper's manuscripts, Section 2)
# ----------------------------------------------------------------------------

#: name -> (seed, B, H, W, K, n_train, k, separation, both)
WORKLOADS = {
    # 16 bands, 512 x 512, parchment / overtext / undertext, 2000 px a class
    "cube16b_512x512_K3": (1000, 16, 512, 512, 3, (2000, 2000, 2000), 2, None, False),
    # 23 bands, 4096 x 4096, 4 partially overlapping classes, 50 000 px a class
    "cube23b_4096x4096_K4": (1001, 23, 4096, 4096, 4, (50000,) * 4, 3, (1.0, 4.0), True),
    # 23 bands, 8192 wide x 6144 high, 6 classes with heavy-tailed sizes
    "cube23b_8192x6144_K6": (1004, 23, 6144, 8192, 6,
                             (1000000, 300000, 100000, 30000, 12000, 5000), 5, (1.0, 4.0), True),
}


def named_workload(name: str) -> Workload:
    seed, B, H, W, K, n_train, k, sep, both = WORKLOADS[name]
    return make_workload(seed, B, H, W, K, n_train, k, separation=sep, both=both, name=name)


def _batch_page(i: int, seed0: int, sizes: Optional[List[int]]) -> Workload:
    """Page i of a batch (its own generators, so pages can be drawn in any
    order or in parallel)."""
    side_choices = sizes if sizes is not None else list(range(512, 3073, 128))
    rng = np.random.Generator(np.random.PCG64(seed0 + i))
    H = int(rng.choice(side_choices))
    W = int(rng.choice(side_choices))
    B = int(rng.integers(12, 24))
    K = int(rng.integers(2, 7))
    n_train = tuple(int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5))))) for _ in range(K))
    return make_workload(seed0 + 1000 + i, B, H, W, K, n_train, K - 1,
                         separation=(1.0, 4.0), both=True, cap_frac=0.5,
                         name=f"batch{i:02d}_{B}b_{H}x{W}_K{K}")


def _batch_page_args(a):
    return _batch_page(*a)


def batch_workloads(count: int = 64, seed0: int = 100300, sizes: Optional[List[int]] = None,
                    workers: int = 0) -> List[Workload]:
    """Uneven batch of pages: sides in {512, 640, ..., 3072}, 12-23 bands,
    2-6 classes, 1k-100k training pixels a class (at most half the class),
    k = K - 1 variates.  With ``workers`` > 1 the pages are drawn by that many
    fresh ("spawn") processes; every page has its own seed, so the pages are
    the same either way."""
    args = [(i, seed0, sizes) for i in range(count)]
    if workers > 1 and count > 1:
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor

        with ProcessPoolExecutor(max_workers=min(workers, count),
                                 mp_context=multiprocessing.get_context("spawn")) as ex:
            return list(ex.map(_batch_page_args, args))
    return [_batch_page(*a) for a in args]
