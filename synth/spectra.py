"""Seeded pages whose canonical-variate spectra are hard on an eigensolver.

Each page is built from class means and covariances chosen in band space
(the same stroke layout and rectangle training labels as ``cubes.py``), so
that the generalized eigenproblem of its training pixels has one of three
awkward shapes:

* ``wide_spread_page``: the class means differ by thousands of DN along the
  band direction of least within-class variance and by about one DN along
  another, so the largest and the smallest non-zero eigenvalue are more than
  1e8 apart;
* ``degenerate_pair_page``: the training pixels of four classes are exact
  images of one another under an integer map R of band space (a quarter
  turn of bands 0 and 1, a sign change of band 2), and every class uses the
  same within-class deviations, closed under R; both scatter matrices then
  commute with R and the two largest eigenvalues are equal in exact
  arithmetic (``perturb`` = p moves one training pixel by p DN in band 3,
  which R leaves alone, splitting them by about 2e-10 p^2 relative);
* ``near_singular_page``: 16-bit data in which one band equals another plus
  a constant except at a few training pixels, so the within-class scatter
  has a condition number above 1e10 while staying positive definite.

Like ``cubes.py`` this module only draws inputs; nothing here computes any
part of Canonical Variates Analysis.
"""
from __future__ import annotations

import math

import numpy as np

from .cubes import Workload, _haar_orthogonal, make_workload


def _cov(rng: np.random.Generator, B: int, lo: float, hi: float, illum: float = 40.0):
    """Random SPD covariance Q diag(s^2) Q^T + illum^2 11^T with stds s
    log-uniform in [lo, hi]; also returns Q and s (columns of Q are the
    directions, s their stds before the shared term)."""
    q = _haar_orthogonal(rng, B)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=B))
    ones = np.ones((B, 1))
    cov = (q * s ** 2) @ q.T + illum ** 2 * (ones @ ones.T)
    return 0.5 * (cov + cov.T), q, s


def wide_spread_page(seed: int = 9100, B: int = 23, H: int = 512, W: int = 512,
                     n: int = 20000) -> Workload:
    """Four classes, one covariance; the class means are offset by d_j a_cj
    along three orthogonal directions u_j of band space with d_1 >> d_2 >> d_3
    (u_1 the direction of least within-class variance), giving non-zero
    eigenvalues roughly in the ratio d_1^2 : d_2^2 : d_3^2 (in units of the
    within-class variance along each direction)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = 4
    cov, q, s = _cov(rng, B, 8.0, 60.0, illum=0.0)
    order = np.argsort(s)
    u1 = q[:, order[0]]          # least within-class variance
    u2 = q[:, order[B // 2]]
    u3 = q[:, order[-1]]         # most within-class variance
    # centred offsets of the four classes along each direction
    a = np.array([[1.0, -1.0, 1.0, -1.0], [1.0, 1.0, -1.0, -1.0], [1.0, -1.0, -1.0, 1.0]])
    d = np.array([300.0 * s[order[0]], 3.0 * s[order[B // 2]], 0.012 * s[order[-1]]])
    base = np.full(B, 2000.0) + 300.0 * np.sin(np.linspace(0.0, math.pi, B))
    means = np.stack([base + d[0] * a[0, c] * u1 + d[1] * a[1, c] * u2 + d[2] * a[2, c] * u3
                      for c in range(K)])
    covs = np.stack([cov] * K)
    return make_workload(seed + 1, B, H, W, K, (n,) * K, K - 1, both=False, means=means, covs=covs,
                         name=f"wide_spread_{B}b_{H}x{W}")


def degenerate_pair_page(seed: int = 9200, B: int = 12, H: int = 384, W: int = 384, n0: int = 500,
                         perturb: int = 0) -> Workload:
    """Four classes with R-symmetric training pixels (see the module text).
    Class c's training pixels are mu_c + D, D = D0 u R D0 u R^2 D0 u R^3 D0
    (4 n0 deviations drawn once from one Gaussian and rounded), with
    mu_c = m + R^c e, e = (400, 0, 240, 0, ..): between-class scatter is
    isotropic in bands 0 and 1, so the top two eigenvalues coincide.  Pixels
    that are not training pixels are Gaussian around their class mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = 4
    cov, _, _ = _cov(rng, B, 15.0, 50.0)
    m = np.rint(2000.0 + 200.0 * np.cos(np.linspace(0.0, 2.0, B)))
    e = np.zeros(B)
    e[0], e[2] = 400.0, 240.0

    def rot(x):
        y = np.array(x, copy=True)
        y[..., 0], y[..., 1] = -x[..., 1], x[..., 0]
        y[..., 2] = -x[..., 2]
        return y

    mus = []
    v = e.copy()
    for _ in range(K):
        mus.append(m + v)
        v = rot(v)
    means = np.stack(mus)
    w = make_workload(seed + 1, B, H, W, K, (4 * n0,) * K, K - 1, both=False, means=means,
                      covs=np.stack([cov] * K), name=f"degenerate_pair_{B}b_{H}x{W}" + (f"_split{perturb}" if perturb else ""))
    # the within-class deviations, closed under R
    z = rng.multivariate_normal(np.zeros(B), cov, size=n0)
    d0 = np.rint(z)
    devs = [d0]
    for _ in range(3):
        devs.append(rot(devs[-1]))
    D = np.concatenate(devs, axis=0)  # (4 n0, B)
    cube = w.cube.reshape(B, -1)
    lab = w.labels.reshape(-1)
    for c in range(K):
        idx = np.flatnonzero(lab == c + 1)
        if idx.size != D.shape[0]:
            raise RuntimeError("class did not get its training pixels")
        vals = means[c][None, :] + D
        if perturb and c == 0:
            vals[0, 3] += float(perturb)
        if vals.min() < 0 or vals.max() > 4095:
            raise RuntimeError("training pixel outside 12 bits")
        cube[:, idx] = vals.T.astype(np.uint16)
    return w


def near_singular_page(seed: int = 9300, B: int = 23, H: int = 512, W: int = 512, n: int = 20000,
                       dead: int = 7, deviants: int = 4) -> Workload:
    """16-bit data (means near 30 000 DN, stds 300-2000 DN); band `dead`
    equals band `dead - 1` plus 100 at every pixel, except that `deviants`
    training pixels of each class carry one DN more in band `dead`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = 4
    covs = []
    for _ in range(K):
        c, _, _ = _cov(rng, B, 300.0, 2000.0, illum=800.0)
        covs.append(c)
    covs = np.stack(covs)
    base = 30000.0 + 3000.0 * np.sin(np.linspace(0.0, 2.5, B))
    means = np.stack([base + rng.normal(0.0, 1500.0, size=B) for _ in range(K)])
    w = make_workload(seed + 1, B, H, W, K, (n,) * K, K - 1, both=False, means=means, covs=covs,
                      max_dn=60000, name=f"near_singular_{B}b_{H}x{W}")
    cube = w.cube.reshape(B, -1)
    cube[dead] = np.minimum(cube[dead - 1].astype(np.int64) + 100, 65534).astype(np.uint16)
    lab = w.labels.reshape(-1)
    for c in range(K):
        idx = np.flatnonzero(lab == c + 1)
        pick = rng.choice(idx, size=deviants, replace=False)
        cube[dead, pick] += 1
    return w
