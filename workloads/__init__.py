"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on upsampled MNIST, colour-transfer images and DOTmark
(Sec. 4.1, Appx. D); none of those datasets is used here. These generators stand
in for them with the same sizes, value ranges and structure. They hold none of
the method's arithmetic: they only build marginals, points and cost matrices,
which are inputs of the problem. Both the CUDA path and the oracle read the same
arrays produced here.

Every generator takes a seed and uses numpy's PCG64 stream for it.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def grid_points(side):
    """Pixel centres (a / (side-1), b / (side-1)) of a side x side grid, row-major."""
    a, b = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1).astype(np.float64) / (side - 1)


def grid_cost(side, kind="sqeuclid"):
    """Grid cost between pixel centres, normalised to max 1 (Sec. 4.1).

    kind: "sqeuclid" (L2 squared) or "l1".
    """
    pts = grid_points(side)
    diff = pts[:, None, :] - pts[None, :, :]
    if kind == "sqeuclid":
        C = (diff ** 2).sum(axis=2)
    elif kind == "l1":
        C = np.abs(diff).sum(axis=2)
    else:
        raise ValueError(kind)
    return C / C.max()


def gaussian_mixture_histogram(rng, side, k, sigma_lo, sigma_hi, floor):
    """A histogram over a side x side grid: k isotropic Gaussians with centres
    uniform on [0, side)^2, widths uniform in [sigma_lo, sigma_hi] pixels and
    weights uniform in [0.2, 1], plus a constant floor, normalised to sum 1."""
    a, b = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    h = np.zeros((side, side))
    for _ in range(k):
        ca, cb = rng.uniform(0, side, size=2)
        s = rng.uniform(sigma_lo, sigma_hi)
        w = rng.uniform(0.2, 1.0)
        h += w * np.exp(-((a - ca) ** 2 + (b - cb) ** 2) / (2 * s * s))
    h = h / h.sum() + floor
    return (h / h.sum()).ravel()


def grid_problem_784(seed):
    """28 x 28 grid (n = m = 784): two 3-Gaussian histograms (sigma 2-6 px) with a
    1e-6 floor; squared-Euclidean grid cost with max 1, float64.
    Stands in for the original-resolution MNIST problems (Sec. 4.1)."""
    rng = _rng(seed)
    r = gaussian_mixture_histogram(rng, 28, 3, 2.0, 6.0, 1e-6)
    c = gaussian_mixture_histogram(rng, 28, 3, 2.0, 6.0, 1e-6)
    return dict(C=grid_cost(28, "sqeuclid"), r=r, c=c)


def grid_problem_4096(seed, kind="sqeuclid", side=64, zero_frac=0.10):
    """64 x 64 grid (n = m = 4096): Gaussian-mixture histograms (3 components,
    sigma 4-12 px) with 10% of the bins set to zero (seeded choice), normalised;
    L1 or squared-Euclidean grid cost with max 1, stored as float32.
    Stands in for the upsampled 64 x 64 MNIST problems (Sec. 4.1, Table 1)."""
    rng = _rng(seed)
    n = side * side
    out = []
    for _ in range(2):
        h = gaussian_mixture_histogram(rng, side, 3, 4.0 * side / 64, 12.0 * side / 64, 0.0)
        zero = rng.choice(n, size=int(round(zero_frac * n)), replace=False)
        h[zero] = 0.0
        out.append(h / h.sum())
    C = grid_cost(side, kind).astype(np.float32)
    return dict(C=C, r=out[0], c=out[1])


def uniform_points_problem(seed, n, m=None, d=2):
    """Points uniform in the unit square, Dirichlet(1) weights (many-small-problems regime)."""
    rng = _rng(seed)
    m = n if m is None else m
    X = rng.uniform(0, 1, size=(n, d)).astype(np.float32)
    Y = rng.uniform(0, 1, size=(m, d)).astype(np.float32)
    r = rng.dirichlet(np.ones(n))
    c = rng.dirichlet(np.ones(m))
    return dict(X=X, Y=Y, r=r, c=c)


def batch_sizes(seed, count=256, lo=256, hi=4096):
    """Problem sizes n_k = m_k drawn uniformly from {lo, ..., hi}."""
    return _rng(seed).integers(lo, hi + 1, size=count)


def gmm_points(rng, n, d, k, mean_scale, sigma):
    means = rng.normal(0.0, mean_scale, size=(k, d))
    comp = rng.integers(0, k, size=n)
    return (means[comp] + sigma * rng.normal(size=(n, d))).astype(np.float32)


def gmm_problem_d64(seed, n=16384, d=64):
    """Two 8-component isotropic Gaussian mixtures in d = 64 (means ~ N(0, 4 I),
    unit widths), uniform weights (high-dimensional point-cloud regime)."""
    rng = _rng(seed)
    X = gmm_points(rng, n, d, 8, 2.0, 1.0)
    Y = gmm_points(rng, n, d, 8, 2.0, 1.0)
    return dict(X=X, Y=Y, r=np.full(n, 1.0 / n), c=np.full(n, 1.0 / n))


def colour_cloud(rng, n, k=16):
    """A 16-component mixture in the RGB cube [0, 1]^3 with widths 0.02-0.1, clipped."""
    means = rng.uniform(0.1, 0.9, size=(k, 3))
    sig = rng.uniform(0.02, 0.1, size=k)
    w = rng.uniform(0.2, 1.0, size=k)
    comp = rng.choice(k, size=n, p=w / w.sum())
    pts = means[comp] + sig[comp, None] * rng.normal(size=(n, 3))
    return np.clip(pts, 0.0, 1.0).astype(np.float32)


def colour_problem(seed, n=1 << 20):
    """Two RGB colour clouds of n points each (d = 3), uniform weights.
    Stands in for the 1024 x 1024 colour-transfer problem (Sec. 4.2, Fig. 3)."""
    rng = _rng(seed)
    X = colour_cloud(rng, n)
    Y = colour_cloud(rng, n)
    return dict(X=X, Y=Y, r=np.full(n, 1.0 / n), c=np.full(n, 1.0 / n))


def random_dense_problem(seed, n, m=None, scale=1.0):
    """Small random problem: C uniform in [0, scale] (float64), r, c Dirichlet(1) plus a
    small floor, for unit tests of single sweeps."""
    rng = _rng(seed)
    m = n if m is None else m
    C = rng.uniform(0, scale, size=(n, m))
    r = rng.dirichlet(np.ones(n)) + 1e-3 / n
    c = rng.dirichlet(np.ones(m)) + 1e-3 / m
    return dict(C=C, r=r / r.sum(), c=c / c.sum())
