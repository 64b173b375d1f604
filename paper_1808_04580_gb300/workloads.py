"""Seeded synthetic point clouds and right-hand sides.

These generators stand in for the paper's data sets, none of which are
available here (the spiral generator of Sec. 6.1, the photo of Sec. 6.2.1,
the crescent-fullmoon set of Sec. 6.2.2).  They hold none of the method's
arithmetic: they only draw inputs, with numpy's ``default_rng(seed)``.

Both the tests' oracle side and the GPU side take their inputs from here.

* ``two_arm_spiral``      -- Sec. 6.1 stand-in: t ~ U[0, 4 pi], arm in {0, 1},
  radius t / (4 pi), angle t + pi * arm, z = 0, plus N(0, 0.02^2) noise on
  all three coordinates.  n = 5000, sigma = 0.5 in the small FP64 case.
* ``helix_classes``       -- Sec. 6.1-like geometry: C classes wound as
  helices of radius up to r, z in [-h, h] (the paper's generator is run
  with h = 10, r = 2 and 5 classes; reading h as the half-height and the
  winding are our own).
* ``voronoi_image``       -- Sec. 6.2.1 stand-in: a W x H image of S random
  Voronoi cells with colours U[0, 1]^3, every pixel's feature = its cell's
  colour + N(0, 0.03^2).  Extremely clustered: S tight blobs in colour space.
* ``gaussian_mixture``    -- many independent graphs: 2-8 clusters with
  centres U[-1, 1]^3 and per-cluster std U[0.05, 0.3].
* ``ball_plus_clusters``  -- 50 % uniform in the unit ball, 50 % in 5 Gaussian
  clusters (centres at radius 0.6, std 0.04).
* ``two_moons``           -- Sec. 6.2.2 stand-in: two interleaved half circles
  in the (x, y) plane with N(0, noise^2) on all three coordinates.
"""
import math

import numpy as np


def rhs(n, nrhs=1, seed=0):
    """x ~ N(0, 1), shape (n,) or (n, nrhs) column blocks."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, nrhs))
    return x[:, 0].copy() if nrhs == 1 else np.asfortranarray(x)


def two_arm_spiral(n=5000, noise=0.02, seed=0):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 4.0 * math.pi, n)
    arm = rng.integers(0, 2, n)
    r = t / (4.0 * math.pi)
    ang = t + math.pi * arm
    v = np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(n)], axis=1)
    v += rng.normal(0.0, noise, (n, 3))
    return v


def helix_classes(n=2000, classes=5, h=10.0, r=2.0, noise=0.1, seed=0):
    rng = np.random.default_rng(seed)
    cls = np.arange(n) % classes
    s = rng.uniform(0.0, 1.0, n)
    ang = 2.0 * math.pi * (s * 1.5 + cls / classes)
    rad = r * (0.25 + 0.75 * s)
    v = np.stack([rad * np.cos(ang), rad * np.sin(ang), h * (2.0 * s - 1.0)], axis=1)
    v += rng.normal(0.0, noise, (n, 3))
    return v, cls


def voronoi_image(width=1000, height=1000, sites=12, noise=0.03, seed=0):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, [width, height], (sites, 2))
    colours = rng.uniform(0.0, 1.0, (sites, 3))
    yy, xx = np.mgrid[0:height, 0:width]
    pix = np.stack([xx.ravel() + 0.5, yy.ravel() + 0.5], axis=1)
    label = np.empty(pix.shape[0], dtype=np.int64)
    chunk = 1 << 18
    for s in range(0, pix.shape[0], chunk):
        p = pix[s:s + chunk]
        dist = ((p[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
        label[s:s + chunk] = dist.argmin(axis=1)
    v = colours[label] + rng.normal(0.0, noise, (pix.shape[0], 3))
    return v, label


def gaussian_mixture(n, seed=0):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 9))
    centres = rng.uniform(-1.0, 1.0, (k, 3))
    std = rng.uniform(0.05, 0.3, k)
    lab = rng.integers(0, k, n)
    return centres[lab] + rng.standard_normal((n, 3)) * std[lab, None]


def many_graph_sizes(graphs=256, n_min=1000, n_max=200000, seed=0):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), graphs))).astype(np.int64)


def many_graphs(graphs=256, n_min=1000, n_max=200000, seed=0):
    sizes = many_graph_sizes(graphs, n_min, n_max, seed)
    return [gaussian_mixture(int(s), seed=seed * 100003 + g + 1) for g, s in enumerate(sizes)]


def _uniform_ball(rng, n, d=3):
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = rng.uniform(0.0, 1.0, n) ** (1.0 / d)
    return g * r[:, None]


def ball_plus_clusters(n=10_000_000, clusters=5, radius=0.6, std=0.04, seed=0):
    rng = np.random.default_rng(seed)
    n_uni = n // 2
    n_cl = n - n_uni
    dirs = rng.standard_normal((clusters, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    centres = radius * dirs
    lab = rng.integers(0, clusters, n_cl)
    pts = np.empty((n, 3))
    pts[:n_uni] = _uniform_ball(rng, n_uni)
    pts[n_uni:] = centres[lab] + rng.standard_normal((n_cl, 3)) * std
    perm = rng.permutation(n)
    return pts[perm]


def five_centres(n=2000, std=0.6, spread=3.0, seed=0):
    """Normal clouds around five centres in U[-spread, spread]^3, each node labelled by
    its nearest centre (the semi-supervised data of the phase-field experiment)."""
    rng = np.random.default_rng(seed)
    cent = rng.uniform(-spread, spread, (5, 3))
    v = cent[rng.integers(0, 5, n)] + rng.standard_normal((n, 3)) * std
    lab = ((v[:, None, :] - cent[None, :, :]) ** 2).sum(axis=2).argmin(axis=1)
    return v, lab


def two_moons(n=500_000, noise=0.05, seed=0):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 2, n)
    t = rng.uniform(0.0, math.pi, n)
    x = np.where(lab == 0, np.cos(t), 1.0 - np.cos(t))
    y = np.where(lab == 0, np.sin(t), 0.5 - np.sin(t))
    v = np.stack([x, y, np.zeros(n)], axis=1) + rng.normal(0.0, noise, (n, 3))
    return v, np.where(lab == 0, -1.0, 1.0)


# Named configurations (parameters of the fast summation go with the data).
CONFIGS = {
    "spiral5k": dict(n=5000, sigma=0.5, N=32, m=4, p=4),
    "image1M": dict(n=1_000_000, sigma=0.1, N=64, m=4, p=4),
    "graphs256": dict(graphs=256, sigma=0.5, N=64, m=4, p=4, nrhs=8),
    "ball10M": dict(n=10_000_000, sigma=0.08, N=128, m=6, p=6),
    "moons500k": dict(n=500_000, sigma=0.2, N=128, m=4, p=4),
}
