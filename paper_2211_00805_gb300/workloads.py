"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: point clouds, distributions and problem lists.  It
contains none of the method's arithmetic (no kNN, no Laplacian, no heat filter, no Sinkhorn), so
both the CUDA path and the FP64 oracle can be fed the same bytes from it.  Every generator takes
an explicit seed and uses ``numpy.random.default_rng``; points are returned as float32 (the CUDA
path's input type) and the oracle receives exactly those values widened to float64.

The paper's own data (a swiss roll in R^10 with Gaussians on it, mass-cytometry organoids, single-
cell time series) are not available; these recipes stand in for them:

* ``sphere``          n points uniform on the unit 2-sphere in R^3 (smooth 2-d manifold);
* ``tanh_manifold``   latents z ~ N(0, I_l) pushed through a fixed random 2-layer tanh map into
                      R^D plus isotropic noise (a curved l-dimensional manifold);
* ``cluster_curves``  Gaussian clusters strung along cubic polynomial trajectories in R^D, shaped
                      like PCA-reduced single-cell data;
* distributions: von Mises-Fisher bumps, softmax-weighted Gaussian bumps, uniform measures on
  unions of clusters, Dirichlet(1) measures on random supports.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ------------------------------------------------------------------------------------ points
def sphere(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform on the unit sphere S^2 in R^3: z ~ N(0, I_3), x = z / |z|."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n, 3))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return z.astype(np.float32)


def tanh_manifold(n: int, latent: int, ambient: int, seed: int, hidden: int = 64,
                  noise: float = 0.01):
    """Latents z ~ N(0, I_latent); x = W2 tanh(W1 z + b1) + N(0, noise^2 I) in R^ambient.

    W1 ~ N(0, 1/latent), b1 ~ N(0, 0.1^2), W2 ~ N(0, 1/hidden).  Returns (X float32 [n, ambient],
    Z float64 [n, latent]).
    """
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, latent)) / math.sqrt(latent)
    b1 = 0.1 * rng.standard_normal(hidden)
    W2 = rng.standard_normal((ambient, hidden)) / math.sqrt(hidden)
    Z = rng.standard_normal((n, latent))
    X = np.tanh(Z @ W1.T + b1) @ W2.T + noise * rng.standard_normal((n, ambient))
    return X.astype(np.float32), Z


def cluster_curves(n: int, dim: int = 30, clusters: int = 20, curves: int = 4, seed: int = 3,
                   spread: float = 0.35):
    """Gaussian clusters placed at consecutive positions along cubic polynomial trajectories.

    Each curve is c(s) = p0 + p1 s + p2 s^2 + p3 s^3, s in [0, 1], with random coefficient vectors
    in R^dim; ``clusters / curves`` cluster centres sit at evenly spaced s on each curve, and every
    cluster's standard deviation is ``spread`` times the distance between consecutive centres on
    its curve so that neighbouring clusters overlap.  All curves start from a shared origin so the
    point cloud is one connected shape.  Returns (X float32 [n, dim], labels int32 [n]).
    """
    rng = np.random.default_rng(seed)
    per = clusters // curves
    centres, sds = [], []
    origin = np.zeros(dim)
    for _ in range(curves):
        coef = rng.standard_normal((3, dim)) * np.array([[2.0], [1.0], [0.6]])
        s = np.linspace(0.15, 1.0, per)
        pts = origin + s[:, None] * coef[0] + (s ** 2)[:, None] * coef[1] + (s ** 3)[:, None] * coef[2]
        gaps = np.linalg.norm(np.diff(np.vstack([origin, pts]), axis=0), axis=1)
        centres.append(pts)
        sds.append(spread * gaps)
    centres = np.vstack(centres)
    sds = np.concatenate(sds)
    labels = rng.integers(0, clusters, size=n).astype(np.int32)
    X = centres[labels] + sds[labels, None] * rng.standard_normal((n, dim))
    return X.astype(np.float32), labels


# ----------------------------------------------------------------------------- distributions
def vmf_bump(X: np.ndarray, centre: np.ndarray, kappa: float) -> np.ndarray:
    """von Mises-Fisher weights exp(kappa <x, c>) on unit vectors, normalised to sum 1 (float32)."""
    w = np.exp(kappa * (np.asarray(X, np.float64) @ np.asarray(centre, np.float64) - 1.0))
    return (w / w.sum()).astype(np.float32)


def softmax_bump(Z: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """softmax(-|z - c|^2 / 2) over the points (float32, sums to 1)."""
    e = -0.5 * np.sum((Z - centre) ** 2, axis=1)
    e -= e.max()
    w = np.exp(e)
    return (w / w.sum()).astype(np.float32)


def cluster_unions(labels: np.ndarray, m: int, per: int, seed: int) -> np.ndarray:
    """m distributions, each uniform over the points of a random union of ``per`` clusters.
    Returns float32 [n, m], columns summing to 1."""
    rng = np.random.default_rng(seed)
    C = int(labels.max()) + 1
    M = np.zeros((len(labels), m))
    for i in range(m):
        pick = rng.choice(C, size=per, replace=False)
        sel = np.isin(labels, pick)
        M[sel, i] = 1.0 / sel.sum()
    return M.astype(np.float32)


def dirichlet_support(n: int, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Dirichlet(1) weights on a random support of round(frac * n) points, zero elsewhere."""
    s = max(1, int(round(frac * n)))
    sup = rng.choice(n, size=s, replace=False)
    w = np.zeros(n)
    w[sup] = rng.dirichlet(np.ones(s))
    return w.astype(np.float32)


# ------------------------------------------------------------------------- named workloads
@dataclass
class Problem:
    """One Sinkhorn problem: points, graph size k, Chebyshev order K, time t, marginals."""
    X: np.ndarray
    k: int
    K: int
    t: float
    a: np.ndarray
    b: np.ndarray
    iters: int
    extra: dict = field(default_factory=dict)


def sphere_pair(n: int = 2000, seed: int = 0, k: int = 10, K: int = 20, t: float = 1.0,
                kappa: float = 20.0, iters: int = 200) -> Problem:
    """n points on S^2; a, b = vMF(kappa) bumps at the antipodal poles +e_z and -e_z."""
    X = sphere(n, seed)
    ez = np.array([0.0, 0.0, 1.0])
    return Problem(X, k, K, t, vmf_bump(X, ez, kappa), vmf_bump(X, -ez, kappa), iters)


def manifold_pair(n: int = 100_000, latent: int = 10, ambient: int = 50, seed: int = 2, k: int = 15,
                  K: int = 30, t: float = 5.0, iters: int = 500) -> Problem:
    """tanh manifold (latent -> ambient); a, b = softmax bumps at two random latent centres."""
    X, Z = tanh_manifold(n, latent, ambient, seed)
    rng = np.random.default_rng(seed + 1000)
    ca, cb = rng.standard_normal(latent), rng.standard_normal(latent)
    return Problem(X, k, K, t, softmax_bump(Z, ca), softmax_bump(Z, cb), iters, dict(Z=Z))


def clusters_barycenter(n: int = 200_000, dim: int = 30, m: int = 32, seed: int = 3, k: int = 10,
                        K: int = 40, t: float = 10.0, iters: int = 300):
    """Cluster-curve points with m uniform-over-3-clusters distributions and uniform weights."""
    X, labels = cluster_curves(n, dim, seed=seed)
    M = cluster_unions(labels, m, 3, seed + 1000)
    alpha = np.full(m, 1.0 / m)
    return dict(X=X, labels=labels, M=M, alpha=alpha, k=k, K=K, t=t, iters=iters)


def manifold_barycenter_grad(n: int = 500_000, latent: int = 6, ambient: int = 40, m: int = 64,
                             seed: int = 4, k: int = 10, K: int = 40, t: float = 8.0,
                             bary_iters: int = 200, sink_iters: int = 200, checkpoint: int = 20):
    """tanh manifold with m softmax-bump inputs (alpha = 1/m) and a further bump as the source."""
    X, Z = tanh_manifold(n, latent, ambient, seed)
    rng = np.random.default_rng(seed + 1000)
    M = np.stack([softmax_bump(Z, rng.standard_normal(latent)) for _ in range(m)], axis=1)
    src = softmax_bump(Z, rng.standard_normal(latent))
    alpha = np.full(m, 1.0 / m)
    return dict(X=X, Z=Z, M=M.astype(np.float32), alpha=alpha, src=src, k=k, K=K, t=t,
                bary_iters=bary_iters, sink_iters=sink_iters, checkpoint=checkpoint)


def treatment_families(outlier=None, seed: int = 0, dim: int = 5, per: int = 500):
    """Synthetic families of the expected-barycenter-effect experiment (Sec. 5): a control family of
    ten standard Gaussians and a treatment family of nine Gaussians shifted by 5 along the first
    axis plus one member centred at `outlier` on that axis (None: a tenth shifted member), `per`
    samples each in R^dim (the paper does not state the dimension).  Every member is the uniform
    distribution on its own samples.  Returns (X [n, dim] float32, MC [n, 10], MT [n, 10] float32)
    with n = 20 per, control samples first."""
    rng = np.random.default_rng(seed)
    centres = [0.0] * 10 + [5.0] * 9 + [5.0 if outlier is None else float(outlier)]
    X = np.concatenate([rng.standard_normal((per, dim)) + np.eye(dim)[0] * c for c in centres])
    M = np.zeros((20 * per, 20), np.float32)
    for i in range(20):
        M[i * per:(i + 1) * per, i] = 1.0 / per
    return X.astype(np.float32), M[:, :10].copy(), M[:, 10:].copy()


def ragged_batch(count: int = 512, seed: int = 5, n_min: int = 1_000, n_max: int = 50_000,
                 t: float = 5.0, iters: int = 200):
    """``count`` independent problems with uneven sizes: n log-uniform in [n_min, n_max], ambient
    dimension uniform in 3..20 (latent max(2, D // 3)), k in {8, 10, 15}, K in {16, 24, 32},
    Dirichlet(1) marginals on independent random 10 % supports."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        D = int(rng.integers(3, 21))
        lat = max(2, D // 3)
        k = int(rng.choice([8, 10, 15]))
        K = int(rng.choice([16, 24, 32]))
        X, _ = tanh_manifold(n, lat, D, seed * 100_003 + p)
        a = dirichlet_support(n, 0.1, rng)
        b = dirichlet_support(n, 0.1, rng)
        out.append(Problem(X, k, K, t, a, b, iters))
    return out
