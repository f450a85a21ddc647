"""Seeded synthetic inputs for the 2D harmonic FMM (points and strengths).

This module draws random numbers only; it holds none of the method's
arithmetic, so both the GPU library's tests and the oracle can consume it.
The paper evaluates on synthetic particle sets (uniform squares, line-like and
clustered sets, Sec. 4.1 and Sec. 5); no public dataset is involved.  Every
generator takes an explicit seed (numpy ``default_rng``); the standard seeds are
``BASE_SEED + workload index (+ snapshot / instance index)``.

Workloads (sizes as used by the tests and the benchmark):
  * ``uniform``        -- x, y ~ U[0,1]^2.
  * ``cluster_mix``    -- 1e6-point headline set: 90 % from 8 Gaussians with
                          centres U[0.1,0.9]^2 and sigma log-uniform in
                          [0.01, 0.1], 10 % uniform background; points outside
                          the unit square are redrawn.
  * ``snapshot``       -- dynamic sequence: snapshot 0 uniform, snapshot k >= 1
                          from 4 Gaussians (fixed seeded centres U[0.2,0.8]^2)
                          with sigma = 0.2 * 0.8^k, redrawn into [0,1]^2.
  * ``batch_sizes`` / ``batch_instance`` -- 512 instances, N_b = floor(10^U(3,5)),
                          each uniform or one Gaussian (centre (0.5,0.5),
                          sigma 0.05) with probability 1/2.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20131106

# Workload indices used to derive seeds.
W_PLAIN_FP64 = 0      # N=1e4 uniform, real strengths, p=20
W_CLUSTER_1M = 1      # N=1e6 Gaussian mixture, complex strengths, p=17
W_DYNAMIC = 2         # 20 snapshots at N=2e6, real strengths U(-1,1)
W_BATCHED = 3         # 512 instances
W_DIFFERENTIATED = 4  # N=1e6 uniform, real strengths, upstream w, v ~ N(0,1)


def rng(workload: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + workload + 1000 * sub)


def uniform(n: int, g: np.random.Generator) -> np.ndarray:
    return g.random((n, 2))


def _gauss_in_square(n: int, centre, sigma: float, g: np.random.Generator) -> np.ndarray:
    out = np.empty((0, 2))
    while out.shape[0] < n:
        need = n - out.shape[0]
        z = g.normal(size=(2 * need + 16, 2)) * sigma + np.asarray(centre)
        ok = np.all((z >= 0.0) & (z <= 1.0), axis=1)
        out = np.vstack([out, z[ok][:need]])
    return out


def cluster_mix(n: int, g: np.random.Generator, n_clusters: int = 8, frac_uniform: float = 0.1) -> np.ndarray:
    n_u = int(round(frac_uniform * n))
    n_c = n - n_u
    centres = g.uniform(0.1, 0.9, size=(n_clusters, 2))
    sigmas = 10.0 ** g.uniform(-2.0, -1.0, size=n_clusters)
    counts = np.full(n_clusters, n_c // n_clusters)
    counts[: n_c - counts.sum()] += 1
    parts = [_gauss_in_square(int(c), centres[i], sigmas[i], g) for i, c in enumerate(counts)]
    parts.append(uniform(n_u, g))
    pts = np.vstack(parts)
    return pts[g.permutation(n)]


def snapshot(n: int, k: int, seed_g: np.random.Generator) -> np.ndarray:
    """Snapshot k of the dynamic sequence; ``seed_g`` fixes the 4 centres."""
    centres = np.random.default_rng(BASE_SEED + W_DYNAMIC).uniform(0.2, 0.8, size=(4, 2))
    if k == 0:
        return uniform(n, seed_g)
    sigma = 0.2 * 0.8 ** k
    counts = np.full(4, n // 4)
    counts[: n - counts.sum()] += 1
    pts = np.vstack([_gauss_in_square(int(c), centres[i], sigma, seed_g) for i, c in enumerate(counts)])
    return pts[seed_g.permutation(n)]


def batch_sizes(n_inst: int, g: np.random.Generator) -> np.ndarray:
    return np.floor(10.0 ** g.uniform(3.0, 5.0, size=n_inst)).astype(np.int64)


def batch_instance(n: int, g: np.random.Generator) -> np.ndarray:
    if g.random() < 0.5:
        return uniform(n, g)
    return _gauss_in_square(n, (0.5, 0.5), 0.05, g)


def real_strengths(n: int, g: np.random.Generator) -> np.ndarray:
    return g.normal(size=n).astype(np.complex128)


def complex_strengths(n: int, g: np.random.Generator) -> np.ndarray:
    return g.normal(size=n) + 1j * g.normal(size=n)


def uniform_real_strengths(n: int, g: np.random.Generator) -> np.ndarray:
    return g.uniform(-1.0, 1.0, size=n).astype(np.complex128)


def leaf_levels(n: int, target_per_leaf: float) -> int:
    """Smallest N_levels with about ``target_per_leaf`` points per leaf or fewer
    (N_f = 4^(N_levels-1) <= n).  Pure sizing arithmetic."""
    lv = 1
    while 4 ** lv <= n and n / 4 ** (lv - 1) > target_per_leaf * 2:
        lv += 1
    return lv
