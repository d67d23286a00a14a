"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle comparisons.

Only random numbers and mesh coordinates are produced here; none of the method's arithmetic
lives in this module.  Mesh perturbation (a smooth, seeded deformation of the uniform grid
that keeps boundary vertices on the boundary):
    x_i <- x_i + A h prod_j sin(pi x_j) sin(2 pi x_{(i+1) mod d} + theta_i),
    theta_i ~ U[0, 2 pi) from the seed, h = 1/n.
"""
import itertools

import numpy as np


def vertices(d, n, amp=0.0, seed=0):
    """(n+1)^d x d vertex coordinates of [0,1]^d, lexicographic with x fastest."""
    g = np.linspace(0.0, 1.0, n + 1)
    X = np.array(list(itertools.product(*([g] * d))))[:, ::-1].copy()
    if amp:
        rng = np.random.default_rng(seed)
        theta = rng.uniform(0.0, 2.0 * np.pi, d)
        bump = np.prod(np.sin(np.pi * X), axis=1)
        disp = np.stack([bump * np.sin(2 * np.pi * X[:, (i + 1) % d] + theta[i]) for i in range(d)], 1)
        X = X + amp / n * disp
    return X


def uniform(size, seed, lo=-1.0, hi=1.0):
    """size values ~ U(lo, hi) in float64 from the given seed."""
    return np.random.default_rng(seed).uniform(lo, hi, size)


def node_noise_mask(d, N1):
    """1.0 at interior velocity nodes of the N1^d grid (x fastest), 0.0 on the boundary."""
    idx = np.indices((N1,) * d).reshape(d, -1)      # idx[0] slowest; the mask is symmetric in the axes
    inner = np.all((idx > 0) & (idx < N1 - 1), axis=0)
    return inner.astype(np.float64)
