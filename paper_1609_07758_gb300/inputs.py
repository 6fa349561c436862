"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module draws random numbers and samples plain functions on grids; it holds
none of the solver's arithmetic (no FEM matrices, no quadrature, no transforms).
All generators use numpy's PCG64 (``default_rng(seed)``).

Workloads (sizes and distributions follow the solver's intended uses; the paper
itself uses only the manufactured 2D problem of its Table 1, and no dataset):

* ``manufactured_params``: integers a, b in [1, 8] for u = sin(pi a x) sin(pi b y)
  and N(0, sigma) noise to add to a load vector (2D, n = 2, K = 64 case).
* ``smooth_sine_rhs``: f = sum_{m=1}^{16} c_m sin(pi a_m x) sin(pi b_m y),
  c_m ~ N(0, 1), a_m, b_m integers U[1, 32], sampled at the dof coordinates
  x_p = (p + 1) h / n, plus U(-1e-3, 1e-3) * max|f| noise (2D, n = 9, K = 1024 case).
* ``gaussian_rhs``: iid N(0, 1) right-hand sides (3D cases).
* ``batch_problems``: per-problem K, n, X, nrhs of the batched 2D case.
"""
import numpy as np


def dof_coordinates(n, K, X):
    """Coordinates of the n K - 1 unknowns of one axis (uniform fine grid of step h / n)."""
    return (np.arange(n * K - 1) + 1.0) * (float(X) / K) / n


def manufactured_params(seed, shape, sigma=1e-3):
    rng = np.random.default_rng(seed)
    a, b = (int(v) for v in rng.integers(1, 9, size=2))
    noise = rng.normal(0.0, sigma, size=shape)
    return a, b, noise


def smooth_sine_rhs(seed, n, K, X=(1.0, 1.0), modes=16, max_freq=32, noise=1e-3, nrhs=1):
    """(nrhs, M, M) FP64 smooth RHS sampled on the dof grid, plus uniform noise."""
    rng = np.random.default_rng(seed)
    x = dof_coordinates(n, K, X[0])
    y = dof_coordinates(n, K, X[1])
    out = np.empty((nrhs, x.size, y.size))
    for r in range(nrhs):
        c = rng.normal(0.0, 1.0, size=modes)
        a = rng.integers(1, max_freq + 1, size=modes)
        b = rng.integers(1, max_freq + 1, size=modes)
        Sx = np.sin(np.pi * np.outer(a, x))          # (modes, M)
        Sy = np.sin(np.pi * np.outer(b, y))
        f = (Sx * c[:, None]).T @ Sy
        f += rng.uniform(-noise, noise, size=f.shape) * np.abs(f).max()
        out[r] = f
    return out


def gaussian_rhs(seed, shape, dtype=np.float64):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape).astype(dtype)


def batch_problems(seed, count=512, k_range=(32, 512), n_range=(2, 8), x_range=(0.5, 4.0),
                   rhs_range=(1, 8)):
    """Independent 2D problems: K (both axes) and n drawn log-uniform, X per axis uniform,
    nrhs uniform; returned as dicts with keys N, K, n, X, alpha, nrhs."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        K = int(np.floor(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1] + 1)))))
        K = min(max(K, k_range[0]), k_range[1])
        n = int(np.floor(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1] + 1)))))
        n = min(max(n, n_range[0]), n_range[1])
        X = (float(rng.uniform(*x_range)), float(rng.uniform(*x_range)))
        nrhs = int(rng.integers(rhs_range[0], rhs_range[1] + 1))
        probs.append({"N": 2, "K": (K, K), "n": n, "X": X, "alpha": 0.0, "nrhs": nrhs})
    return probs


def batch_rhs(seed, index, prob):
    """N(0,1) right-hand sides (nrhs, M_1, .., M_N) of problem `index` of a batch."""
    rng = np.random.default_rng([seed, index])
    shape = (prob["nrhs"],) + tuple(prob["n"] * k - 1 for k in prob["K"])
    return rng.standard_normal(size=shape)
