"""Seeded synthetic QAP instances (Koopmans-Beckmann flow F, distance D).

This module only draws random numbers and lays them out as integer matrices.
It holds none of the dual-ascent arithmetic, so both the CUDA path and the CPU
oracle may take their inputs from it.

The paper measures on QAPLIB instances (nug, tai, kra, tho; Sec. 6, Table 1).
Those files are not available here, so every workload is a synthetic stand-in
with the same structure: symmetric integer F and D with zero diagonals, N from
8 to 35, Manhattan grids (nug-like), Euclidean points with clustered heavy-tailed
flows (tai-b / kra-like).  All draws use ``numpy.random.default_rng(seed)`` and
rounding is floor(x + 0.5).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_symmetric", "grid_manhattan", "clustered_euclid", "instance",
    "subproblem_nodes", "poisson_requests", "WORKLOADS",
]


def _sym_from_upper(N: int, vals: np.ndarray) -> np.ndarray:
    iu = np.triu_indices(N, 1)
    M = np.zeros((N, N), dtype=np.int64)
    M[iu] = vals
    M = M + M.T
    return M.astype(np.int32)


def _round(x: np.ndarray) -> np.ndarray:
    return np.floor(x + 0.5).astype(np.int64)


def uniform_symmetric(N: int, seed: int = 0, hi: int = 9):
    """F and D symmetric, zero diagonal, off-diagonal uniform integers in [0, hi].

    Draw order: the upper triangle of F (row-major), then that of D.
    """
    rng = np.random.default_rng(seed)
    npairs = N * (N - 1) // 2
    F = _sym_from_upper(N, rng.integers(0, hi + 1, size=npairs))
    D = _sym_from_upper(N, rng.integers(0, hi + 1, size=npairs))
    return F, D


def grid_manhattan(N: int, rows: int, cols: int, seed: int = 0,
                   p_zero: float = 0.4, hi: int = 10):
    """D = Manhattan distance on a rows x cols grid (location l at (l // cols, l % cols)).

    F symmetric: each pair i<k is 0 with probability p_zero, else uniform in [1, hi].
    Draw order: the zero mask for all pairs, then the values for all pairs.
    """
    assert rows * cols == N
    rng = np.random.default_rng(seed)
    loc = np.array([(l // cols, l % cols) for l in range(N)], dtype=np.int64)
    D = (np.abs(loc[:, None, 0] - loc[None, :, 0]) +
         np.abs(loc[:, None, 1] - loc[None, :, 1])).astype(np.int32)
    npairs = N * (N - 1) // 2
    zero = rng.random(npairs) < p_zero
    vals = rng.integers(1, hi + 1, size=npairs)
    F = _sym_from_upper(N, np.where(zero, 0, vals))
    return F, D


def clustered_euclid(N: int, seed: int = 0, clusters: int = 5,
                     mu: float = 3.0, sigma: float = 1.0, p_inter_zero: float = 0.9):
    """D = rounded Euclidean distance between N points uniform in a 100 x 100 square.

    F symmetric and clustered: labels = permutation(N) % clusters; intra-cluster
    pairs carry round(lognormal(mu, sigma)); inter-cluster pairs are 0 with
    probability p_inter_zero, else round(lognormal(mu, sigma)).
    Draw order: points, labels, lognormal values for all pairs, zero mask for all pairs.
    """
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 100.0, size=(N, 2))
    labels = rng.permutation(N) % clusters
    npairs = N * (N - 1) // 2
    ln = _round(rng.lognormal(mu, sigma, size=npairs))
    u = rng.random(npairs)
    iu = np.triu_indices(N, 1)
    intra = labels[iu[0]] == labels[iu[1]]
    F = _sym_from_upper(N, np.where(intra | (u >= p_inter_zero), ln, 0))
    diff = pts[:, None, :] - pts[None, :, :]
    D = _round(np.sqrt((diff ** 2).sum(-1))).astype(np.int32)
    np.fill_diagonal(D, 0)
    return F, D


# Named workloads: (generator, kwargs, iterations).
WORKLOADS = {
    "uniform_n8": (uniform_symmetric, dict(N=8, seed=0), 50),
    "grid_n12": (grid_manhattan, dict(N=12, rows=3, cols=4, seed=0), 100),
    "clustered_n20": (clustered_euclid, dict(N=20, seed=0), 200),
    "clustered_n25": (clustered_euclid, dict(N=25, seed=0), 100),
    "clustered_n30": (clustered_euclid, dict(N=30, seed=0), 50),
    "clustered_n35": (clustered_euclid, dict(N=35, seed=0), 300),
}


def instance(name: str):
    """Return (F, D, iterations) of a named workload."""
    gen, kw, iters = WORKLOADS[name]
    F, D = gen(**kw)
    return F, D, iters


def subproblem_nodes(N: int = 25, count: int = 256, kmin: int = 1, kmax: int = 15,
                     seed_base: int = 1000):
    """Branch-and-bound nodes of one instance: node s fixes k facilities to k locations.

    Node s draws from default_rng(seed_base + s): k = integers(kmin, kmax + 1), then
    k distinct facilities, then k distinct locations, paired in draw order.
    Returns a list of (facilities, locations) int32 arrays.
    """
    nodes = []
    for s in range(count):
        rng = np.random.default_rng(seed_base + s)
        k = int(rng.integers(kmin, kmax + 1))
        fac = rng.choice(N, size=k, replace=False).astype(np.int32)
        loc = rng.choice(N, size=k, replace=False).astype(np.int32)
        nodes.append((fac, loc))
    return nodes


def poisson_requests(count: int = 1000, rate: float = 50.0, nmin: int = 12, nmax: int = 30,
                     seed: int = 7):
    """Bound requests: Poisson arrivals (exponential gaps) with N uniform in [nmin, nmax].

    Request r uses clustered_euclid(N_r, seed=r).  Returns (arrival_s, N) arrays.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    Ns = rng.integers(nmin, nmax + 1, size=count)
    return np.cumsum(gaps), Ns.astype(np.int32)
