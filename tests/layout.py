"""Test-side helpers: canonical compact layouts and permutation costs.

The library exports its state in the compact layouts declared in
include/rlt2.h.  These helpers build the same layouts from the oracle's dense
arrays (indexed by the paper's subscripts) with plain numpy indexing, and
evaluate the QAP objective and the conservation identity; none of the
dual-ascent arithmetic is here.
"""
from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=8)
def tile_indices(N: int):
    """Index arrays of the tiles (i, j, k, n), i != k, j != n, in export order.

    Tile t = ((i*N + j)*(N-1) + k')*(N-1) + n' where k' (n') is the rank of k
    among the facilities != i (of n among the locations != j).
    Returns i, j, k, n (int64 arrays of length N^2 (N-1)^2).
    """
    i, j, kk, nn = np.meshgrid(np.arange(N), np.arange(N), np.arange(N - 1), np.arange(N - 1),
                               indexing="ij")
    i, j, kk, nn = (a.reshape(-1) for a in (i, j, kk, nn))
    k = kk + (kk >= i)
    n = nn + (nn >= j)
    return i, j, k, n


def _skip2(r, a, b):
    """r-th element (ascending) of [0, N) with a and b removed (arrays)."""
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    x = r + (r >= lo)
    x = x + (x >= hi)
    return x


def compact_y(c: np.ndarray) -> np.ndarray:
    N = c.shape[0]
    i, j, k, n = tile_indices(N)
    return c[i, j, k, n]


def compact_z(d: np.ndarray) -> np.ndarray:
    """[tiles, N-2, N-2] view of the dense d[i,j,k,n,p,q] (rows p, cols q ascending)."""
    N = d.shape[0]
    i, j, k, n = tile_indices(N)
    m = N - 2
    r = np.arange(m)
    out = np.empty((len(i), m, m), dtype=d.dtype)
    flat = d.reshape(-1)
    base = ((i * N + j) * N + k) * N + n
    for rr in range(m):
        p = _skip2(np.full_like(i, rr), i, k)
        q = _skip2(r[None, :], j[:, None], n[:, None])
        out[:, rr, :] = flat[(base * N + p)[:, None] * N + q]
    return out


def qap_cost(F, D, perm, B_lin=None, const=0):
    """Q(pi) = sum_{i != k} F[i,k] D[pi_i, pi_k] (+ linear and constant terms)."""
    perm = np.asarray(perm)
    F = np.asarray(F, np.int64)
    D = np.asarray(D, np.int64)
    Q = (F * D[np.ix_(perm, perm)]).sum() - (np.diag(F) * np.diag(D)[perm]).sum()
    if B_lin is not None:
        Q += np.asarray(B_lin, np.int64)[np.arange(len(perm)), perm].sum()
    return int(Q + const)


def reduced_along(perm, LB, b, c, d=None):
    """LB + sum of the reduced costs that the solution pi uses (Eq. (5))."""
    perm = np.asarray(perm)
    N = len(perm)
    idx = np.arange(N)
    tot = int(LB) + int(b[idx, perm].sum())
    I, K = np.meshgrid(idx, idx, indexing="ij")
    off = I != K
    tot += int(c[I[off], perm[I[off]], K[off], perm[K[off]]].sum())
    if d is not None:
        I, K, P = np.meshgrid(idx, idx, idx, indexing="ij")
        ok = (I != K) & (I != P) & (K != P)
        I, K, P = I[ok], K[ok], P[ok]
        tot += int(d[I, perm[I], K, perm[K], P, perm[P]].sum())
    return tot


def brute_force_qap(F, D, B_lin=None, const=0):
    """Optimum of the QAP by enumerating all N! permutations (N <= 9)."""
    import itertools
    N = F.shape[0]
    F = np.asarray(F, np.int64)
    D = np.asarray(D, np.int64)
    perms = np.array(list(itertools.permutations(range(N))), dtype=np.int64)
    best = None
    for chunk in np.array_split(perms, max(1, len(perms) // 20000)):
        Dp = D[chunk[:, :, None], chunk[:, None, :]]
        Q = (F[None] * Dp).sum(axis=(1, 2)) - (np.diag(F)[None] * np.diag(D)[chunk]).sum(1)
        if B_lin is not None:
            Q = Q + np.asarray(B_lin, np.int64)[np.arange(N)[None, :], chunk].sum(1)
        m = int(Q.min())
        best = m if best is None else min(best, m)
    return best + const


_K1 = np.uint64(0x9E3779B97F4A7C15)
_K2 = np.uint64(0x632BE59BD9B4E019)


def state_hash(a) -> int:
    """Order-sensitive 64-bit hash of an integer array: sum_e a_e * w_e (mod 2^64),
    w_e = (e * K1 + K2) | 1 odd, so any single changed entry changes the hash."""
    a = np.ascontiguousarray(a).reshape(-1)
    h = np.uint64(0)
    step = 1 << 22
    with np.errstate(over="ignore"):
        for s in range(0, a.size, step):
            e = np.arange(s, min(s + step, a.size), dtype=np.uint64)
            w = (e * _K1 + _K2) | np.uint64(1)
            h = h + (a[s:s + step].astype(np.int64).astype(np.uint64) * w).sum(dtype=np.uint64)
    return int(h)
