"""Pins of the oracle's Hungarian method against values fixed outside it.

* hand traces of the method on small matrices (the tie-breaking rule of
  reading R6: smallest column among equal distances, labels change only on a
  strict improvement);
* N!-enumeration: S is the minimum over all permutations, sigma attains it,
  and (u, v) is a dual certificate (M - u - v >= 0, zero on sigma,
  sum u + sum v = S) -- the LP duality of the assignment problem;
* scipy.optimize.linear_sum_assignment optimum values for n up to 64;
* the exact duals: started from u = v = 0 the method ends at the optimal dual
  with the largest v subject to v <= 0 (the minimum competitive prices
  p = -v of the assignment market, which an exact ascending auction -- the
  Hungarian method -- reaches whatever the order of the rows).  That dual is
  computed independently: for any optimal assignment sigma (scipy), v_j is
  the shortest distance to column j from a source joined to every column by a
  0-weight edge, in the graph with an edge sigma(i) -> j of weight
  M[i][j] - M[i][sigma(i)] (Bellman-Ford), and u_i = M[i][sigma(i)] -
  v_sigma(i).  This pins (u, v) themselves, not only their optimality.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment


def test_hand_trace_2x2_tie(orc):
    # M = [[1,2],[3,4]]: both assignments cost 5.
    # row 0: dist=[1,2] -> delta 1, column 0 free; u0=1.
    # row 1: dist=[3,4] -> column 0 (matched to row 0), u1=3;
    #        scan row 0: red(col 1) = 2-1-0 = 1, not < dist 1 -> delta 1, column 1 free.
    #        labelled: u1=4, u0=2, v0=-1.  -> identity, u=[2,4], v=[-1,0]
    S, sig, u, v, (steps, relax) = orc.lap(np.array([[1, 2], [3, 4]]))
    assert S == 5
    assert list(sig) == [0, 1]
    assert list(u) == [2, 4] and list(v) == [-1, 0]
    assert (steps, relax) == (3, 5)


def test_hand_trace_3x3(orc):
    # M = [[4,1,3],[2,0,5],[3,2,2]], optimum 1+2+2 = 5.
    # row 0: dist [4,1,3] -> column 1 (u0=1).
    # row 1: dist [2,0,5] -> column 1 (row 0); scan row 0: red [3,-,2]:
    #        dist [2,-,2] -> tie at 2, column 0 wins; u1=2, u0=3, v1=-2.
    # row 2: dist [3,4,2] -> column 2 free, u2=2.
    S, sig, u, v, (steps, relax) = orc.lap(np.array([[4, 1, 3], [2, 0, 5], [3, 2, 2]]))
    assert S == 5
    assert list(sig) == [1, 0, 2]
    assert list(u) == [3, 2, 2] and list(v) == [0, -2, 0]
    assert (steps, relax) == (4, 11)


def test_hand_trace_all_zero(orc):
    # every distance ties at 0: columns are taken in ascending order, no potential moves
    S, sig, u, v, (steps, relax) = orc.lap(np.zeros((3, 3), np.int64))
    assert S == 0 and list(sig) == [0, 1, 2]
    assert not u.any() and not v.any()
    assert (steps, relax) == (6, 14)


def _check_certificate(M, S, sig, u, v):
    n = M.shape[0]
    red = M - u[:, None] - v[None, :]
    assert (red >= 0).all()
    assert (red[np.arange(n), sig] == 0).all()
    assert u.sum() + v.sum() == S
    assert sorted(sig) == list(range(n))
    assert M[np.arange(n), sig].sum() == S


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("hi", [2, 9, 1000])
def test_enumeration(orc, n, hi):
    rng = np.random.default_rng(100 * n + hi)
    perms = np.array(list(itertools.permutations(range(n))))
    count = 60 if n <= 6 else 15
    Ms = rng.integers(0, hi + 1, size=(count, n, n))
    S, sig, u, v, work = orc.lap_batch(Ms)
    for t in range(count):
        M = Ms[t]
        best = M[np.arange(n)[None, :], perms].sum(1).min()
        assert S[t] == best
        _check_certificate(M, S[t], sig[t], u[t], v[t])
        # every row insertion takes at least one step and at most (rows so far) + 1
        assert n <= work[t, 0] <= n * (n + 1) // 2


@pytest.mark.parametrize("n", [8, 10, 18, 28, 29, 30, 33, 35, 64])
def test_scipy_values(orc, n):
    rng = np.random.default_rng(n)
    Ms = np.concatenate([rng.integers(0, 50, size=(8, n, n)),
                         rng.integers(0, 3, size=(4, n, n)),        # many ties
                         (rng.random((4, n, n)) < 0.7) * rng.integers(1, 10**6, size=(4, n, n))])
    S, sig, u, v, _ = orc.lap_batch(Ms)
    for t in range(len(Ms)):
        r, c = linear_sum_assignment(Ms[t])
        assert S[t] == Ms[t][r, c].sum()
        _check_certificate(Ms[t], S[t], sig[t], u[t], v[t])


def test_batch_equals_single(orc):
    rng = np.random.default_rng(5)
    Ms = rng.integers(0, 20, size=(10, 9, 9))
    S, sig, u, v, _ = orc.lap_batch(Ms)
    for t in range(10):
        s1, g1, u1, v1, _ = orc.lap(Ms[t])
        assert s1 == S[t] and (g1 == sig[t]).all() and (u1 == u[t]).all() and (v1 == v[t]).all()


def _minimum_price_duals(M):
    n = M.shape[0]
    r, c = linear_sum_assignment(M)
    sig = np.empty(n, np.int64)
    sig[r] = c
    row_of = np.empty(n, np.int64)
    row_of[c] = r
    W = M[row_of, :] - M[row_of, np.arange(n)][:, None]   # W[k, j]: edge k -> j
    d = np.zeros(n, np.int64)
    for _ in range(n + 1):
        nd = np.minimum(d, (d[:, None] + W).min(0))
        if (nd == d).all():
            break
        d = nd
    assert (nd == d).all()  # no negative cycle: sigma is optimal
    return M[np.arange(n), sig] - d[sig], d


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 18, 28, 33])
def test_duals_are_the_minimum_price_duals(orc, n):
    rng = np.random.default_rng(700 + n)
    Ms = np.concatenate([rng.integers(0, 3, size=(40, n, n)),         # heavy ties
                         rng.integers(0, 20, size=(40, n, n)),
                         rng.integers(0, 10**6, size=(20, n, n))])
    S, sig, u, v, _ = orc.lap_batch(Ms)
    for t in range(len(Ms)):
        cu, cv = _minimum_price_duals(Ms[t])
        assert (u[t] == cu).all() and (v[t] == cv).all(), t
