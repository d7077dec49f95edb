"""Pins of the oracle's FP64 form (reading R14: the paper's real division,
Sec. 4.2; class sums re-split as T/s, Sec. 4.3) against facts fixed outside it.

* Integer-valued inputs: the FP64 Hungarian is exact on integers below 2^53,
  so on integer matrices it must take every decision of the int64 Hungarian
  (itself pinned by hand traces and enumeration) and return the same S,
  assignment, duals and work counts.
* Exact divisions: on instances whose flows are multiples of 12 (N - 2) every
  division of the first pass is exact and every class sum is divisible by its
  class size, where the integer split of reading R3/R4 and the real division
  coincide: the whole first pass, operation by operation, must equal the
  int64 form element by element.
* N!-enumeration on real-valued matrices: S is the minimum and (u, v) a dual
  certificate up to rounding.
* Conservation (every operation keeps each solution's cost): Q(pi) equals LB
  plus the reduced costs along pi, up to rounding, for every permutation.
* RLT1 special case: the first pass on symmetric F, D gives the
  Gilmore-Lawler bound (scipy), exactly.
* LB stays below the brute-force optimum and never decreases (up to rounding).
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from paper_1510_02065_gb300 import instances as I
from tests.layout import brute_force_qap

OPS = ["spread_B_to_C", "spread_C_to_D", "complementary_D", "concentrate_D_to_C",
       "complementary_C", "concentrate_C_to_B", "concentrate_B_to_LB"]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 20])
def test_lap_equals_int_form_on_integers(orc, n):
    rng = np.random.default_rng(n)
    for trial in range(25):
        hi = [2, 5, 100, 10**6][trial % 4]
        M = rng.integers(0, hi, (n, n))
        S, sig, u, v, work = orc.lap(M)
        Sf, sigf, uf, vf, workf = orc.lap_f64(M.astype(np.float64))
        assert Sf == S and (sigf == sig).all() and work == workf
        assert (uf == u).all() and (vf == v).all()


def _certificate(M, S, sig, u, v, tol):
    n = M.shape[0]
    R = M - u[:, None] - v[None, :]
    assert R.min() >= -tol
    assert np.abs(R[np.arange(n), sig]).max() <= tol
    assert abs(u.sum() + v.sum() - S) <= tol * n
    assert sorted(sig) == list(range(n))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_lap_enumeration_real(orc, n):
    rng = np.random.default_rng(100 + n)
    perms = np.array(list(itertools.permutations(range(n))))
    for _ in range(10):
        M = rng.integers(0, 1000, (n, n)) / 7.0
        S, sig, u, v, _ = orc.lap_f64(M)
        best = M[np.arange(n)[None, :], perms].sum(1).min()
        assert abs(S - best) <= 1e-12 * max(1.0, best)
        assert abs(M[np.arange(n), sig].sum() - S) <= 1e-12 * max(1.0, S)
        _certificate(M, S, sig, u, v, 1e-9)


@pytest.mark.parametrize("n", [10, 28, 33])
def test_lap_scipy_real(orc, n):
    rng = np.random.default_rng(200 + n)
    for _ in range(4):
        M = rng.uniform(0, 50, (n, n))
        S, sig, u, v, _ = orc.lap_f64(M)
        r, c = linear_sum_assignment(M)
        assert abs(S - M[r, c].sum()) <= 1e-9 * S
        _certificate(M, S, sig, u, v, 1e-9)


def _divisible(N, seed):
    """Flows multiples of 12 (N - 2): every first-pass division is exact."""
    F, D = I.uniform_symmetric(N, seed=seed, hi=6)
    return (F * 12 * (N - 2)).astype(np.int32), D


@pytest.mark.parametrize("N,seed", [(4, 0), (5, 1), (6, 2), (7, 3)])
def test_first_pass_equals_int_form_when_divisions_are_exact(orc, N, seed):
    F, D = _divisible(N, seed)
    a = orc.State(F, D)
    f = orc.StateF64(F, D)
    for op in OPS:
        ra = getattr(a, op)()
        rf = getattr(f, op)()
        if op == "concentrate_B_to_LB":
            assert rf == ra
        assert (f.b == a.b).all(), op
        assert (f.c == a.c).all(), op
        assert (f.d == a.d).all(), op
    assert f.work() == {k: v for k, v in a.work().items() if k != "max_abs"}


def _conservation(F, D, st, perms):
    N = st.N
    P = np.asarray(perms)
    idx = np.arange(N)
    F64 = np.asarray(F, np.float64)
    D64 = np.asarray(D, np.float64)
    Q = (F64[None] * D64[P[:, :, None], P[:, None, :]]).sum((1, 2))
    Q -= (np.diag(F64)[None] * np.diag(D64)[P]).sum(1)
    tot = st.LB + st.b[idx[None, :], P].sum(1)
    I_, K_ = np.meshgrid(idx, idx, indexing="ij")
    off = I_ != K_
    Ii, Kk = I_[off], K_[off]
    tot = tot + st.c[Ii[None, :], P[:, Ii], Kk[None, :], P[:, Kk]].sum(1)
    if st.d is not None:
        I3, K3, P3 = np.meshgrid(idx, idx, idx, indexing="ij")
        ok = (I3 != K3) & (I3 != P3) & (K3 != P3)
        I3, K3, P3 = I3[ok], K3[ok], P3[ok]
        tot = tot + st.d[I3[None, :], P[:, I3], K3[None, :], P[:, K3], P3[None, :], P[:, P3]].sum(1)
    return float(np.abs(Q - tot).max() / max(1.0, Q.max()))


@pytest.mark.parametrize("rlt1", [False, True])
@pytest.mark.parametrize("N,seed", [(4, 0), (5, 1), (6, 2)])
def test_conservation_every_operation(orc, N, seed, rlt1):
    # With D present, the six-way transfer makes complementary submatrices of D
    # equal, so the transfer on C moves nothing; in RLT1 mode (no D) it does.
    F, D = I.uniform_symmetric(N, seed=seed)
    F[0, 1] += 1  # asymmetric flows: the complementary transfers move real amounts
    st = orc.StateF64(F, D, rlt1_only=rlt1)
    perms = list(itertools.permutations(range(N)))
    ops = [op for op in OPS if not (rlt1 and op.endswith("_D") or rlt1 and op == "concentrate_D_to_C")]
    for it in range(3):
        for op in ops:
            r = getattr(st, op)()
            if op == "concentrate_B_to_LB":
                st.add_LB(r)
            assert _conservation(F, D, st, perms) <= 1e-12, (it, op)
    assert st.b.min() >= -1e-9 and st.c.min() >= -1e-9
    assert rlt1 or st.d.min() >= -1e-9


def test_rlt1_first_pass_is_gilmore_lawler(orc):
    for seed in range(4):
        F, D = I.uniform_symmetric(7, seed=seed)
        st = orc.StateF64(F, D, rlt1_only=True)
        lb = st.iterate()
        N = 7
        G = np.zeros((N, N))
        for i in range(N):
            for j in range(N):
                ks = [k for k in range(N) if k != i]
                ns = [n for n in range(N) if n != j]
                M = np.outer(F[i, ks], D[j, ns]).astype(np.float64)
                r, c = linear_sum_assignment(M)
                G[i, j] = M[r, c].sum()
        r, c = linear_sum_assignment(G)
        assert lb == G[r, c].sum()


@pytest.mark.parametrize("N,seed", [(5, 0), (6, 1), (7, 2)])
def test_lb_below_optimum_and_monotone(orc, N, seed):
    F, D = I.uniform_symmetric(N, seed=seed)
    opt = brute_force_qap(F, D)
    st = orc.StateF64(F, D)
    hist = st.run(8)
    assert hist[-1] <= opt * (1 + 1e-12)
    assert (np.diff(hist) >= -1e-9 * opt).all()
    assert hist[-1] > 0


def test_range_forms_equal_whole(orc):
    F, D = I.uniform_symmetric(6, seed=5)
    a = orc.StateF64(F, D)
    b = orc.StateF64(F, D)
    a.iterate()
    b.iterate()
    a.spread_B_to_C()
    b.spread_B_to_C()
    a.spread_C_to_D()
    b.spread_C_to_D_range(0, 2)
    b.spread_C_to_D_range(2, 6)
    a.complementary_D()
    b.complementary_D_range(0, 3)
    b.complementary_D_range(3, 6)
    a.concentrate_D_to_C()
    b.concentrate_D_to_C_range(0, 1)
    b.concentrate_D_to_C_range(1, 6)
    assert (a.c == b.c).all() and (a.d == b.d).all()
