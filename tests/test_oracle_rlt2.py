"""Pins of the oracle's RLT2 dual ascent (Algorithm 1) against facts fixed outside it.

* Conservation (Sec. 4: every operation keeps the cost of every feasible
  solution): Q(pi) = LB + b along pi + c along pi + d along pi, for every
  permutation pi, after each of the seven operations.  Exact in integers and
  independent of every tie-break; a dropped term, a wrong index or a wrong
  share anywhere breaks it.
* Dual feasibility: all reduced costs stay >= 0 (Sec. 4); hence LB is
  monotone and never exceeds the brute-force QAP optimum.
* RLT1 special case (Sec. 6, strong branching): on symmetric F, D with no
  linear term the first pass gives the Gilmore-Lawler bound, computed here
  independently with scipy.
* The lexicographic rank of Eq. (11)'s six complementary coefficients,
  checked against Python's own tuple ordering.
* Hand-derived integer spreading (reading R3) on a one-entry B.
* The subproblem (fixed assignments) reduction against brute force.
* Every value the method produces stays below 4U, the bound the int32 guard
  of the library relies on.
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from paper_1510_02065_gb300 import instances as I
from tests.layout import brute_force_qap, qap_cost

OPS = ["spread_B_to_C", "spread_C_to_D", "complementary_D", "concentrate_D_to_C",
       "complementary_C", "concentrate_C_to_B", "concentrate_B_to_LB"]


def conservation_residual(F, D, st, perms, B_lin=None, const=0):
    """max over perms of |Q(pi) - (LB + reduced costs along pi)| (vectorised)."""
    N = st.N
    P = np.asarray(perms)
    idx = np.arange(N)
    F64 = np.asarray(F, np.int64)
    D64 = np.asarray(D, np.int64)
    Q = (F64[None] * D64[P[:, :, None], P[:, None, :]]).sum((1, 2))
    Q -= (np.diag(F64)[None] * np.diag(D64)[P]).sum(1)
    if B_lin is not None:
        Q += np.asarray(B_lin, np.int64)[idx[None, :], P].sum(1)
    Q += const
    tot = np.full(len(P), st.LB, np.int64) + st.b[idx[None, :], P].sum(1)
    I_, K_ = np.meshgrid(idx, idx, indexing="ij")
    off = I_ != K_
    Ii, Kk = I_[off], K_[off]
    tot += st.c[Ii[None, :], P[:, Ii], Kk[None, :], P[:, Kk]].sum(1)
    if st.d is not None:
        I3, K3, P3 = np.meshgrid(idx, idx, idx, indexing="ij")
        ok = (I3 != K3) & (I3 != P3) & (K3 != P3)
        I3, K3, P3 = I3[ok], K3[ok], P3[ok]
        tot += st.d[I3[None, :], P[:, I3], K3[None, :], P[:, K3], P3[None, :], P[:, P3]].sum(1)
    return int(np.abs(Q - tot).max())


def _meaningless_masks(N):
    idx = np.arange(N)
    i, j, k, n = np.meshgrid(idx, idx, idx, idx, indexing="ij")
    mc = (i == k) | (j == n)
    i, j, k, n, p, q = np.meshgrid(idx, idx, idx, idx, idx, idx, indexing="ij")
    md = (i == k) | (i == p) | (k == p) | (j == n) | (j == q) | (n == q)
    return mc, md


def nonneg(st):
    """All reduced costs >= 0 and every entry without meaning (a repeated
    facility or location) still 0."""
    ok = (st.b >= 0).all() and (st.c >= 0).all()
    mc, md = _meaningless_masks(st.N)
    ok = ok and not st.c[mc].any()
    if st.d is not None:
        ok = ok and (st.d >= 0).all() and not st.d[md].any()
    return ok


def step_all(st, F, D, perms, B_lin=None, const=0):
    """Run one pass operation by operation, checking conservation after each."""
    for op in OPS:
        r = getattr(st, op)()
        if op == "concentrate_B_to_LB":
            st.add_LB(r)
        assert conservation_residual(F, D, st, perms, B_lin, const) == 0, op
        assert nonneg(st), op


@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (5, 2), (6, 3)])
def test_conservation_every_operation_all_perms(orc, N, seed):
    F, D = I.uniform_symmetric(N, seed=seed)
    perms = list(itertools.permutations(range(N)))
    st = orc.State(F, D)
    assert conservation_residual(F, D, st, perms) == 0
    lbs = []
    for _ in range(6):
        step_all(st, F, D, perms)
        lbs.append(st.LB)
    assert all(a <= b for a, b in zip(lbs, lbs[1:]))
    assert lbs[-1] <= brute_force_qap(F, D)


def test_conservation_asymmetric_with_linear_term(orc):
    rng = np.random.default_rng(11)
    N = 6
    F = rng.integers(0, 8, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 8, size=(N, N)).astype(np.int32)
    np.fill_diagonal(F, 0)
    np.fill_diagonal(D, 0)
    Bl = rng.integers(0, 30, size=(N, N))
    perms = list(itertools.permutations(range(N)))
    st = orc.State(F, D, B_lin=Bl, lb_const=17)
    for _ in range(4):
        step_all(st, F, D, perms, Bl, 17)
    assert st.LB <= brute_force_qap(F, D, Bl, 17)


def test_uniform_n8_bound_below_optimum(orc):
    F, D, iters = I.instance("uniform_n8")
    opt = brute_force_qap(F, D)
    st = orc.State(F, D)
    hist = st.run(iters)
    assert (np.diff(hist) >= 0).all()
    assert hist[-1] <= opt
    assert nonneg(st)
    rng = np.random.default_rng(0)
    perms = np.array([rng.permutation(8) for _ in range(2000)])
    assert conservation_residual(F, D, st, perms) == 0


def test_rlt1_first_pass_is_gilmore_lawler(orc):
    for N, seed in [(6, 0), (9, 1), (12, 2)]:
        F, D = I.uniform_symmetric(N, seed=seed)
        st = orc.State(F, D, rlt1_only=True)
        lb1 = st.iterate()
        # Gilmore-Lawler: L_ij = LAP over (F_ik D_jn)_{k != i, n != j}; GLB = LAP(L)
        L = np.zeros((N, N), np.int64)
        for i in range(N):
            for j in range(N):
                ks = [k for k in range(N) if k != i]
                ns = [n for n in range(N) if n != j]
                M = np.outer(F[i, ks].astype(np.int64), D[j, ns].astype(np.int64))
                r, c = linear_sum_assignment(M)
                L[i, j] = M[r, c].sum()
        r, c = linear_sum_assignment(L)
        assert lb1 == L[r, c].sum()


def test_complementary_D_lexicographic_rank(orc):
    """After the transfer, a class's members are floor(T/6) + [rank < T mod 6],
    rank taken from Python's ordering of the six index tuples."""
    N = 5
    F, D = I.uniform_symmetric(N, seed=4)
    st = orc.State(F, D)
    st.spread_B_to_C()
    st.spread_C_to_D()
    rng = np.random.default_rng(1)
    d = st.d
    # scramble D so that class sums leave every remainder, then transfer
    valid = np.zeros_like(d, dtype=bool)
    for i, j, k, n, p, q in itertools.product(range(N), repeat=6):
        if len({i, k, p}) == 3 and len({j, n, q}) == 3:
            valid[i, j, k, n, p, q] = True
    d[valid] = rng.integers(0, 50, size=int(valid.sum()))
    before = d.copy()
    st.complementary_D()
    seen = set()
    rems = set()
    for i, j, k, n, p, q in zip(*np.nonzero(valid)):
        pairs = ((i, j), (k, n), (p, q))
        key = frozenset(pairs)
        if key in seen:
            continue
        seen.add(key)
        members = sorted(tuple(x for pr in order for x in pr)
                         for order in itertools.permutations(pairs))
        T = sum(int(before[m]) for m in members)
        rems.add(T % 6)
        for rank, m in enumerate(members):
            assert d[m] == T // 6 + (1 if rank < T % 6 else 0)
    assert len(seen) == 10 * 60    # C(5,3) facility triples x 5*4*3 location triples
    assert rems == set(range(6))


def test_complementary_C_first_member_takes_odd_unit(orc):
    N = 4
    F = np.array([[0, 1, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]], np.int32)
    D = np.array([[0, 3, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]], np.int32)
    st = orc.State(F, D)
    # c_0011 = F01 * D01 = 3, its complement c_1100 = F10 * D10 = 0
    assert st.c[0, 0, 1, 1] == 3 and st.c[1, 1, 0, 0] == 0
    st.complementary_C()
    assert st.c[0, 0, 1, 1] == 2 and st.c[1, 1, 0, 0] == 1


def test_spread_integer_shares_by_hand(orc):
    N = 4
    Z = np.zeros((N, N), np.int32)
    Bl = np.zeros((N, N), np.int64)
    Bl[1, 2] = 5            # spread over the N-1 = 3 rows k in {0, 2, 3}: 2, 2, 1
    st = orc.State(Z, Z, B_lin=Bl)
    st.spread_B_to_C()
    assert st.b[1, 2] == 0
    for k, share in zip([0, 2, 3], [2, 2, 1]):
        for n in [0, 1, 3]:
            assert st.c[1, 2, k, n] == share
    assert st.c.sum() == 5 * 3
    # c_1203 = 2 spread over the N-2 = 2 rows p in {1, 2}: 1, 1
    st.spread_C_to_D()
    assert st.c.sum() == 0
    # c_1,2,0,0 = 2 goes to rows p in {2, 3} (p not in {1, 0}), columns q not in {2, 0}
    assert st.d[1, 2, 0, 0, 2, 1] == 1 and st.d[1, 2, 0, 0, 3, 3] == 1
    # c_1,2,3,1 = 1 over rows {0, 2}: 1, 0
    assert st.d[1, 2, 3, 1, 0, 0] == 1 and st.d[1, 2, 3, 1, 2, 0] == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_subproblem_reduction_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    N = 7
    F = rng.integers(0, 9, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 9, size=(N, N)).astype(np.int32)
    np.fill_diagonal(F, 0)
    np.fill_diagonal(D, 0)
    k = 2 + seed
    fac = rng.choice(N, size=k, replace=False)
    loc = rng.choice(N, size=k, replace=False)
    Fp, Dp, Bl, cst = orc.subproblem(F, D, fac, loc)
    free_f = [a for a in range(N) if a not in fac]
    free_l = [l for l in range(N) if l not in loc]
    for perm in itertools.permutations(range(N - k)):
        full = np.empty(N, np.int64)
        full[fac] = loc
        full[free_f] = np.array(free_l)[list(perm)]
        assert qap_cost(F, D, full) == qap_cost(Fp, Dp, perm, Bl, cst)
    # the bound of the node never exceeds the best completion
    st = orc.State(Fp, Dp, B_lin=Bl, lb_const=cst)
    hist = st.run(5)
    assert hist[-1] <= brute_force_qap(Fp, Dp, Bl, cst)


@pytest.mark.parametrize("name,iters", [("uniform_n8", 50), ("grid_n12", 20)])
def test_values_stay_below_guard(orc, name, iters):
    F, D, _ = I.instance(name)
    N = F.shape[0]
    off = ~np.eye(N, dtype=bool)
    U = int(F[off].astype(np.int64).sum()) * int(D[off].max())
    st = orc.State(F, D)
    st.run(iters)
    assert 0 < st.work()["max_abs"] <= 4 * U


@pytest.mark.slow
def test_clustered_n20_first_passes(orc):
    F, D, _ = I.instance("clustered_n20")
    st = orc.State(F, D)
    hist = st.run(2)
    assert hist[0] > 0 and hist[1] >= hist[0]
    assert nonneg(st)
    rng = np.random.default_rng(3)
    perms = np.array([rng.permutation(20) for _ in range(200)])
    assert conservation_residual(F, D, st, perms) == 0


# ---------------------------------------------------------------- paired form

def _lower_tiles_zero(st):
    """Paired form (reading R13): every submatrix D_ijkn with i > k stays 0."""
    N = st.N
    idx = np.arange(N)
    i = idx[:, None, None, None]
    k = idx[None, None, :, None]
    low = np.broadcast_to(i > k, (N, N, N, N))
    return not st.d[low].any()


@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (5, 2), (6, 3)])
def test_paired_conservation_every_operation_all_perms(orc, N, seed):
    """The complementary-submatrix form keeps every solution's cost after each
    operation, keeps the reduced costs >= 0 and the other half of D at 0, and
    bounds the optimum."""
    F, D = I.uniform_symmetric(N, seed=seed)
    perms = list(itertools.permutations(range(N)))
    st = orc.State(F, D, paired=True)
    lbs = []
    for _ in range(6):
        step_all(st, F, D, perms)
        assert _lower_tiles_zero(st)
        lbs.append(st.LB)
    assert all(a <= b for a, b in zip(lbs, lbs[1:]))
    assert lbs[-1] <= brute_force_qap(F, D)


def test_paired_asymmetric_linear_term_and_half_the_laps(orc):
    rng = np.random.default_rng(12)
    N = 6
    F = rng.integers(0, 8, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 8, size=(N, N)).astype(np.int32)
    np.fill_diagonal(F, 0)
    np.fill_diagonal(D, 0)
    Bl = rng.integers(0, 30, size=(N, N))
    perms = list(itertools.permutations(range(N)))
    st = orc.State(F, D, B_lin=Bl, lb_const=9, paired=True)
    full = orc.State(F, D, B_lin=Bl, lb_const=9)
    for _ in range(3):
        step_all(st, F, D, perms, Bl, 9)
        full.iterate()
    assert st.LB <= brute_force_qap(F, D, Bl, 9)
    # per pass: N^2 (N-1)^2 / 2 D-LAPs + N^2 C-LAPs + 1, against N^2 (N-1)^2 + N^2 + 1
    per_pass = N * N * (N - 1) ** 2
    assert st.work()["laps"] == 3 * (per_pass // 2 + N * N + 1)
    assert full.work()["laps"] == 3 * (per_pass + N * N + 1)


def test_paired_three_way_split_by_hand(orc):
    """One class of N = 3 (the only one: facilities 0 < 1 < 2, locations
    0, 1, 2): after spreading c (from one unit of flow) and the 3-way split,
    the three members with first facility below the second hold T split as
    floor(T/3) + [t < T mod 3] in lexicographic order, the other three 0."""
    F = np.zeros((3, 3), np.int32)
    D = np.zeros((3, 3), np.int32)
    F[0, 1] = 7          # c_{0j1n} = 7 * D[j,n]
    D[0, 1] = D[1, 0] = 1
    st = orc.State(F, D, paired=True)
    st.spread_B_to_C()
    st.spread_C_to_D()
    d = st.d
    # the pair (i,j,k,n) = (0,0,1,1) and (0,1,1,0) carry c = 7; one row p = 2
    # with one column q = 2: d_{0,0,1,1,2,2} = 7 and d_{0,1,1,0,2,2} = 7
    assert d[0, 0, 1, 1, 2, 2] == 7 and d[0, 1, 1, 0, 2, 2] == 7
    st.complementary_D()
    # class {(0,0),(1,1),(2,2)}: T = 7; members d_001122, d_002211, d_112200 get 3, 2, 2
    assert (d[0, 0, 1, 1, 2, 2], d[0, 0, 2, 2, 1, 1], d[1, 1, 2, 2, 0, 0]) == (3, 2, 2)
    assert (d[1, 1, 0, 0, 2, 2], d[2, 2, 0, 0, 1, 1], d[2, 2, 1, 1, 0, 0]) == (0, 0, 0)
    # class {(0,1),(1,0),(2,2)}: T = 7 as well
    assert (d[0, 1, 1, 0, 2, 2], d[0, 1, 2, 2, 1, 0], d[1, 0, 2, 2, 0, 1]) == (3, 2, 2)


def test_paired_uniform_n8_below_optimum(orc):
    F, D, iters = I.instance("uniform_n8")
    opt = brute_force_qap(F, D)
    st = orc.State(F, D, paired=True)
    hist = st.run(iters)
    assert (np.diff(hist) >= 0).all() and hist[-1] <= opt
    assert nonneg(st) and _lower_tiles_zero(st)
    rng = np.random.default_rng(1)
    perms = np.array([rng.permutation(8) for _ in range(2000)])
    assert conservation_residual(F, D, st, perms) == 0


# ------------------------------------------------------------- warm start

@pytest.mark.parametrize("paired", [False, True])
@pytest.mark.parametrize("N,seed,f,l", [(5, 0, 1, 3), (6, 1, 0, 5), (6, 2, 4, 2)])
def test_child_conserves_every_completion(orc, N, seed, f, l, paired):
    """The warm-started child of a node fixing f -> l: for every permutation
    with pi(f) = l, Q(pi) equals the child's LB plus its reduced costs along
    the restricted permutation (child indices renumbered in ascending order);
    the child's reduced costs are >= 0, its bound starts at or above the
    parent's and stays below the optimum of the node after further passes."""
    F, D = I.uniform_symmetric(N, seed=seed)
    par = orc.State(F, D, paired=paired)
    par.run(3)
    ch = par.child(f, l)
    assert ch.N == N - 1 and ch.LB >= par.LB
    fa = [a for a in range(N) if a != f]
    lo = [a for a in range(N) if a != l]
    perms = []
    for rest in itertools.permutations(lo):
        perms.append(list(rest))
    # the child's permutation pi' maps child facility x to child location index of pi(fa[x])
    child_perms = [[lo.index(v) for v in p] for p in perms]
    full = []
    for p in perms:
        q = np.empty(N, np.int64)
        q[f] = l
        q[fa] = p
        full.append(q)
    Q = np.array([qap_cost(F, D, q) for q in full])
    for _ in range(3):
        st_pass = np.array(child_perms)
        # residual of the child's identity: its own conservation against the full Q
        resid = conservation_residual_vs(ch, st_pass, Q)
        assert resid == 0
        assert nonneg(ch)
        ch.iterate()
    node_opt = int(Q.min())
    assert ch.LB <= node_opt


def conservation_residual_vs(st, P, Q):
    """max |Q - (LB + reduced costs along the permutations P)| for a state."""
    N = st.N
    idx = np.arange(N)
    tot = np.full(len(P), st.LB, np.int64) + st.b[idx[None, :], P].sum(1)
    I_, K_ = np.meshgrid(idx, idx, indexing="ij")
    off = I_ != K_
    Ii, Kk = I_[off], K_[off]
    tot += st.c[Ii[None, :], P[:, Ii], Kk[None, :], P[:, Kk]].sum(1)
    if st.d is not None:
        I3, K3, P3 = np.meshgrid(idx, idx, idx, indexing="ij")
        ok = (I3 != K3) & (I3 != P3) & (K3 != P3)
        I3, K3, P3 = I3[ok], K3[ok], P3[ok]
        tot += st.d[I3[None, :], P[:, I3], K3[None, :], P[:, K3], P3[None, :], P[:, P3]].sum(1)
    return int(np.abs(np.asarray(Q, np.int64) - tot).max())
