"""Parity of the CUDA dual ascent (rlt2_create / rlt2_iterate) with the oracle.

* full state (B, C, D in the compact layouts) and LB after every pass, bit for
  bit, on the 8- and 12-facility workloads and on small ragged cases (N = 3..7,
  asymmetric costs, linear terms, constants);
* the 20-facility workload: two passes against the live oracle, then all 200
  passes against the stored LB history and state hashes written by
  tests/golden/make_golden.py (oracle only);
* RLT1 mode (no D) up to N = 40, which exercises two column slots per lane in
  the C -> B and B -> LB kernels;
* the stopping rule of Algorithm 1;
* the 30-facility headline workload in the launch configuration the benchmark
  times, and a 34-facility instance (two column slots per lane, two-location
  chunks): the first pass against the oracle, later passes through properties
  that hold at any size (conservation on sampled permutations, non-negative
  reduced costs, monotone LB).
"""
import json
import os

import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from tests.layout import compact_y, compact_z, state_hash, tile_indices

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STORES = [rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_CLASSES]


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


def assert_same_state(ctx, st, where=""):
    N = st.N
    x, y = ctx.state(0), ctx.state(1)
    assert (x == st.b.reshape(-1)).all(), "B differs " + where
    assert (y == compact_y(st.c)).all(), "C differs " + where
    if st.d is not None:
        z = ctx.state(2).reshape(-1, N - 2, N - 2)
        zo = compact_z(st.d)
        bad = np.nonzero(z != zo)
        assert bad[0].size == 0, "D differs %s at %d entries, first tile %s" % (
            where, bad[0].size, bad[0][:3])
    assert ctx.bound()[1] == st.LB, where


@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("name", ["uniform_n8", "grid_n12"])
def test_full_state_every_pass(gpu, orc, name, store):
    F, D, iters = I.instance(name)
    st = orc.State(F, D)
    with rlt2.Context(F, D, store=store) as ctx:
        assert_same_state(ctx, st, "at init")
        for t in range(iters):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))
        gold = json.load(open(os.path.join(GOLDEN, "lb_%s.json" % name)))
        assert list(ctx.history()) == gold["lb"]
        w = ctx.work()
        ow = st.work()
        assert (w["laps"], w["steps"], w["relaxations"]) == (ow["laps"], ow["steps"], ow["relaxations"])


@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (5, 2), (6, 3), (7, 4)])
def test_small_ragged_asymmetric_with_linear_term(gpu, orc, N, seed, store):
    rng = np.random.default_rng(seed)
    F = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    Bl = rng.integers(0, 40, size=(N, N)).astype(np.int32)
    st = orc.State(F, D, B_lin=Bl, lb_const=123)
    with rlt2.Context(F, D, B_lin=Bl, lb_const=123, use_graph=(seed % 2 == 0), store=store) as ctx:
        assert_same_state(ctx, st, "at init")
        for t in range(8):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))


def test_subproblem_node(gpu, orc):
    F, D = I.clustered_euclid(14, seed=5)
    fac = np.array([3, 9, 0], np.int32)
    loc = np.array([7, 1, 12], np.int32)
    Fp, Dp, Bl, cst = orc.subproblem(F, D, fac, loc)
    st = orc.State(Fp, Dp, B_lin=Bl, lb_const=cst)
    with rlt2.Context(Fp, Dp, B_lin=Bl.astype(np.int32), lb_const=cst) as ctx:
        ctx.iterate(6)
        ref = st.run(6)
        assert list(ctx.history()) == list(ref)
        assert_same_state(ctx, st, "after 6 passes")


def test_graph_nograph_profile_agree(gpu, orc):
    F, D = I.uniform_symmetric(9, seed=7)
    hs = []
    for kw in (dict(use_graph=True), dict(use_graph=False), dict(profile=True),
               dict(profile=True, use_graph=False)):
        with rlt2.Context(F, D, **kw) as ctx:
            ctx.iterate(5)
            hs.append(list(ctx.history()))
            if kw.get("profile"):
                ms, passes = ctx.stage_times()
                assert passes == 5 and all(m >= 0 for m in ms) and ms[1] > 0
    assert hs[0] == hs[1] == hs[2] == hs[3] == list(orc.State(F, D).run(5))


@pytest.mark.parametrize("store", STORES)
def test_clustered_n20_against_oracle_and_golden(gpu, orc, store):
    F, D, iters = I.instance("clustered_n20")
    gold = json.load(open(os.path.join(GOLDEN, "lb_clustered_n20.json")))
    st = orc.State(F, D)
    with rlt2.Context(F, D, store=store) as ctx:
        for t in range(2):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))
        done = 2
        for t in sorted(int(k) for k in gold["hash"]):
            if t <= done:
                continue
            ctx.iterate(t - done)
            done = t
            h = gold["hash"][str(t)]
            N = 20
            assert state_hash(ctx.state(0)) == h["x"], "B hash after pass %d" % t
            assert state_hash(ctx.state(1)) == h["y"], "C hash after pass %d" % t
            assert state_hash(ctx.state(2).reshape(-1, N - 2, N - 2)) == h["z"], "D hash after %d" % t
        assert done == iters
        assert list(ctx.history()) == gold["lb"]


@pytest.mark.parametrize("N", [12, 20, 33, 34, 40])
def test_rlt1_mode(gpu, orc, N):
    F, D = I.clustered_euclid(N, seed=N)
    st = orc.State(F, D, rlt1_only=True)
    with rlt2.Context(F, D, rlt1_only=True) as ctx:
        for t in range(4):
            ctx.iterate(1)
            st.iterate()
            x, y = ctx.state(0), ctx.state(1)
            assert (x == st.b.reshape(-1)).all()
            assert (y == compact_y(st.c)).all()
            assert ctx.bound()[1] == st.LB


def test_stopping_rule(gpu, orc):
    F, D, _ = I.instance("uniform_n8")
    ref = orc.State(F, D).run(50)
    # UB reached: stop right after the pass whose LB attains it
    with rlt2.Context(F, D, ub=float(ref[2])) as ctx:
        ctx.iterate(20)
        lb, ex, it = ctx.bound()
        assert it == 3 and ex == ref[2]
    # progress below K (LB' / UB < K)
    ub = 690.0
    K = 0.005
    inc = np.diff(np.concatenate([[0], ref]))
    first = int(np.nonzero(inc / ub < K)[0][0])
    with rlt2.Context(F, D, ub=ub, min_progress=K) as ctx:
        ctx.iterate(40)
        lb, ex, it = ctx.bound()
        assert it == first + 1 and ex == ref[first]


def _conservation_sample(F, D, N, LB, x, y, z, perms):
    """max |Q(pi) - (LB + reduced costs along pi)| over the sampled permutations."""
    m, n = N - 1, N - 2
    F64, D64 = F.astype(np.int64), D.astype(np.int64)
    idx = np.arange(N)
    worst = 0
    I3, K3, P3 = np.meshgrid(idx, idx, idx, indexing="ij")
    ok = (I3 != K3) & (I3 != P3) & (K3 != P3)
    I3, K3, P3 = I3[ok], K3[ok], P3[ok]
    I2, K2 = np.meshgrid(idx, idx, indexing="ij")
    o2 = I2 != K2
    I2, K2 = I2[o2], K2[o2]
    for pi in perms:
        Q = int((F64 * D64[np.ix_(pi, pi)]).sum() - (np.diag(F64) * np.diag(D64)[pi]).sum())
        tot = int(LB) + int(x.reshape(N, N)[idx, pi].sum())
        J2, N2 = pi[I2], pi[K2]
        t2 = ((I2 * N + J2) * m + (K2 - (K2 > I2))) * m + (N2 - (N2 > J2))
        tot += int(y[t2].astype(np.int64).sum())
        J, Nn, Q3 = pi[I3], pi[K3], pi[P3]
        t = ((I3 * N + J) * m + (K3 - (K3 > I3))) * m + (Nn - (Nn > J))
        r = P3 - (P3 > I3) - (P3 > K3)
        s = Q3 - (Q3 > J) - (Q3 > Nn)
        tot += int(z[(t * n + r) * n + s].astype(np.int64).sum())
        worst = max(worst, abs(Q - tot))
    return worst


def _first_pass_then_properties(orc, F, D, N, seed, store=rlt2.RLT2_STORE_TILES):
    paired = store == rlt2.RLT2_STORE_PAIRS
    """First pass against the oracle (LB, all of B and C, 200,000 sampled D
    entries), then three passes checked through properties that hold at any
    size: non-negative reduced costs, monotone LB, conservation on 100
    sampled permutations."""
    rng = np.random.default_rng(seed)
    perms = [rng.permutation(N) for _ in range(100)]
    st = orc.State(F, D, paired=paired)
    with rlt2.Context(F, D, store=store) as ctx:
        ctx.iterate(1)
        st.iterate()
        assert ctx.bound()[1] == st.LB
        assert (ctx.state(0) == st.b.reshape(-1)).all()
        assert (ctx.state(1) == compact_y(st.c)).all()
        z = ctx.state(2)
        i, j, k, n = [a.astype(np.int64) for a in tile_indices(N)]
        sel = rng.integers(0, len(i), size=200000)
        rr = rng.integers(0, N - 2, size=sel.size)
        ss = rng.integers(0, N - 2, size=sel.size)
        lo, hi = np.minimum(i[sel], k[sel]), np.maximum(i[sel], k[sel])
        p = rr + (rr >= lo)
        p = p + (p >= hi)
        lo, hi = np.minimum(j[sel], n[sel]), np.maximum(j[sel], n[sel])
        q = ss + (ss >= lo)
        q = q + (q >= hi)
        ref = st.d[i[sel], j[sel], k[sel], n[sel], p, q]
        got = z[(sel * (N - 2) + rr) * (N - 2) + ss]
        assert (got == ref).all()
        st.close()
        hist = [ctx.bound()[1]]
        for t in range(3):
            ctx.iterate(1)
            hist.append(ctx.bound()[1])
        x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
        assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
        assert all(a <= b for a, b in zip(hist, hist[1:]))
        assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0


@pytest.mark.slow
@pytest.mark.parametrize("store", STORES)
def test_headline_n30(gpu, orc, store):
    """The 30-facility workload in the launch configuration the benchmark times."""
    F, D, _ = I.instance("clustered_n30")
    _first_pass_then_properties(orc, F, D, 30, 30, store)


@pytest.mark.slow
@pytest.mark.parametrize("store", STORES)
def test_two_slot_lanes_n34(gpu, orc, store):
    """N = 34: LAPs of size 32 and 33 take two column slots per lane, and the
    fused pass over D works on chunks of two locations with per-piece copies.
    The oracle takes the spreading and complementary operations in full and the
    D -> C concentration on three facility slices (tiles D_ijkn with i in the
    slice); 10^6 sampled entries of those tiles after the first pass must agree,
    then three more passes are checked through properties."""
    N = 34
    F, D = I.clustered_euclid(N, seed=N)
    rng = np.random.default_rng(N)
    perms = [rng.permutation(N) for _ in range(100)]
    st = orc.State(F, D)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    slices = (0, N // 2, N - 1)
    for a in slices:
        st.concentrate_D_to_C_range(a, a + 1)
    with rlt2.Context(F, D, store=store) as ctx:
        ctx.iterate(1)
        z = ctx.state(2)
        i, j, k, n = [a.astype(np.int64) for a in tile_indices(N)]
        per = N * (N - 1) ** 2
        for a in slices:
            sel = a * per + rng.integers(0, per, size=1000000)
            rr = rng.integers(0, N - 2, size=sel.size)
            ss = rng.integers(0, N - 2, size=sel.size)
            lo, hi = np.minimum(i[sel], k[sel]), np.maximum(i[sel], k[sel])
            p = rr + (rr >= lo)
            p = p + (p >= hi)
            lo, hi = np.minimum(j[sel], n[sel]), np.maximum(j[sel], n[sel])
            q = ss + (ss >= lo)
            q = q + (q >= hi)
            ref = st.d[i[sel], j[sel], k[sel], n[sel], p, q]
            got = z[(sel * (N - 2) + rr) * (N - 2) + ss]
            assert (got == ref).all(), "D differs in slice i = %d" % a
        st.close()
        hist = [ctx.bound()[1]]
        for t in range(3):
            ctx.iterate(1)
            hist.append(ctx.bound()[1])
        x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
        assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
        assert all(a <= b for a, b in zip(hist, hist[1:]))
        assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0


def test_stores_agree_and_sizes(gpu, orc):
    """Both stores give the same trajectory (LB history, B, C, D) on an
    instance with a linear term; the class-sum store is the smaller one."""
    F, D = I.clustered_euclid(16, seed=3)
    Bl = np.random.default_rng(3).integers(0, 50, size=(16, 16)).astype(np.int32)
    res = []
    for store in STORES:
        with rlt2.Context(F, D, B_lin=Bl, lb_const=7, store=store) as ctx:
            ctx.iterate(12)
            res.append((list(ctx.history()), ctx.state(0), ctx.state(1), ctx.state(2)))
    assert res[0][0] == res[1][0] == list(orc.State(F, D, B_lin=Bl, lb_const=7).run(12))
    for a, b in zip(res[0][1:], res[1][1:]):
        assert (a == b).all()
    for N in (16, 30, 35, 64):
        assert rlt2.rlt2_state_bytes(N, store=rlt2.RLT2_STORE_CLASSES) < rlt2.rlt2_state_bytes(N)


def test_unknown_store_rejected(gpu):
    F, D = I.uniform_symmetric(6, seed=1)
    with pytest.raises(rlt2.Rlt2Error) as e:
        rlt2.Context(F, D, store=3)
    assert e.value.code == rlt2.RLT2_E_INVAL


def shapes_that_fit(N, store):
    """D->C shapes (opts.lanes, opts.cta_warps) that can solve instances of size N."""
    sh = [dict(lanes=32, cta_warps=w) for w in (4, 16, 32)]
    if N <= 16 and store != rlt2.RLT2_STORE_PAIRS:
        sh.insert(0, dict(lanes=16))
    return sh


@pytest.mark.parametrize("store", STORES + [rlt2.RLT2_STORE_PAIRS])
@pytest.mark.parametrize("N", [5, 8, 13, 16, 17, 21])
def test_every_dlap_shape_agrees(gpu, orc, N, store):
    """D->C in every shape that fits (half-warps for N <= 16 in the tile and
    class-sum stores; whole warps in CTAs of 4, 16 and 32 warps) and in the
    autotuned one gives the same state after every pass, equal to the
    oracle's, and the same Hungarian work counts (LAPs, steps, relaxations)."""
    F, D = I.clustered_euclid(N, seed=40 + N)
    Bl = np.random.default_rng(N).integers(0, 30, size=(N, N)).astype(np.int32)
    paired = store == rlt2.RLT2_STORE_PAIRS
    st = orc.State(F, D, B_lin=Bl, lb_const=3, paired=paired)
    shapes = shapes_that_fit(N, store) + [dict()]
    ctxs = [rlt2.Context(F, D, B_lin=Bl, lb_const=3, store=store, **kw) for kw in shapes]
    try:
        for t in range(6):   # an unmeasured pass and one per candidate shape: tuning is done
            st.iterate()
            for c, kw in zip(ctxs, shapes):
                c.iterate(1)
                if N <= 13:
                    assert_same_state(c, st, "%s, pass %d" % (kw, t + 1))
                else:
                    assert c.bound()[1] == st.LB, kw
                    assert (c.state(1) == compact_y(st.c)).all(), kw
        ow = st.work()
        ref = (ow["laps"], ow["steps"], ow["relaxations"])
        for c, kw in zip(ctxs, shapes):
            w = c.work()
            assert (w["laps"], w["steps"], w["relaxations"]) == ref, kw
            lanes, warps, tuning = c.dlap_shape()
            assert not tuning and lanes in (16, 32) and warps in (4, 16, 32), (kw, lanes, warps)
            if kw:
                assert lanes == kw["lanes"] and warps == kw.get("cta_warps", 4), kw
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("store", STORES)
def test_dlap_shapes_agree_at_size(gpu, store):
    """N = 30: every CTA shape of the whole-warp D->C kernel gives the same LB,
    C and sampled D after each of three passes, and the same work counts
    (pass 1 is checked against the oracle in test_headline_n30)."""
    N = 30
    F, D = I.clustered_euclid(N, seed=N + 5)
    ref = None
    for kw in shapes_that_fit(N, store):
        with rlt2.Context(F, D, store=store, **kw) as c:
            got = []
            for t in range(3):
                c.iterate(1)
                z = c.state(2)
                got.append((c.bound()[1], c.state(1).copy(), z[:: 1 + z.size // 500000].copy()))
            w = c.work()
            got.append((w["laps"], w["steps"], w["relaxations"]))
        if ref is None:
            ref = got
            continue
        for a_, b_ in zip(got[:-1], ref[:-1]):
            assert a_[0] == b_[0], kw
            assert (a_[1] == b_[1]).all() and (a_[2] == b_[2]).all(), kw
        assert got[-1] == ref[-1], kw


def test_tuned_shape_is_remembered(gpu):
    """A context tunes its D->C shape on its first passes and reports it; a
    later context of the same store and row width starts in that shape with
    no tuning passes; a forced shape never tunes."""
    F, D = I.clustered_euclid(19, seed=2)          # W = 20: a width no other test of this module tunes
    with rlt2.Context(F, D, store=rlt2.RLT2_STORE_PAIRS) as a:
        first = a.dlap_shape()
        passes = 0
        while a.dlap_shape()[2] and passes < 8:
            a.iterate(1)
            passes += 1
        assert not a.dlap_shape()[2] and passes <= 6
        tuned = a.dlap_shape()
    F2, D2 = I.clustered_euclid(18, seed=3)        # N = 18: the same row width
    with rlt2.Context(F2, D2, store=rlt2.RLT2_STORE_PAIRS) as b:
        assert b.dlap_shape() == tuned
    with rlt2.Context(F2, D2, store=rlt2.RLT2_STORE_PAIRS, lanes=32, cta_warps=16) as c:
        assert c.dlap_shape() == (32, 16, False)
    assert first[2] or first == tuned


def test_unknown_shapes_rejected(gpu):
    F, D = I.uniform_symmetric(6, seed=1)
    for kw in (dict(lanes=8), dict(lanes=12), dict(cta_warps=5), dict(cta_warps=-1),
               dict(lanes=16, cta_warps=4), dict(lanes=16, store=rlt2.RLT2_STORE_PAIRS)):
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.Context(F, D, **kw)
        assert e.value.code == rlt2.RLT2_E_INVAL, kw
    F, D = I.uniform_symmetric(20, seed=1)
    with pytest.raises(rlt2.Rlt2Error) as e:   # half-warps cover rows of at most 16 columns
        rlt2.Context(F, D, lanes=16)
    assert e.value.code == rlt2.RLT2_E_INVAL


def test_group_rejects_a_context_twice(gpu):
    """Two descriptors of one dual state would race in the same launches."""
    F, D = I.uniform_symmetric(6, seed=1)
    with rlt2.Context(F, D) as a, rlt2.Context(F, D) as b:
        with pytest.raises(rlt2.Rlt2Error) as e:
            rlt2.rlt2_group_create([a.ctx, b.ctx, a.ctx])
        assert e.value.code == rlt2.RLT2_E_INVAL
        g = rlt2.rlt2_group_create([a.ctx, b.ctx])
        rlt2.rlt2_group_destroy(g)


# ------------------------------------------------------------ pair store

PAIRS = rlt2.RLT2_STORE_PAIRS


@pytest.mark.parametrize("name", ["uniform_n8", "grid_n12"])
def test_pairs_full_state_every_pass(gpu, orc, name):
    """The pair store (complementary submatrices of Sec. 6) against the
    oracle's paired form: B, C, D (pair sums in the tiles with i < k, zeros in
    the others) and LB after every pass, and the D->C work (half the LAPs)."""
    F, D, iters = I.instance(name)
    st = orc.State(F, D, paired=True)
    with rlt2.Context(F, D, store=PAIRS) as ctx:
        for t in range(min(iters, 20)):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))
        w, ow = ctx.work(), st.work()
        assert (w["laps"], w["steps"], w["relaxations"]) == (ow["laps"], ow["steps"], ow["relaxations"])


@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (5, 2), (6, 3), (7, 4)])
def test_pairs_small_ragged_with_linear_term(gpu, orc, N, seed):
    rng = np.random.default_rng(seed + 50)
    F = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    Bl = rng.integers(0, 40, size=(N, N)).astype(np.int32)
    st = orc.State(F, D, B_lin=Bl, lb_const=5, paired=True)
    with rlt2.Context(F, D, B_lin=Bl, lb_const=5, store=PAIRS, use_graph=(seed % 2 == 1)) as ctx:
        for t in range(6):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))


def test_pairs_clustered_n20(gpu, orc):
    F, D, _ = I.instance("clustered_n20")
    st = orc.State(F, D, paired=True)
    with rlt2.Context(F, D, store=PAIRS) as ctx:
        for t in range(3):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))


@pytest.mark.slow
def test_pairs_headline_n30(gpu, orc):
    F, D, _ = I.instance("clustered_n30")
    _first_pass_then_properties(orc, F, D, 30, 31, PAIRS)


def _sliced_first_pass_then_properties(orc, F, D, N, store, seed):
    """The oracle's spreading and complementary operations in full and its
    D -> C concentration on three facility slices; 10^6 sampled D entries of
    those slices after the first pass must agree, then three passes are checked
    through properties."""
    paired = store == PAIRS
    rng = np.random.default_rng(seed)
    perms = [rng.permutation(N) for _ in range(100)]
    st = orc.State(F, D, paired=paired)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    slices = (0, N // 2, N - 2 if paired else N - 1)
    for a in slices:
        st.concentrate_D_to_C_range(a, a + 1)
    with rlt2.Context(F, D, store=store) as ctx:
        ctx.iterate(1)
        z = ctx.state(2)
        i, j, k, n = [a.astype(np.int64) for a in tile_indices(N)]
        per = N * (N - 1) ** 2
        for a in slices:
            sel = a * per + rng.integers(0, per, size=1000000)
            rr = rng.integers(0, N - 2, size=sel.size)
            ss = rng.integers(0, N - 2, size=sel.size)
            lo, hi = np.minimum(i[sel], k[sel]), np.maximum(i[sel], k[sel])
            p = rr + (rr >= lo)
            p = p + (p >= hi)
            lo, hi = np.minimum(j[sel], n[sel]), np.maximum(j[sel], n[sel])
            q = ss + (ss >= lo)
            q = q + (q >= hi)
            ref = st.d[i[sel], j[sel], k[sel], n[sel], p, q]
            got = z[(sel * (N - 2) + rr) * (N - 2) + ss]
            assert (got == ref).all(), "D differs in slice i = %d" % a
        st.close()
        hist = [ctx.bound()[1]]
        for t in range(3):
            ctx.iterate(1)
            hist.append(ctx.bound()[1])
        x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
        assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
        assert all(a <= b for a, b in zip(hist, hist[1:]))
        assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0


@pytest.mark.slow
@pytest.mark.parametrize("N,store", [(31, rlt2.RLT2_STORE_TILES), (31, rlt2.RLT2_STORE_CLASSES),
                                     (32, rlt2.RLT2_STORE_TILES), (32, PAIRS)])
def test_column_slot_boundary(gpu, orc, N, store):
    """N = 31: the widest D -> C tiles with one column slot per lane (31
    columns, the LAP's dead column as the sentinel of the packed Hungarian);
    N = 32: the narrowest with two (32 columns, no free lane)."""
    F, D = I.clustered_euclid(N, seed=N + 2)
    _sliced_first_pass_then_properties(orc, F, D, N, store, N)


@pytest.mark.slow
def test_pairs_n34_two_column_slots(gpu, orc):
    """N = 34 in the pair store: two column slots per lane in the LAPs (the
    pair store's fused pass still fits chunks of four locations); the oracle's
    D->C on three facility slices, 10^6 sampled D entries, then properties."""
    N = 34
    F, D = I.clustered_euclid(N, seed=N + 1)
    rng = np.random.default_rng(N)
    perms = [rng.permutation(N) for _ in range(100)]
    st = orc.State(F, D, paired=True)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    slices = (0, N // 2, N - 2)
    for a in slices:
        st.concentrate_D_to_C_range(a, a + 1)
    with rlt2.Context(F, D, store=PAIRS) as ctx:
        ctx.iterate(1)
        z = ctx.state(2)
        i, j, k, n = [a.astype(np.int64) for a in tile_indices(N)]
        per = N * (N - 1) ** 2
        for a in slices:
            sel = a * per + rng.integers(0, per, size=1000000)
            rr = rng.integers(0, N - 2, size=sel.size)
            ss = rng.integers(0, N - 2, size=sel.size)
            lo, hi = np.minimum(i[sel], k[sel]), np.maximum(i[sel], k[sel])
            p = rr + (rr >= lo)
            p = p + (p >= hi)
            lo, hi = np.minimum(j[sel], n[sel]), np.maximum(j[sel], n[sel])
            q = ss + (ss >= lo)
            q = q + (q >= hi)
            ref = st.d[i[sel], j[sel], k[sel], n[sel], p, q]
            got = z[(sel * (N - 2) + rr) * (N - 2) + ss]
            assert (got == ref).all(), "D differs in slice i = %d" % a
        st.close()
        hist = [ctx.bound()[1]]
        for t in range(3):
            ctx.iterate(1)
            hist.append(ctx.bound()[1])
        x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
        assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
        assert all(a <= b for a, b in zip(hist, hist[1:]))
        assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0
