"""Parity of the CUDA FP64 form (rlt2_f64_*) with the oracle's FP64 form.

Both sides perform the same IEEE double operations in the same order, so every
comparison here is bit for bit (the bit patterns of the doubles, signed zeros
included):
* the FP64 Hungarian kernel on batches of real-valued, tied and integer
  matrices, n = 1..64 (one and two column slots per lane), ragged counts;
* the full state (B, C, D in the compact layouts), LB and work after every pass
  on the 8- and 12-facility workloads, small asymmetric instances with linear
  terms and constants, and two passes of the 20-facility workload; all 200
  passes of that workload against the oracle's stored LB bit patterns and
  state hashes;
* RLT1 mode up to N = 40 (two column slots in C -> B and B -> LB);
* the 30-facility workload (the benchmark's configuration) and N = 33 (D -> C
  LAPs on two column slots): the first pass on sampled entries of three
  facility slices against the oracle, then properties that hold at any size.
"""
import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from tests.layout import compact_y, compact_z, tile_indices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


def bits(a):
    return np.ascontiguousarray(a, np.float64).view(np.int64)


def same(a, b):
    return np.array_equal(bits(a), bits(np.asarray(b, np.float64)))


@pytest.mark.parametrize("n", [1, 2, 3, 7, 17, 28, 31, 32, 33, 40, 63, 64])
def test_lap_batch_parity(gpu, orc, n):
    torch = gpu
    rng = np.random.default_rng(n)
    count = 37
    kinds = [rng.uniform(0, 50, (n, n)), rng.integers(0, 4, (n, n)).astype(np.float64),
             rng.integers(0, 1000, (n, n)) / 7.0]
    M = np.stack([kinds[p % 3] * (1 + p // 3) for p in range(count)])
    dM = torch.tensor(M, dtype=torch.float64, device="cuda")
    dS = torch.zeros(count, dtype=torch.float64, device="cuda")
    dA = torch.zeros((count, n), dtype=torch.int32, device="cuda")
    dU = torch.zeros((count, n), dtype=torch.float64, device="cuda")
    dV = torch.zeros((count, n), dtype=torch.float64, device="cuda")
    dW = torch.zeros((count, 2), dtype=torch.int64, device="cuda")
    rc = rlt2.rlt2_f64_lap_batch(dM.data_ptr(), n, count, dS.data_ptr(), dA.data_ptr(), dU.data_ptr(),
                                 dV.data_ptr(), dW.data_ptr())
    assert rc == rlt2.RLT2_OK
    S, A, U, V, W = orc.lap_batch_f64(M)
    assert same(dS.cpu().numpy(), S)
    assert (dA.cpu().numpy() == A).all()
    assert same(dU.cpu().numpy(), U) and same(dV.cpu().numpy(), V)
    assert (dW.cpu().numpy() == W[:, :2]).all()
    assert same(dM.cpu().numpy(), M)  # the input is left unchanged


def assert_same_state(ctx, st, where=""):
    N = st.N
    assert same(ctx.state(0), st.b.reshape(-1)), "B differs " + where
    assert same(ctx.state(1), compact_y(st.c)), "C differs " + where
    if st.d is not None:
        z = ctx.state(2).reshape(-1, N - 2, N - 2)
        zo = compact_z(st.d)
        bad = np.nonzero(bits(z) != bits(zo))
        assert bad[0].size == 0, "D differs %s at %d entries, first tiles %s" % (where, bad[0].size, bad[0][:3])
    lb, _ = ctx.bound()
    assert same(lb, st.LB), where


@pytest.mark.parametrize("name,passes", [("uniform_n8", 10), ("grid_n12", 4)])
def test_full_state_every_pass(gpu, orc, name, passes):
    F, D, _ = I.instance(name)
    st = orc.StateF64(F, D)
    with rlt2.ContextF64(F, D) as ctx:
        assert_same_state(ctx, st, "at init")
        hist = []
        for t in range(passes):
            ctx.iterate(1)
            hist.append(st.iterate())
            assert_same_state(ctx, st, "after pass %d" % (t + 1))
        assert same(ctx.history(), hist)
        w = ctx.work()
        ow = st.work()
        assert (w[0], w[1], w[2]) == (ow["laps"], ow["steps"], ow["relaxations"])


@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (5, 2), (6, 3), (7, 4)])
def test_small_ragged_asymmetric_with_linear_term(gpu, orc, N, seed):
    rng = np.random.default_rng(seed)
    F = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    D = rng.integers(0, 12, size=(N, N)).astype(np.int32)
    Bl = rng.integers(0, 40, size=(N, N)) / 3.0
    const = 17.25
    st = orc.StateF64(F, D, B_lin=Bl, lb_const=const)
    with rlt2.ContextF64(F, D, B_lin=Bl, lb_const=const) as ctx:
        assert_same_state(ctx, st, "at init")
        for t in range(6):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))


@pytest.mark.parametrize("N", [12, 33, 40])
def test_rlt1_mode(gpu, orc, N):
    F, D = I.clustered_euclid(N, seed=N)
    st = orc.StateF64(F, D, rlt1_only=True)
    with rlt2.ContextF64(F, D, rlt1_only=True) as ctx:
        for t in range(3):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "rlt1 after pass %d" % (t + 1))


@pytest.mark.slow
def test_n20_two_passes(gpu, orc):
    F, D, _ = I.instance("clustered_n20")
    st = orc.StateF64(F, D)
    with rlt2.ContextF64(F, D) as ctx:
        for t in range(2):
            ctx.iterate(1)
            st.iterate()
            assert_same_state(ctx, st, "after pass %d" % (t + 1))


def test_n20_against_golden_200_passes(gpu):
    """All 200 passes of the 20-facility workload against the bit patterns of
    the oracle's LB history and state hashes (tests/golden/lb_f64_clustered_n20.json,
    written by tests/golden/make_golden.py --f64 from the oracle alone)."""
    import json
    import os
    from tests.layout import state_hash
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "lb_f64_clustered_n20.json")))
    F, D, iters = I.instance("clustered_n20")
    N = 20
    with rlt2.ContextF64(F, D) as ctx:
        done = 0
        for t in sorted(int(k) for k in gold["hash"]):
            ctx.iterate(t - done)
            done = t
            h = gold["hash"][str(t)]
            assert state_hash(bits(ctx.state(0))) == h["x"], "B after pass %d" % t
            assert state_hash(bits(ctx.state(1))) == h["y"], "C after pass %d" % t
            assert state_hash(bits(ctx.state(2).reshape(-1, N - 2, N - 2))) == h["z"], "D after pass %d" % t
        assert done == iters
        assert list(bits(ctx.history())) == gold["lb_bits"]


def _first_pass_then_properties(orc, F, D, N, seed):
    """The oracle takes the spreading and complementary operations in full and
    D -> C on three facility slices; 10^6 sampled D entries of those slices
    after the first pass must agree bit for bit; two more passes are then
    checked through properties (reduced costs >= -1e-9 |LB|, LB non-decreasing
    up to rounding, conservation on sampled permutations to 1e-9 relative)."""
    rng = np.random.default_rng(seed)
    st = orc.StateF64(F, D)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    slices = (0, N // 2, N - 1)
    for a in slices:
        st.concentrate_D_to_C_range(a, a + 1)
    with rlt2.ContextF64(F, D) as ctx:
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
            assert same(got, ref), "slice %d" % a
        del z
        st.close()
        ctx.iterate(2)
        hist = ctx.history()
        assert len(hist) == 3 and hist[0] > 0
        assert (np.diff(hist) >= -1e-9 * hist[-1]).all()
        x = ctx.state(0).reshape(N, N)
        y = ctx.state(1)
        z = ctx.state(2)
        tol = 1e-9 * hist[-1]
        assert x.min() >= -tol and y.min() >= -tol and z.min() >= -tol
        # conservation on sampled permutations: Q(pi) = LB + b + c + d along pi
        m = N - 1
        for _ in range(20):
            perm = rng.permutation(N)
            Fi = np.asarray(F, np.float64)
            Dp = np.asarray(D, np.float64)[np.ix_(perm, perm)]
            Q = (Fi * Dp).sum() - (np.diag(Fi) * np.diag(Dp)).sum()
            tot = hist[-1] + x[np.arange(N), perm].sum()
            for a in range(N):
                for b in range(N):
                    if a == b:
                        continue
                    kk, nn = b - (b > a), perm[b] - (perm[b] > perm[a])
                    t = ((a * N + perm[a]) * m + kk) * m + nn
                    tot += y[t]
                    for c in range(N):
                        if c in (a, b):
                            continue
                        r = c - (c > a) - (c > b)
                        lo, hi = min(perm[a], perm[b]), max(perm[a], perm[b])
                        s = perm[c] - (perm[c] > lo) - (perm[c] > hi)
                        tot += z[(t * (N - 2) + r) * (N - 2) + s]
            assert abs(Q - tot) <= 1e-9 * Q


@pytest.mark.slow
def test_headline_n30_first_pass_then_properties(gpu, orc):
    """The 30-facility workload of the benchmark."""
    F, D, _ = I.instance("clustered_n30")
    _first_pass_then_properties(orc, F, D, 30, 30)


@pytest.mark.slow
def test_two_slot_lanes_n33(gpu, orc):
    """N = 33: the D -> C LAPs span 33 location columns (two slots per lane)."""
    F, D = I.clustered_euclid(33, seed=33)
    _first_pass_then_properties(orc, F, D, 33, 33)


def test_errors(gpu):
    F, D = I.clustered_euclid(6, seed=1)
    with rlt2.ContextF64(F, D, max_iters=2) as ctx:
        with pytest.raises(rlt2.Rlt2Error) as e:
            ctx.iterate(3)
        assert e.value.code == rlt2.RLT2_E_STATE
        with pytest.raises(rlt2.Rlt2Error) as e:
            ctx.iterate(-1)
        assert e.value.code == rlt2.RLT2_E_INVAL
        out = np.zeros(5)
        rc = rlt2.lib().rlt2_f64_get_state(ctx.ctx, 0, out.ctypes.data_as(rlt2._dblp), 5)
        assert rc == rlt2.RLT2_E_INVAL
        ctx.iterate(2)
        assert ctx.bound()[1] == 2
    with rlt2.ContextF64(F, D, rlt1_only=True) as ctx:
        with pytest.raises(rlt2.Rlt2Error):
            ctx.state(2)
