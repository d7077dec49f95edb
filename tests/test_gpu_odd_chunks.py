"""Odd sizes where the fused pass over D works on chunks of two locations and
its last chunk holds one location: N = 35 (the 35-facility workload, 300
passes) and N = 33, in the tile store and the class-sum store (both move two
locations per chunk from N = 33 on), and N = 35 in the pair store (chunks of
four locations, the last of three).

The fused pass (spreading C -> D of Sec. 4.2 with the transfer between
complementary costs of Sec. 4.3, Eq. (11)) assigns a class to the chunk of
the location of its smallest facility, so the one-location chunk holds every
class whose smallest facility sits at location N - 1.  The first pass is
checked against the oracle in full where the oracle can take it on all host
cores (LB, all of B and C) and on sampled D entries: 10^6 uniform ones and
2 x 10^5 drawn from the classes of the last chunk.  Later passes are checked
through properties that hold at any size: non-negative reduced costs,
monotone LB, conservation on sampled permutations.  The 300 passes of the
35-facility workload run in both stores, which must agree bit for bit.
"""
import os

import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I
from paper_1510_02065_gb300 import rlt2
from tests.layout import compact_y
from tests.test_gpu_rlt2 import _conservation_sample

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TILES, CLASSES, PAIRS = rlt2.RLT2_STORE_TILES, rlt2.RLT2_STORE_CLASSES, rlt2.RLT2_STORE_PAIRS


@pytest.fixture(scope="module")
def gpu():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build
    build.build()
    rlt2.lib()
    return t


def _rank2(x, a, b):
    """Rank of x among [0, N) without a and b (x not in {a, b})."""
    return x - (x > a) - (x > b)


def export_index(N, i, j, k, n, p, q):
    """Position of d_ijknpq in the compact export (tile, row, column)."""
    m = N - 1
    t = ((i * N + j) * m + (k - (k > i))) * m + (n - (n > j))
    return (t * (N - 2) + _rank2(p, i, k)) * (N - 2) + _rank2(q, j, n)


def uniform_entries(rng, N, count):
    """count random entries (i, j, k, n, p, q): distinct facilities, distinct locations."""
    fac = np.argsort(rng.random((count, N)), axis=1)[:, :3]
    loc = np.argsort(rng.random((count, N)), axis=1)[:, :3]
    return fac[:, 0], loc[:, 0], fac[:, 1], loc[:, 1], fac[:, 2], loc[:, 2]


def last_chunk_entries(rng, N, count):
    """Entries of classes whose smallest facility is at location N - 1, each
    member ordering of the class equally likely."""
    fac = np.sort(np.argsort(rng.random((count, N)), axis=1)[:, :3], axis=1)
    other = np.argsort(rng.random((count, N - 1)), axis=1)[:, :2]   # locations 0..N-2
    loc = np.concatenate([np.full((count, 1), N - 1), other], axis=1)
    order = np.argsort(rng.random((count, 3)), axis=1)
    f = np.take_along_axis(fac, order, 1)
    l = np.take_along_axis(loc, order, 1)
    return f[:, 0], l[:, 0], f[:, 1], l[:, 1], f[:, 2], l[:, 2]


def check_sampled_D(st, z, N, rng):
    for name, draw, cnt in (("uniform", uniform_entries, 1000000),
                            ("last chunk", last_chunk_entries, 200000)):
        i, j, k, n, p, q = draw(rng, N, cnt)
        ref = st.d[i, j, k, n, p, q]
        got = z[export_index(N, i, j, k, n, p, q)]
        bad = np.nonzero(got != ref)[0]
        assert bad.size == 0, "D differs at %d of %d %s entries, first (i,j,k,n,p,q) = %s" % (
            bad.size, cnt, name, [int(a[bad[0]]) for a in (i, j, k, n, p, q)])


def properties_after(ctx, F, D, N, passes, rng):
    hist = [ctx.bound()[1]]
    for _ in range(passes):
        ctx.iterate(1)
        hist.append(ctx.bound()[1])
    x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
    assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
    assert all(a <= b for a, b in zip(hist, hist[1:]))
    perms = [rng.permutation(N) for _ in range(100)]
    assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0


@pytest.mark.parametrize("store", [TILES, CLASSES])
@pytest.mark.parametrize("N", [33, 35])
def test_first_pass_full_and_last_chunk(gpu, orc, N, store):
    """Pass 1 in full (LB, B, C) against the oracle on all host cores, sampled D
    with the last one-location chunk drawn on purpose, then three passes by
    properties."""
    if N == 35:
        F, D, _ = I.instance("clustered_n35")
    else:
        F, D = I.clustered_euclid(N, seed=N)
    rng = np.random.default_rng(1000 + N)
    st = orc.State(F, D)
    st.iterate_threaded(os.cpu_count() or 1)
    with rlt2.Context(F, D, store=store) as ctx:
        ctx.iterate(1)
        assert ctx.bound()[1] == st.LB
        assert (ctx.state(0) == st.b.reshape(-1)).all(), "B differs"
        assert (ctx.state(1) == compact_y(st.c)).all(), "C differs"
        check_sampled_D(st, ctx.state(2), N, rng)
        st.close()
        properties_after(ctx, F, D, N, 3, rng)


def test_pairs_n35_three_location_last_chunk(gpu, orc):
    """N = 35 in the pair store: chunks of four locations, the last of three.
    The oracle's paired form takes the spreading and complementary operations
    in full and D -> C on three facility slices (tiles D_ijkn with i in the
    slice); 10^6 sampled entries of each slice's tiles must agree, then three
    passes are checked through properties."""
    N = 35
    F, D, _ = I.instance("clustered_n35")
    rng = np.random.default_rng(N + 7)
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
        for a in slices:
            i, j, k, n, p, q = uniform_entries(rng, N, 1000000)
            # move facility a into the first place of each entry's tile
            at_k, at_p = k == a, p == a
            keep = (i == a) | at_k | at_p
            i2 = np.where(at_k, k, np.where(at_p, p, i))
            j2 = np.where(at_k, n, np.where(at_p, q, j))
            k2 = np.where(at_k, i, np.where(at_p, k, k))
            n2 = np.where(at_k, j, np.where(at_p, n, n))
            p2 = np.where(at_k, p, np.where(at_p, i, p))
            q2 = np.where(at_k, q, np.where(at_p, j, q))
            i2, j2, k2, n2, p2, q2 = (x[keep] for x in (i2, j2, k2, n2, p2, q2))
            assert (i2 == a).all()
            ref = st.d[i2, j2, k2, n2, p2, q2]
            got = z[export_index(N, i2, j2, k2, n2, p2, q2)]
            assert (got == ref).all(), "D differs in slice i = %d" % a
        st.close()
        properties_after(ctx, F, D, N, 3, rng)


def test_n35_300_passes_stores_agree(gpu):
    """The configured run: 300 passes of the 35-facility workload in the tile
    store and in the class-sum store give the same LB after every pass and the
    same B, C and sampled D at the end; the end state passes the properties."""
    N = 35
    F, D, iters = I.instance("clustered_n35")
    assert iters == 300
    rng = np.random.default_rng(35300)
    res = {}
    i, j, k, n, p, q = uniform_entries(rng, N, 2000000)
    idx = export_index(N, i, j, k, n, p, q)
    for store in (TILES, CLASSES):
        with rlt2.Context(F, D, store=store) as ctx:
            ctx.iterate(iters)
            hist = list(ctx.history())
            x, y, z = ctx.state(0), ctx.state(1), ctx.state(2)
            assert len(hist) == iters
            assert x.min() >= 0 and y.min() >= 0 and z.min() >= 0
            assert all(a <= b for a, b in zip(hist, hist[1:]))
            perms = [rng.permutation(N) for _ in range(50)]
            assert _conservation_sample(F, D, N, hist[-1], x, y, z, perms) == 0
            res[store] = (hist, x, y, z[idx].copy())
            del z
    a, b = res[TILES], res[CLASSES]
    assert a[0] == b[0]
    for u, w in zip(a[1:], b[1:]):
        assert (u == w).all()
