"""Large instances, beyond the sizes at which the D->C kernel's larger CTA
shapes stop fitting in shared memory and the fused pass moves fewer locations
per chunk: N = 41, 44, 53 and 64 (the largest the library accepts; about 52 GB
on the device) in the class-sum store, N = 44 and 48 in the tile store (45 GB
at 48) and in the pair store.

The oracle cannot hold D at N = 64 (N^6 dense entries), so the first pass is
checked on sampled tiles (read from device memory): the D -> C input of a
tile in pass 1 follows from F
and D alone (spread of c = F D over the N - 2 rows with the integer split of
reading R3, then the six-way split of the class sums of reading R4), written
out here per tile and checked against the oracle's state at N = 5..7 on the
CPU; the oracle's Hungarian then gives the tile's duals, which the class-sum
store keeps on the device for every tile, and its residual tile, which the
tile store holds.  Two more passes are checked through properties (monotone
LB, non-negative B and C).
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from paper_1510_02065_gb300 import instances as I


def pass1_tile(F, D, i, j, k, n):
    """D->C input of tile (i, j, k, n) in pass 1 of the integer form (rows p
    not in {i, k}, columns q not in {j, n}, ascending), from F and D alone."""
    N = F.shape[0]
    m = N - 2
    rows = np.array([p for p in range(N) if p not in (i, k)])
    cols = np.array([q for q in range(N) if q not in (j, n)])
    P, Q = np.meshgrid(rows, cols, indexing="ij")
    fac = np.stack([np.full_like(P, i), np.full_like(P, k), P])
    loc = np.stack([np.full_like(Q, j), np.full_like(Q, n), Q])
    order = np.argsort(fac, axis=0)
    a, b, c = np.take_along_axis(fac, order, 0)
    la, lb, lc = np.take_along_axis(loc, order, 0)
    F64 = F.astype(np.int64)
    D64 = D.astype(np.int64)

    def spread(x, lx, y, ly, z):  # row z's share of c_{x lx y ly} (R3)
        cv = F64[x, y] * D64[lx, ly]
        t = z - (z > x) - (z > y)
        return cv // m + (t < cv % m)

    # the six members in lexicographic order of their index tuples (Eq. (11))
    members = [(a, la, b, lb, c), (a, la, c, lc, b), (b, lb, a, la, c),
               (b, lb, c, lc, a), (c, lc, a, la, b), (c, lc, b, lb, a)]
    T = sum(spread(*mm) for mm in members)
    own = [(a == i) & (b == k), (a == i) & (c == k), (b == i) & (a == k),
           (b == i) & (c == k), (c == i) & (a == k), (c == i) & (b == k)]
    rank = np.select(own, [0, 1, 2, 3, 4, 5], -1)
    assert (rank >= 0).all()
    return T // 6 + (rank < T % 6)


def pass1_pair_tile(F, D, i, j, k, n):
    """The same for the pair store (reading R13), i < k: the class sum of the
    six spread values split three ways over d_ijknpq, d_ijpqkn, d_knpqij (the
    class's members whose first facility is below the second), in that order."""
    assert i < k
    N = F.shape[0]
    m = N - 2
    rows = np.array([p for p in range(N) if p not in (i, k)])
    cols = np.array([q for q in range(N) if q not in (j, n)])
    P, Q = np.meshgrid(rows, cols, indexing="ij")
    fac = np.stack([np.full_like(P, i), np.full_like(P, k), P])
    loc = np.stack([np.full_like(Q, j), np.full_like(Q, n), Q])
    order = np.argsort(fac, axis=0)
    a, b, c = np.take_along_axis(fac, order, 0)
    la, lb, lc = np.take_along_axis(loc, order, 0)
    F64 = F.astype(np.int64)
    D64 = D.astype(np.int64)

    def spread(x, lx, y, ly, z):
        cv = F64[x, y] * D64[lx, ly]
        t = z - (z > x) - (z > y)
        return cv // m + (t < cv % m)

    members = [(a, la, b, lb, c), (a, la, c, lc, b), (b, lb, a, la, c),
               (b, lb, c, lc, a), (c, lc, a, la, b), (c, lc, b, lb, a)]
    T = sum(spread(*mm) for mm in members)
    pos = np.where(P > k, 0, np.where(P > i, 1, 2))  # (i,k,p), (i,p,k), (p,i,k)
    return T // 3 + (pos < T % 3)


@pytest.mark.parametrize("N,seed", [(5, 0), (6, 1), (7, 2)])
def test_pass1_pair_tile_formula_equals_oracle(orc, N, seed):
    F, D = I.clustered_euclid(N, seed=seed)
    F[2, 0] += 7
    st = orc.State(F, D, paired=True)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    for i in range(N):
        for k in range(i + 1, N):
            for j in range(N):
                for n in range(N):
                    if j == n:
                        continue
                    rows = [p for p in range(N) if p not in (i, k)]
                    cols = [q for q in range(N) if q not in (j, n)]
                    assert (pass1_pair_tile(F, D, i, j, k, n) == st.d[i, j, k, n][np.ix_(rows, cols)]).all()


@pytest.mark.parametrize("N,seed", [(5, 0), (6, 1), (7, 2)])
def test_pass1_tile_formula_equals_oracle(orc, N, seed):
    F, D = I.clustered_euclid(N, seed=seed)
    F[0, 2] += 5  # asymmetric flows
    st = orc.State(F, D)
    st.spread_B_to_C()
    st.spread_C_to_D()
    st.complementary_D()
    for i in range(N):
        for k in range(N):
            for j in range(N):
                for n in range(N):
                    if i == k or j == n:
                        continue
                    rows = [p for p in range(N) if p not in (i, k)]
                    cols = [q for q in range(N) if q not in (j, n)]
                    assert (pass1_tile(F, D, i, j, k, n) == st.d[i, j, k, n][np.ix_(rows, cols)]).all()


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_02065_gb300 import build, rlt2
    build.build()
    return rlt2


def _d2h_int32(ptr, count):
    name = ctypes.util.find_library("cudart") or "/usr/local/cuda/lib64/libcudart.so"
    rt = ctypes.CDLL(name)
    out = np.empty(count, np.int32)
    rc = rt.cudaMemcpy(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(ptr), ctypes.c_size_t(count * 4),
                       ctypes.c_int(2))  # device to host
    assert rc == 0, rc
    return out


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("N", [41, 44, 53, 64])
def test_class_store_large_first_pass_sampled(orc, N):
    rlt2 = _gpu()
    F, D = I.clustered_euclid(N, seed=N)
    m, n = N - 1, N - 2
    W = rlt2.rlt2_row_stride(N)
    U0 = (n + 3) & ~3
    DS = U0 + W
    rng = np.random.default_rng(N)
    with rlt2.Context(F, D, store=rlt2.RLT2_STORE_CLASSES, max_iters=4) as ctx:
        ctx.iterate(1)
        lb1 = ctx.bound()[1]
        du = rlt2.rlt2_device_state(ctx.ctx, 3)
        assert du
        tiles = rng.integers(0, N * N * m * m, size=120)
        for t in tiles:
            t = int(t)
            nn, rest = t % m, t // m
            kk, ij = rest % m, rest // m
            i, j = divmod(ij, N)
            k, nl = kk + (kk >= i), nn + (nn >= j)
            M = pass1_tile(F, D, i, j, k, nl)
            _, _, u, v, _ = orc.lap(M)
            got = _d2h_int32(du + t * DS * 4, DS)
            cols = [q for q in range(N) if q not in (j, nl)]
            assert (got[:n] == u).all(), ("u", t)
            assert (got[U0 + np.array(cols)] == v).all(), ("v", t)
            assert got[U0 + j] == 0 and got[U0 + nl] == 0
        ctx.iterate(2)
        hist = ctx.history()
        assert len(hist) == 3 and hist[0] == lb1 > 0
        assert (np.diff(hist) >= 0).all()
        assert ctx.state(0).min() >= 0 and ctx.state(1).min() >= 0


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("N", [44, 48])
def test_tile_store_large_first_pass_sampled(orc, N):
    rlt2 = _gpu()
    F, D = I.clustered_euclid(N, seed=N)
    m, n = N - 1, N - 2
    W = rlt2.rlt2_row_stride(N)
    TS = n * W
    rng = np.random.default_rng(N)
    with rlt2.Context(F, D, store=rlt2.RLT2_STORE_TILES, max_iters=4) as ctx:
        ctx.iterate(1)
        lb1 = ctx.bound()[1]
        z = rlt2.rlt2_device_state(ctx.ctx, 2)
        assert z
        for t in rng.integers(0, N * N * m * m, size=120):
            t = int(t)
            nn, rest = t % m, t // m
            kk, ij = rest % m, rest // m
            i, j = divmod(ij, N)
            k, nl = kk + (kk >= i), nn + (nn >= j)
            M = pass1_tile(F, D, i, j, k, nl)
            _, _, u, v, _ = orc.lap(M)
            got = _d2h_int32(z + t * TS * 4, TS).reshape(n, W)
            cols = [q for q in range(N) if q not in (j, nl)]
            assert (got[:, cols] == M - u[:, None] - v[None, :]).all(), t
            assert (got[:, [j, nl]] == 0).all() and (got[:, N:] == 0).all()
        ctx.iterate(2)
        hist = ctx.history()
        assert len(hist) == 3 and hist[0] == lb1 > 0
        assert (np.diff(hist) >= 0).all()
        assert ctx.state(0).min() >= 0 and ctx.state(1).min() >= 0


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("N", [44, 48])
def test_pair_store_large_first_pass_sampled(orc, N):
    """The pair store (Sec. 6's complementary submatrices, reading R13): pair
    tiles (i < k) indexed ((C(k,2) + i) N + j)(N-1) + n'."""
    rlt2 = _gpu()
    F, D = I.clustered_euclid(N, seed=N + 1)
    m, n = N - 1, N - 2
    W = rlt2.rlt2_row_stride(N)
    TS = n * W
    rng = np.random.default_rng(N + 1)
    with rlt2.Context(F, D, store=rlt2.RLT2_STORE_PAIRS, max_iters=4) as ctx:
        ctx.iterate(1)
        lb1 = ctx.bound()[1]
        z = rlt2.rlt2_device_state(ctx.ctx, 2)
        assert z
        npairs = N * (N - 1) // 2
        for th in rng.integers(0, npairs * N * m, size=120):
            th = int(th)
            nn, rest = th % m, th // m
            j, pr = rest % N, rest // N
            k = int((1 + np.sqrt(1 + 8 * pr)) // 2)
            while k * (k - 1) // 2 > pr:
                k -= 1
            while (k + 1) * k // 2 <= pr:
                k += 1
            i = pr - k * (k - 1) // 2
            nl = nn + (nn >= j)
            M = pass1_pair_tile(F, D, i, j, k, nl)
            _, _, u, v, _ = orc.lap(M)
            got = _d2h_int32(z + th * TS * 4, TS).reshape(n, W)
            cols = [q for q in range(N) if q not in (j, nl)]
            assert (got[:, cols] == M - u[:, None] - v[None, :]).all(), th
        ctx.iterate(2)
        hist = ctx.history()
        assert len(hist) == 3 and hist[0] == lb1 > 0
        assert (np.diff(hist) >= 0).all()
        assert ctx.state(0).min() >= 0 and ctx.state(1).min() >= 0
