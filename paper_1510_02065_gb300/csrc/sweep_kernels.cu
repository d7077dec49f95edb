// sweep_kernels.cu -- initialisation and the spreading passes (sm_103a).
//
// spread_x_to_y_kernel: spread B -> C (Sec. 4.2), c'_ijkn = c_ijkn + the share
// of b_ij of row k, one small pass over C.
// p1_kernel performs the next two operations of the loop of Algorithm 1 in one
// read and one write of D:
//   spread C -> D   (Sec. 4.2): every d_ijknpq of row p gains the share of c'_ijkn,
//   complementary D (Sec. 4.3, Eq. (11)): the six members of each class are
//                   replaced by the equal split of their sum, the odd units going
//                   to the members of lowest lexicographic rank.
// A cost x spread over m rows gives the t-th row (ascending) floor(x/m) + [t < x mod m].
//
// Work unit: one CTA per facility triple i < k < p and chunk of JC locations j
// (the location of the smallest facility).  A class {(i,j),(k,n),(p,q)} has six
// members in six tiles; for a fixed triple each member kind is one tile row:
//   kind 1  d_ijknpq  tile (i,j,k,n) row p      kind 4  d_knpqij  tile (k,n,p,q) row i
//   kind 2  d_ijpqkn  tile (i,j,p,q) row k      kind 5  d_pqijkn  tile (p,q,i,j) row k
//   kind 3  d_knijpq  tile (k,n,i,j) row p      kind 6  d_pqknij  tile (p,q,k,n) row i
// Kinds 1, 2, 3, 5 are whole tile rows owned by this CTA; kinds 4 and 6 are the
// JC columns j of rows shared with the CTAs of the other chunks.  Tile columns
// are indexed by location, so those JC columns are one aligned piece (16 bytes
// for JC = 4) of the row.  The CTA stages everything in shared memory with
// asynchronous copies (cp.async, all in flight at once), splits every class,
// and writes rows and pieces back with 16-byte stores; two CTAs per SM overlap
// one's copies with the other's arithmetic.  With i < k < p the lexicographic
// ranks of kinds 1..6 are 0..5.
#include <cstring>

#include "device.cuh"
#include "kernels.h"

namespace rlt2 {

constexpr int kP1Threads = 512;
constexpr int kP1Warps = kP1Threads / 32;

__device__ __forceinline__ int tidx_n(int N, int a, int b, int c, int d)
{
    const int m = N - 1;
    return ((a * N + b) * m + (c - (c > a))) * m + (d - (d > b));
}

// t-th of m shares of x >= 0 (reading of Sec. 4.2 in integers); fm divides by m
__device__ __forceinline__ int share(int x, const FastDiv &fm, int t)
{
    const int q = (int)fdiv((unsigned)x, fm);
    return q + (t < x - q * (int)fm.d ? 1 : 0);
}

// Shared-memory layout of one work unit (offsets in ints, all 16-byte aligned).
// Rows of kinds 1 and 3 are indexed (jj, location), pitch W; rows of kinds 2
// and 5 likewise, read by column, with pitch S25 = 4 x odd (W, or W + 4 when
// W / 4 is even): a column read across 32 rows then meets 8 distinct banks,
// the fewest 16-byte-aligned rows allow.  The JC-location pieces of kinds 4
// and 6 are indexed (a, l') with l' = l - (l > a) the rank of l among the
// locations != a, and m|1 (odd) pieces per a: the layout of the tensor box of
// zmap, and a conflict-free 16-byte read of pieces (qq, nn) across lanes qq.
struct P1Layout {
    int S13, S25, P46, H6p;
    int A1, A3, A2, A5, A4, A6, H1, H3, H2, H5, H4, H6;
    int HU;     // class-sum store: u of each H entry's tile row, same offsets from HU as from H1
    int total;
};

__host__ __device__ inline int up4(int x) { return (x + 3) & ~3; }

// paired: the pair store's pass moves only kinds 1, 2 and 4 (A3, A5, A6 empty).
__host__ __device__ inline P1Layout p1_layout(int N, int W, int JC, bool sym, bool paired = false)
{
    P1Layout L;
    L.S13 = W;
    L.S25 = (W / 4) % 2 ? W : W + 4;
    L.P46 = JC * ((N - 1) | 1);
    L.H6p = N | 1;
    int o = 0;
    L.A1 = o; o += JC * N * L.S13;
    L.A3 = o; o += paired ? 0 : JC * N * L.S13;
    L.A2 = o; o += JC * N * L.S25;
    L.A5 = o; o += paired ? 0 : JC * N * L.S25;
    o = (o + 31) & ~31;  // tensor-copy destinations on 128-byte boundaries
    L.A4 = o; o += (N * L.P46 + 31) & ~31;
    L.A6 = o; o += paired ? 0 : up4(N * L.P46);
    L.H1 = o; o += up4(JC * N);
    L.H3 = o; o += up4(JC * N);
    L.H2 = o; o += up4(JC * N);
    L.H5 = o; o += up4(JC * N);
    L.H4 = o; o += up4(N * N);
    L.H6 = o; o += up4(N * L.H6p);
    L.HU = o;
    if (sym) o += o - L.H1;
    L.total = o;
    return L;
}

size_t p1_smem_bytes(int N, int JC, bool sym, bool paired)
{
    return (size_t)p1_layout(N, up4(N), JC, sym, paired).total * 4;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

bool encode_zmap(NodeDesc &nd, int JC)
{
    nd.zmap_ok = 0;
    std::memset(&nd.zmap, 0, sizeof(nd.zmap));
    if (JC != 4 || (!nd.p.z && !nd.p.du)) return false;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t N = (cuuint64_t)nd.N, m = N - 1, W = (cuuint64_t)nd.W, n = N - 2;
    // tile store: (column, row, n', k', i*N + j); class-sum store: the v row of
    // every tile as (column, -, n', k', i*N + j) with the tile's dual stride
    const cuuint64_t R = nd.p.z ? W : (cuuint64_t)nd.DS;  // ints per row step
    const cuuint64_t rows = nd.p.z ? n : 1;
    cuuint64_t dim[5] = {W, rows, m, m, N * N};
    cuuint64_t stride[4] = {R * 4, R * rows * 4, R * rows * m * 4, R * rows * m * m * 4};
    cuuint32_t box[5] = {4, 1, (cuuint32_t)(m | 1), 1, (cuuint32_t)N};
    if (nd.paired) {
        // pair store: (column, row, n', j, pair(i,k)); the box takes every
        // location a of the first facility: (4, 1, m|1, N, 1)
        dim[3] = N;
        dim[4] = N * (N - 1) / 2;
        stride[2] = W * n * m * 4;
        stride[3] = W * n * m * N * 4;
        box[3] = (cuuint32_t)N;
        box[4] = 1;
    }
    const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
    void *base = nd.p.z ? (void *)nd.p.z : (void *)(nd.p.du + nd.U0);
    if (fn(&nd.zmap, CU_TENSOR_MAP_DATA_TYPE_INT32, 5, base, dim, stride, box, estride,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    nd.zmap_ok = 1;
    return true;
}

int p1_chunk(int N, bool sym, bool paired)
{
#ifdef RLT2_P1_JC
    if (p1_smem_bytes(N, RLT2_P1_JC, sym, paired) <= 200 * 1024) return RLT2_P1_JC;  // build-time override
#endif
    for (int jc : {4, 2}) if (p1_smem_bytes(N, jc, sym, paired) <= 112 * 1024) return jc;
    return 1;
}

// Tile and tile row of a full row of kind q (0: kind 1, 1: kind 3, 2: kind 2,
// 3: kind 5), location j of the smallest facility, other location x.
__device__ __forceinline__ void full_row(int q, int N, int i, int k, int pp, int j, int x, int &t,
                                         int &row)
{
    if (q == 0) { t = tidx_n(N, i, j, k, x); row = pp - 2; }        // d_ijkxpq: tile (i,j,k,x), row p
    else if (q == 1) { t = tidx_n(N, k, x, i, j); row = pp - 2; }   // d_kxijpq: tile (k,x,i,j), row p
    else if (q == 2) { t = tidx_n(N, i, j, pp, x); row = k - 1; }   // d_ijpxkn: tile (i,j,p,x), row k
    else { t = tidx_n(N, pp, x, i, j); row = k - 1; }               // d_pxijkn: tile (p,x,i,j), row k
}

template <int JC>
__device__ __forceinline__ void cp_async_piece(void *dst, const void *src)
{
    if constexpr (JC == 4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else if constexpr (JC == 2)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

template <int JC>
__device__ __forceinline__ void copy_piece(int *dst, const int *src)
{
    if constexpr (JC == 4) *reinterpret_cast<int4 *>(dst) = *reinterpret_cast<const int4 *>(src);
    else if constexpr (JC == 2) *reinterpret_cast<int2 *>(dst) = *reinterpret_cast<const int2 *>(src);
    else *dst = *src;
}

// JC consecutive ints of shared memory (JC-aligned) to registers and back.
template <int JC>
__device__ __forceinline__ void load_piece(int (&r)[JC], const int *src)
{
    if constexpr (JC == 4) {
        const int4 v = *reinterpret_cast<const int4 *>(src);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else if constexpr (JC == 2) {
        const int2 v = *reinterpret_cast<const int2 *>(src);
        r[0] = v.x; r[1] = v.y;
    } else {
        r[0] = *src;
    }
}

template <int JC>
__device__ __forceinline__ void store_piece(int *dst, const int (&r)[JC])
{
    if constexpr (JC == 4) *reinterpret_cast<int4 *>(dst) = make_int4(r[0], r[1], r[2], r[3]);
    else if constexpr (JC == 2) *reinterpret_cast<int2 *>(dst) = make_int2(r[0], r[1]);
    else *dst = r[0];
}

// Gather, for every member tile of the work unit, c' (yS) into its H slot
// and, with the class-sum store, u of the member's row into the HU slot at the
// same offset: one 4-byte cp.async each, all in flight with the bulk copies.
template <int JC, bool SYM>
__device__ __forceinline__ void p1_gather_c(const P1Layout &L, int N, int i, int k, int pp, int j0, int jc,
                                            const FastDiv &fN, const int *yS, const int *du, int DS, int *sm)
{
    const int NN = N * N;
    for (int e = threadIdx.x; e < 4 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        int t, row;
        full_row(q, N, i, k, pp, j, x, t, row);
        const int h = (q == 0 ? L.H1 : q == 1 ? L.H3 : q == 2 ? L.H2 : L.H5) + jj * N + x;
        cp_async4(sm + h, yS + t);
        if constexpr (SYM) cp_async4(sm + L.HU + (h - L.H1), du + (size_t)t * DS + row);
    }
    for (int e = threadIdx.x; e < 2 * NN; e += kP1Threads) {
        const int kind = e >= NN, r2 = e - kind * NN;
        const int a = (int)fdiv((unsigned)r2, fN), l = r2 - a * N;
        if (l == a) continue;
        const int t = kind ? tidx_n(N, pp, a, k, l) : tidx_n(N, k, a, pp, l);
        const int h = (kind ? L.H6 + a * L.H6p : L.H4 + a * N) + l;
        cp_async4(sm + h, yS + t);
        if constexpr (SYM) cp_async4(sm + L.HU + (h - L.H1), du + (size_t)t * DS + i);
    }
}

// Turn every H slot into the share of its c' for the member's row (kinds 1, 3:
// row p - 2 of the tile; kinds 2, 5: row k - 1; kinds 4, 6: row i), minus u of
// that row with the class-sum store.  Slots never gathered hold garbage and
// stay unused.
template <bool SYM>
__device__ __forceinline__ void p1_shares(const P1Layout &L, int N, int i, int k, int pp, const FastDiv &fn,
                                          int *sm)
{
    const int end = L.HU;
    for (int h = L.H1 + threadIdx.x; h < end; h += kP1Threads) {
        const int row = h < L.H2 ? pp - 2 : h < L.H4 ? k - 1 : i;
        int val = share(sm[h], fn, row);
        if constexpr (SYM) val -= sm[L.HU + (h - L.H1)];
        sm[h] = val;
    }
}

// One work unit of the fused pass over D in the tile store: an instance's
// facility triple i < k < p and chunk of JC locations j0.. of i (jc of them
// in the instance's last chunk).  ONE (a group of one instance): the instance
// is the kernel parameter g.first.
struct P1Unit {
    const NodeDesc *nd;
    int i, k, pp, j0, jc;
    bool live;   // the instance's stopping rule has not fired
};

template <int JC, bool ONE>
__device__ __forceinline__ P1Unit p1_unit(const Group &g, int u)
{
    P1Unit w;
    w.nd = ONE ? &g.first
               : &g.nodes[find_node(g.nodes, g.B, u, [](const NodeDesc &d) { return (long long)d.cta_base; })];
    const int bid = u - w.nd->cta_base, nchunks = w.nd->nchunks;
    const int4 tr = g.triples[bid / nchunks];
    w.i = tr.x;
    w.k = tr.y;
    w.pp = tr.z;
    w.j0 = (bid % nchunks) * JC;
    w.jc = min(JC, w.nd->N - w.j0);
    w.live = !*w.nd->p.stop;
    return w;
}

// Start every load of unit w into the layout at sm, all in flight at once:
// every full row by one bulk copy and, where the map exists (JC = 4), the
// JC-location pieces of kinds 4 and 6 by one tensor copy per kind (rows i of
// tiles (k,a,p,l), resp. (p,a,k,l), all a and l), all completing on bar;
// else one aligned cp.async per piece.  Then c' of every member tile (4-byte
// cp.async into the H arrays).  The caller commits the cp.async group.
template <int JC, bool ONE>
__device__ __forceinline__ void p1_issue(const Group &g, const P1Unit &w, int *sm, uint64_t *bar)
{
    const NodeDesc &nd = *w.nd;
    const int N = nd.N, W = nd.W, NN = N * N;
    const FastDiv fN = nd.fN;
    const P1Layout L = p1_layout(N, W, JC, false);
    const size_t TS = (size_t)(N - 2) * W;
    const int i = w.i, k = w.k, pp = w.pp, j0 = w.j0, jc = w.jc;
    int *__restrict__ z = nd.p.z;
    const bool tma = JC == 4 && nd.zmap_ok;
    const void *zmap = &nd.zmap;
    const unsigned rowBytes = (unsigned)W * 4u;
    if (threadIdx.x == 0) {
        if (!ONE && tma) tensormap_acquire(zmap);
        const unsigned pieceBytes = tma ? 2u * (unsigned)(N * L.P46) * 4u : 0u;
        mbar_arrive_expect_tx(bar, (unsigned)(4 * jc * (N - 1)) * rowBytes + pieceBytes);
        if (tma) {
            tensor_load5(sm + L.A4, zmap, j0, i, 0, pp - 1, k * N, bar);  // kind 4: tile (k,a,p,l), row i
            tensor_load5(sm + L.A6, zmap, j0, i, 0, k, pp * N, bar);      // kind 6: tile (p,a,k,l), row i
        }
    }
    for (int e = threadIdx.x; e < 4 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        int t, row;
        full_row(q, N, i, k, pp, j, x, t, row);
        const int base = q == 0 ? L.A1 : q == 1 ? L.A3 : q == 2 ? L.A2 : L.A5;
        const int pitch = q < 2 ? L.S13 : L.S25;
        bulk_load_tx(sm + base + (jj * N + x) * pitch, z + t * TS + (size_t)row * W, rowBytes, bar);
    }
    for (int e = tma ? 2 * NN : threadIdx.x; e < 2 * NN; e += kP1Threads) {
        const int kind = e >= NN, r2 = e - kind * NN;
        const int a = (int)fdiv((unsigned)r2, fN), l = r2 - a * N;
        if (l == a) continue;
        // kind 4: row i of tile (k,a,p,l); kind 6: row i of tile (p,a,k,l)
        const int t = kind ? tidx_n(N, pp, a, k, l) : tidx_n(N, k, a, pp, l);
        cp_async_piece<JC>(sm + (kind ? L.A6 : L.A4) + a * L.P46 + (l - (l > a)) * JC,
                           z + t * TS + (size_t)i * W + j0);
    }
    p1_gather_c<JC, false>(L, N, i, k, pp, j0, jc, fN, nd.p.yS, nullptr, 0, sm);
}

// Shares of c' and the split of every class {(i,j),(k,nn),(p,qq)}, j in the
// chunk, in shared memory (the loads of unit w have landed and the CTA is
// synchronised): one warp per nn, lanes over qq, each lane the JC classes of
// its (nn, qq).  Their members of kinds 4 and 6 are exactly the pieces
// (nn, qq) and (qq, nn), which move as one vector each.
template <int JC>
__device__ __forceinline__ void p1_split(const P1Unit &w, int *sm)
{
    const NodeDesc &nd = *w.nd;
    const int N = nd.N;
    const P1Layout L = p1_layout(N, nd.W, JC, false);
    const int i = w.i, k = w.k, pp = w.pp, j0 = w.j0, jc = w.jc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    p1_shares<false>(L, N, i, k, pp, nd.fn, sm);
    __syncthreads();
    for (int nn = warp; nn < N; nn += kP1Warps) {
        const int *h4 = sm + L.H4 + nn * N, *h6 = sm + L.H6 + nn;
        for (int qq = lane; qq < N; qq += 32) {
            if (qq == nn) continue;
            int *a4 = sm + L.A4 + nn * L.P46 + (qq - (qq > nn)) * JC;   // piece (nn, qq)
            int *a6 = sm + L.A6 + qq * L.P46 + (nn - (nn > qq)) * JC;   // piece (qq, nn)
            int p4[JC], p6[JC];
            load_piece<JC>(p4, a4);
            load_piece<JC>(p6, a6);
            const int h46 = h4[qq] + h6[qq * L.H6p];
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const int j = j0 + jj;
                if (jj >= jc || j == nn || j == qq) continue;
                const int rn = jj * N + nn, rq = jj * N + qq;
                int *a1 = sm + L.A1 + rn * L.S13 + qq, *a3 = sm + L.A3 + rn * L.S13 + qq;
                int *a2 = sm + L.A2 + rq * L.S25 + nn, *a5 = sm + L.A5 + rq * L.S25 + nn;
                const int T = *a1 + sm[L.H1 + rn] + *a2 + sm[L.H2 + rq] + *a3 + sm[L.H3 + rn] + p4[jj] +
                              *a5 + sm[L.H5 + rq] + p6[jj] + h46;
                const int q6 = T / 6, rm = T - 6 * q6;
                *a1 = q6 + (0 < rm);      // ranks: d_ijknpq 0, d_ijpqkn 1, d_knijpq 2,
                *a2 = q6 + (1 < rm);      //        d_knpqij 3, d_pqijkn 4, d_pqknij 5
                *a3 = q6 + (2 < rm);
                p4[jj] = q6 + (3 < rm);
                *a5 = q6 + (4 < rm);
                p6[jj] = q6 + (5 < rm);
            }
            store_piece<JC>(a4, p4);
            store_piece<JC>(a6, p6);
        }
    }
}

// Write unit w back: whole rows by bulk stores (after the split's shared
// writes are made visible to the async proxy), pieces by one tensor store
// per kind or by vector stores; every thread commits its bulk stores as one
// group.  The layout at sm stays in use until those groups have been read.
template <int JC>
__device__ __forceinline__ void p1_store(const P1Unit &w, int *sm)
{
    const NodeDesc &nd = *w.nd;
    const int N = nd.N, W = nd.W, NN = N * N;
    const FastDiv fN = nd.fN;
    const P1Layout L = p1_layout(N, W, JC, false);
    const size_t TS = (size_t)(N - 2) * W;
    const int i = w.i, k = w.k, pp = w.pp, j0 = w.j0, jc = w.jc;
    int *__restrict__ z = nd.p.z;
    const bool tma = JC == 4 && nd.zmap_ok;
    const void *zmap = &nd.zmap;
    const unsigned rowBytes = (unsigned)W * 4u;
    fence_proxy_async_smem();
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        int t, row;
        full_row(q, N, i, k, pp, j, x, t, row);
        const int base = q == 0 ? L.A1 : q == 1 ? L.A3 : q == 2 ? L.A2 : L.A5;
        const int pitch = q < 2 ? L.S13 : L.S25;
        bulk_store(z + t * TS + (size_t)row * W, sm + base + (jj * N + x) * pitch, rowBytes);
    }
    if (tma && threadIdx.x == 0) {
        tensor_store5(zmap, j0, i, 0, pp - 1, k * N, sm + L.A4);
        tensor_store5(zmap, j0, i, 0, k, pp * N, sm + L.A6);
    }
    bulk_commit();
    for (int e = tma ? 2 * NN : threadIdx.x; e < 2 * NN; e += kP1Threads) {
        const int kind = e >= NN, r2 = e - kind * NN;
        const int a = (int)fdiv((unsigned)r2, fN), l = r2 - a * N;
        if (l == a) continue;
        const int t = kind ? tidx_n(N, pp, a, k, l) : tidx_n(N, k, a, pp, l);
        copy_piece<JC>(z + t * TS + (size_t)i * W + j0,
                       sm + (kind ? L.A6 : L.A4) + a * L.P46 + (l - (l > a)) * JC);
    }
}

// One CTA per unit of the group; yS holds c' (C plus the spread of B) per
// tile.  The loads, the split and the stores of a CTA follow one another;
// two CTAs per SM overlap them.
template <int JC, bool ONE>
__global__ void __launch_bounds__(kP1Threads, 2) p1_kernel(const __grid_constant__ Group g)
{
    if (blockIdx.x == 0 && threadIdx.x < 2) g.counter[threadIdx.x] = 0;  // work counters of the D -> C sweep
    const P1Unit w = p1_unit<JC, ONE>(g, blockIdx.x);
    if (!w.live) return;
    extern __shared__ __align__(128) int sm[];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    p1_issue<JC, ONE>(g, w, sm, &bar);
    cp_async_wait_all();
    if (__syncthreads_or(!mbar_wait(&bar, 0))) {
        // give up: record it, let the copies in flight land (bounded), leave
        if (threadIdx.x == 0) atomicOr(&g.status->err, kDevTimeout);
        mbar_wait(&bar, 0);
        __syncthreads();
        return;
    }
    p1_split<JC>(w, sm);
    p1_store<JC>(w, sm);
    bulk_wait_read_all();  // shared memory stays valid until the bulk stores have read it
}

// Tile of the pair store holding D_abcd (a < c): ((pair(a,c) N + b)(N-1) + d').
__device__ __forceinline__ int tidx_h(int N, int a, int b, int c, int d)
{
    return ((pair_index(a, c) * N + b) * (N - 1)) + (d - (d > b));
}

// The same pass for the pair store (reading of Sec. 6's complementary
// submatrices): of each class only the members of tiles whose first facility
// is below the second exist -- kind 1 (tile (i,j,k,n), row p), kind 2 (tile
// (i,j,p,q), row k) and kind 4 (tile (k,n,p,q), row i) -- each holding the sum
// with its complement (kinds 3, 5 and 6), whose c' shares it also receives;
// the class sum is split equally over the three, in lexicographic order.
template <int JC, bool ONE>
__global__ void __launch_bounds__(kP1Threads, 2) p1_pair_kernel(const __grid_constant__ Group g)
{
    if (blockIdx.x == 0 && threadIdx.x < 2) g.counter[threadIdx.x] = 0;  // work counters of the D -> C sweep
    const NodeDesc &nd =
        ONE ? g.first
            : g.nodes[find_node(g.nodes, g.B, blockIdx.x, [](const NodeDesc &d) { return (long long)d.cta_base; })];
    const PassState p = nd.p;
    if (*p.stop) return;
    const int N = nd.N, W = nd.W, nchunks = nd.nchunks;
    const FastDiv fN = nd.fN, fn = nd.fn;
    const int bid = blockIdx.x - nd.cta_base;
    extern __shared__ __align__(128) int sm[];
    const P1Layout L = p1_layout(N, W, JC, false, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t TS = (size_t)(N - 2) * W;
    const int4 tr = g.triples[bid / nchunks];
    const int i = tr.x, k = tr.y, pp = tr.z;
    const int j0 = (bid % nchunks) * JC;
    const int jc = min(JC, N - j0);
    int *__restrict__ z = p.z;
    const int NN = N * N;

    __shared__ __align__(8) uint64_t bar;
    const bool tma = JC == 4 && nd.zmap_ok;
    const void *zmap = &nd.zmap;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!ONE && tma) tensormap_acquire(zmap);
    }
    __syncthreads();
    const unsigned rowBytes = (unsigned)W * 4u;
    if (threadIdx.x == 0) {
        const unsigned pieceBytes = tma ? (unsigned)(N * L.P46) * 4u : 0u;
        mbar_arrive_expect_tx(&bar, (unsigned)(2 * jc * (N - 1)) * rowBytes + pieceBytes);
        if (tma) tensor_load5(sm + L.A4, zmap, j0, i, 0, 0, pair_index(k, pp), &bar);  // kind 4: tiles (k,a,p,l), row i
    }
    for (int e = threadIdx.x; e < 2 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        // kind 1: tile (i,j,k,x) row p; kind 2: tile (i,j,p,x) row k
        const int t = q == 0 ? tidx_h(N, i, j, k, x) : tidx_h(N, i, j, pp, x);
        const int row = q == 0 ? pp - 2 : k - 1;
        int *dst = q == 0 ? sm + L.A1 + (jj * N + x) * L.S13 : sm + L.A2 + (jj * N + x) * L.S25;
        bulk_load_tx(dst, z + t * TS + (size_t)row * W, rowBytes, &bar);
    }
    for (int e = tma ? NN : threadIdx.x; e < NN; e += kP1Threads) {
        const int a = (int)fdiv((unsigned)e, fN), l = e - a * N;
        if (l == a) continue;
        cp_async_piece<JC>(sm + L.A4 + a * L.P46 + (l - (l > a)) * JC,
                           z + (size_t)tidx_h(N, k, a, pp, l) * TS + (size_t)i * W + j0);
    }
    // c' of all six member tiles (the complements' shares join their pairs)
    p1_gather_c<JC, false>(L, N, i, k, pp, j0, jc, fN, p.yS, nullptr, 0, sm);

    asm volatile("cp.async.wait_all;" ::: "memory");
    if (__syncthreads_or(!mbar_wait(&bar, 0))) {
        if (threadIdx.x == 0) atomicOr(&g.status->err, kDevTimeout);
        mbar_wait(&bar, 0);
        __syncthreads();
        return;
    }
    p1_shares<false>(L, N, i, k, pp, fn, sm);
    __syncthreads();

    for (int nn = warp; nn < N; nn += kP1Warps) {
        const int *h4 = sm + L.H4 + nn * N, *h6 = sm + L.H6 + nn;
        for (int qq = lane; qq < N; qq += 32) {
            if (qq == nn) continue;
            int *a4 = sm + L.A4 + nn * L.P46 + (qq - (qq > nn)) * JC;   // piece (nn, qq)
            int p4[JC];
            load_piece<JC>(p4, a4);
            const int h46 = h4[qq] + h6[qq * L.H6p];
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const int j = j0 + jj;
                if (jj >= jc || j == nn || j == qq) continue;
                const int rn = jj * N + nn, rq = jj * N + qq;
                int *a1 = sm + L.A1 + rn * L.S13 + qq;
                int *a2 = sm + L.A2 + rq * L.S25 + nn;
                const int T = *a1 + sm[L.H1 + rn] + sm[L.H3 + rn] + *a2 + sm[L.H2 + rq] + sm[L.H5 + rq] +
                              p4[jj] + h46;
                const int q3 = T / 3, rm = T - 3 * q3;
                *a1 = q3 + (0 < rm);      // d_ijknpq, d_ijpqkn, d_knpqij in lexicographic order
                *a2 = q3 + (1 < rm);
                p4[jj] = q3 + (2 < rm);
            }
            store_piece<JC>(a4, p4);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();

    for (int e = threadIdx.x; e < 2 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        const int t = q == 0 ? tidx_h(N, i, j, k, x) : tidx_h(N, i, j, pp, x);
        const int row = q == 0 ? pp - 2 : k - 1;
        const int *src = q == 0 ? sm + L.A1 + (jj * N + x) * L.S13 : sm + L.A2 + (jj * N + x) * L.S25;
        bulk_store(z + t * TS + (size_t)row * W, src, rowBytes);
    }
    if (tma && threadIdx.x == 0) tensor_store5(zmap, j0, i, 0, 0, pair_index(k, pp), sm + L.A4);
    bulk_commit();
    for (int e = tma ? NN : threadIdx.x; e < NN; e += kP1Threads) {
        const int a = (int)fdiv((unsigned)e, fN), l = e - a * N;
        if (l == a) continue;
        copy_piece<JC>(z + (size_t)tidx_h(N, k, a, pp, l) * TS + (size_t)i * W + j0,
                       sm + L.A4 + a * L.P46 + (l - (l > a)) * JC);
    }
    bulk_wait_read_all();  // shared memory stays valid until the bulk stores have read it
}

// The same pass for an instance in the class-sum store.  The reduced cost of a
// member is (its value from the class sum) - u_row - v_col of its tile's last
// LAP, and the six values of a class sum back to T (the split is lossless), so
// spread C -> D followed by the transfer between complementary costs is
//   T <- T + sum over the six members of (share of c' - u_row) - v_col,
// the split itself being implicit in the store.  The CTA stages the v rows and
// v pieces of the member tiles exactly as the tile-store pass stages tile rows
// (same layout, bulk and tensor copies from du instead of z) and the per-tile
// (share - u_row) terms in the H arrays; T is read and written in place.
template <int JC, bool ONE>
__global__ void __launch_bounds__(kP1Threads, 2) p1_sym_kernel(const __grid_constant__ Group g)
{
    if (blockIdx.x == 0 && threadIdx.x < 2) g.counter[threadIdx.x] = 0;  // work counters of the D -> C sweep
    const NodeDesc &nd =
        ONE ? g.first
            : g.nodes[find_node(g.nodes, g.B, blockIdx.x, [](const NodeDesc &d) { return (long long)d.cta_base; })];
    const PassState p = nd.p;
    if (*p.stop) return;
    const int N = nd.N, W = nd.W, nchunks = nd.nchunks;
    const FastDiv fN = nd.fN, fn = nd.fn;
    const int bid = blockIdx.x - nd.cta_base;
    extern __shared__ __align__(128) int sm[];
    const P1Layout L = p1_layout(N, W, JC, true);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tri = bid / nchunks;
    const int4 tr = g.triples[tri];
    const int i = tr.x, k = tr.y, pp = tr.z;
    const int j0 = (bid % nchunks) * JC;
    const int jc = min(JC, N - j0);
    const int *__restrict__ yS = p.yS;
    const int *__restrict__ du = p.du;
    const int DS = nd.DS, U0 = nd.U0;
    const int NN = N * N;
    int *__restrict__ Tb = p.T + (long long)tri * NN * N;  // this triple's classes [j][n][q]

    __shared__ __align__(8) uint64_t bar;
    const bool tma = JC == 4 && nd.zmap_ok;
    const void *zmap = &nd.zmap;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!ONE && tma) tensormap_acquire(zmap);
    }
    __syncthreads();
    const unsigned rowBytes = (unsigned)W * 4u;
    if (threadIdx.x == 0) {
        const unsigned pieceBytes = tma ? 2u * (unsigned)(N * L.P46) * 4u : 0u;
        mbar_arrive_expect_tx(&bar, (unsigned)(4 * jc * (N - 1)) * rowBytes + pieceBytes);
        if (tma) {
            tensor_load5(sm + L.A4, zmap, j0, 0, 0, pp - 1, k * N, &bar);  // v of tiles (k,a,p,l)
            tensor_load5(sm + L.A6, zmap, j0, 0, 0, k, pp * N, &bar);      // v of tiles (p,a,k,l)
        }
    }
    for (int e = threadIdx.x; e < 4 * JC * N; e += kP1Threads) {
        const int qj = (int)fdiv((unsigned)e, fN), x = e - qj * N;
        const int q = qj / JC, jj = qj % JC, j = j0 + jj;
        if (jj >= jc || x == j) continue;
        int t, row;
        full_row(q, N, i, k, pp, j, x, t, row);
        const int base = q == 0 ? L.A1 : q == 1 ? L.A3 : q == 2 ? L.A2 : L.A5;
        const int pitch = q < 2 ? L.S13 : L.S25;
        bulk_load_tx(sm + base + (jj * N + x) * pitch, du + (size_t)t * DS + U0, rowBytes, &bar);
    }
    for (int e = tma ? 2 * NN : threadIdx.x; e < 2 * NN; e += kP1Threads) {
        const int kind = e >= NN, r2 = e - kind * NN;
        const int a = (int)fdiv((unsigned)r2, fN), l = r2 - a * N;
        if (l == a) continue;
        const int t = kind ? tidx_n(N, pp, a, k, l) : tidx_n(N, k, a, pp, l);
        cp_async_piece<JC>(sm + (kind ? L.A6 : L.A4) + a * L.P46 + (l - (l > a)) * JC,
                           du + (size_t)t * DS + U0 + j0);
    }

    // ---- c' and u of every member tile at the member's row, gathered while
    // the copies fly; H <- share of c' - u below
    p1_gather_c<JC, true>(L, N, i, k, pp, j0, jc, fN, yS, du, DS, sm);

    asm volatile("cp.async.wait_all;" ::: "memory");
    if (__syncthreads_or(!mbar_wait(&bar, 0))) {
        if (threadIdx.x == 0) atomicOr(&g.status->err, kDevTimeout);
        mbar_wait(&bar, 0);
        __syncthreads();
        return;
    }
    p1_shares<true>(L, N, i, k, pp, fn, sm);
    __syncthreads();

    // ---- new class sums: warp per location n, lanes over q, each lane the
    // chunk's classes of its (n, q)
    for (int nn = warp; nn < N; nn += kP1Warps) {
        const int *h4 = sm + L.H4 + nn * N, *h6 = sm + L.H6 + nn;
        for (int qq = lane; qq < N; qq += 32) {
            if (qq == nn) continue;
            int p4[JC], p6[JC];
            load_piece<JC>(p4, sm + L.A4 + nn * L.P46 + (qq - (qq > nn)) * JC);
            load_piece<JC>(p6, sm + L.A6 + qq * L.P46 + (nn - (nn > qq)) * JC);
            const int h46 = (int)((unsigned)h4[qq] + (unsigned)h6[qq * L.H6p]);
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const int j = j0 + jj;
                if (jj >= jc || j == nn || j == qq) continue;
                const int rn = jj * N + nn, rq = jj * N + qq;
                // modular (unsigned) sums: the partial sums may leave int32,
                // the new class sum (a sum of six reduced costs) does not
                const unsigned vsum = (unsigned)sm[L.A1 + rn * L.S13 + qq] + (unsigned)sm[L.A3 + rn * L.S13 + qq] +
                                      (unsigned)sm[L.A2 + rq * L.S25 + nn] + (unsigned)sm[L.A5 + rq * L.S25 + nn] +
                                      (unsigned)p4[jj] + (unsigned)p6[jj];
                const unsigned hsum = (unsigned)sm[L.H1 + rn] + (unsigned)sm[L.H3 + rn] + (unsigned)sm[L.H2 + rq] +
                                      (unsigned)sm[L.H5 + rq] + (unsigned)h46;
                int *Tc = Tb + (j * N + nn) * N + qq;
                *Tc = (int)((unsigned)*Tc + hsum - vsum);
            }
        }
    }
}

// Reduced costs of D of a class-sum-store instance in the tile-store layout.
__global__ void materialize_kernel(const NodeDesc nd, int *out)
{
    const int N = nd.N, n = N - 2, m = N - 1, W = nd.W;
    const long long total = nd.tiles * n;  // (tile, row) pairs
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long t = e / n;
        const int r = (int)(e - t * n);
        const int nn = (int)(t % m), kk = (int)((t / m) % m), ij = (int)(t / ((long long)m * m));
        const int i = ij / N, j = ij % N, k = kk + (kk >= i), nl = nn + (nn >= j);
        const int lo = min(i, k), hi = max(i, k);
        int ep = r + (r >= lo);
        ep += (ep >= hi);
        const SymRow sr = sym_row(N, i, j, k, nl, ep);
        const int *d = nd.p.du + t * nd.DS;
        int *o = out + t * nd.TS + (long long)r * W;
        for (int f = 0; f < W; ++f)
            o[f] = (f < N && f != j && f != nl)
                       ? sym_member(nd.p.T[sr.base + (long long)f * sr.stride], sr.rank) - d[r] - d[nd.U0 + f]
                       : 0;
    }
}

cudaError_t launch_materialize(const NodeDesc &nd, int *out, cudaStream_t s)
{
    long long blocks = (nd.tiles * (nd.N - 2) + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    materialize_kernel<<<(unsigned)blocks, 256, 0, s>>>(nd, out);
    return cudaGetLastError();
}

// ------------------------------------------------ warm-started children
//
// The child of a node fixing facility f to location l inherits the node's
// dual state restricted to the permutations with pi(f) = l (indices of the
// child: the other facilities and locations, ascending):
//   LB' = LB + b_fl,  b'_kn = b_kn + c_flkn + c_knfl,
//   c'_knpq = c_knpq + d_flknpq + d_knflpq + d_knpqfl,  d' = d restricted.

// c_ijkn of an instance (i != k, j != n) from its reduced C.
__device__ __forceinline__ int c_at(const NodeDesc &nd, int i, int j, int k, int n)
{
    const int N = nd.N, m = N - 1;
    return nd.p.yC[(((size_t)i * N + j) * m + (k - (k > i))) * m + (n - (n > j))];
}

// d_ijknpq of an instance in the tile or pair store (distinct i, k, p;
// distinct j, n, q); the pair store's tiles with i > k hold 0.
__device__ __forceinline__ int d_at(const NodeDesc &nd, int i, int j, int k, int n, int p, int q)
{
    const int N = nd.N, m = N - 1;
    size_t t;
    if (nd.paired) {
        if (i > k) return 0;
        t = ((size_t)pair_index(i, k) * N + j) * m + (n - (n > j));
    } else {
        t = (((size_t)i * N + j) * m + (k - (k > i))) * m + (n - (n > j));
    }
    const int lo = min(i, k), hi = max(i, k);
    const int r = p - (p > lo) - (p > hi);
    return nd.p.z[t * nd.TS + (size_t)r * nd.W + q];
}

__global__ void child_bc_kernel(const NodeDesc par, const NodeDesc ch, int f, int l)
{
    const int M = ch.N, N = par.N, m = M - 1;
    const long long nb = (long long)M * M, nc = (long long)M * M * m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nb + nc;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nb) {
            const int x = (int)(e / M), y = (int)(e % M);
            const int k = x + (x >= f), n = y + (y >= l);
            ch.p.x[e] = par.p.x[k * N + n] + c_at(par, f, l, k, n) + c_at(par, k, n, f, l);
        } else {
            const long long t = e - nb;
            const int w1 = (int)(t % m), u1 = (int)((t / m) % m);
            const int xy = (int)(t / ((long long)m * m)), x = xy / M, y = xy % M;
            const int u = u1 + (u1 >= x), w = w1 + (w1 >= y);
            const int k = x + (x >= f), n = y + (y >= l), p = u + (u >= f), q = w + (w >= l);
            int v = c_at(par, k, n, p, q);
            if (par.p.z)
                v += d_at(par, f, l, k, n, p, q) + d_at(par, k, n, f, l, p, q) + d_at(par, k, n, p, q, f, l);
            ch.p.yC[t] = v;
        }
    }
}

// One thread per (child tile, row); the row is written whole (columns without
// coefficient 0).
__global__ void child_d_kernel(const NodeDesc par, const NodeDesc ch, int f, int l)
{
    const int M = ch.N, m = M - 1, n2 = M - 2, W = ch.W;
    const long long total = ch.dtiles * n2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long th = e / n2;
        const int r = (int)(e - th * n2);
        int x, y, u, w;
        const int w1 = (int)(th % m);
        if (ch.paired) {
            const long long pj = th / m;
            y = (int)(pj % M);
            pair_of((int)(pj / M), x, u);
            w = w1 + (w1 >= y);
        } else {
            const int u1 = (int)((th / m) % m), xy = (int)(th / ((long long)m * m));
            x = xy / M;
            y = xy % M;
            u = u1 + (u1 >= x);
            w = w1 + (w1 >= y);
        }
        const int lo = min(x, u), hi = max(x, u);
        int rr = r + (r >= lo);
        rr += (rr >= hi);                       // the row's child facility
        // parent indices of the tile's facilities and locations and of the row's facility
        const int k = x + (x >= f), n = y + (y >= l), p = u + (u >= f), q = w + (w >= l);
        const int pr = rr + (rr >= f);
        int *out = ch.p.z + th * ch.TS + (size_t)r * W;
        for (int z = 0; z < W; ++z)
            out[z] = (z < M && z != y && z != w) ? d_at(par, k, n, p, q, pr, z + (z >= l)) : 0;
    }
}

__global__ void child_scalars_kernel(const NodeDesc par, const NodeDesc ch, int f, int l)
{
    *ch.p.LB = *par.p.LB + par.p.x[f * par.N + l];
    *ch.p.iter = 0;
    *ch.p.stop = 0;
}

cudaError_t launch_child(const NodeDesc &par, const NodeDesc &ch, int f, int l, cudaStream_t s)
{
    const long long nbc = (long long)ch.N * ch.N * (1 + (long long)(ch.N - 1) * (ch.N - 1));
    long long blocks = (nbc + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    child_bc_kernel<<<(unsigned)blocks, 256, 0, s>>>(par, ch, f, l);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ch.p.z) {
        blocks = (ch.dtiles * (ch.N - 2) + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        child_d_kernel<<<(unsigned)blocks, 256, 0, s>>>(par, ch, f, l);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    child_scalars_kernel<<<1, 1, 0, s>>>(par, ch, f, l);
    return cudaGetLastError();
}

// Costs spreading from B to C (Sec. 4.2): c'_ijkn = c_ijkn + the share of b_ij
// of row k (k' = rank of k among the facilities != i), written to yS.  One
// thread per tile of the group.
template <bool ONE>
__global__ void spread_x_to_y_kernel(Group g)
{
    if (ONE && *g.first.p.stop) return;
    for (long long T = blockIdx.x * (long long)blockDim.x + threadIdx.x; T < g.tiles;
         T += (long long)gridDim.x * blockDim.x) {
        const NodeDesc &nd =
            ONE ? g.first : g.nodes[find_node(g.nodes, g.B, T, [](const NodeDesc &d) { return d.tile_base; })];
        if (*nd.p.stop) continue;
        const unsigned t = (unsigned)(T - nd.tile_base);
        const unsigned ij = fdiv(t, nd.fmm);
        const unsigned e = t - ij * nd.fmm.d;
        const int kk = (int)fdiv(e, nd.fm);
        nd.p.yS[t] = nd.p.yC[t] + share(nd.p.x[ij], nd.fm, kk);
    }
}

cudaError_t launch_spread_x(const Group &g, cudaStream_t s)
{
    long long blocks = (g.tiles + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (g.B == 1) spread_x_to_y_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(g);
    else spread_x_to_y_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(g);
    return cudaGetLastError();
}

// c_ijkn <- f_ik * d_jn  (initialisation of Algorithm 1)
__global__ void init_y_kernel(int *yC, int N, const int32_t *F, const int32_t *D)
{
    const int m = N - 1;
    const long long tiles = (long long)N * N * m * m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tiles;
         t += (long long)gridDim.x * blockDim.x) {
        const int nn = (int)(t % m), kk = (int)((t / m) % m);
        const int ij = (int)(t / ((long long)m * m));
        const int i = ij / N, j = ij % N;
        const int k = kk + (kk >= i), n = nn + (nn >= j);
        yC[t] = F[i * N + k] * D[j * N + n];
    }
}

__global__ void init_scalars_kernel(PassState p, long long lb_const)
{
    *p.LB = lb_const;
    *p.iter = 0;
    *p.stop = 0;
}

cudaError_t launch_init(const NodeDesc &nd, const int32_t *F, const int32_t *D,
                        const int32_t *Blin, long long lb_const, cudaStream_t s)
{
    const PassState &p = nd.p;
    cudaError_t e = cudaSuccess;
    if (p.z) e = cudaMemsetAsync(p.z, 0, (size_t)nd.dtiles * nd.TS * 4, s);
    if (e == cudaSuccess && p.T) e = cudaMemsetAsync(p.T, 0, (size_t)make_geom(nd.N).classes_ints * 4, s);
    if (e == cudaSuccess && p.du) e = cudaMemsetAsync(p.du, 0, (size_t)nd.tiles * nd.DS * 4, s);
    if (e != cudaSuccess) return e;
    long long grid = (nd.tiles + 255) / 256;
    if (grid > 8192) grid = 8192;
    init_y_kernel<<<(unsigned)grid, 256, 0, s>>>(p.yC, nd.N, F, D);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (Blin) e = cudaMemcpyAsync(p.x, Blin, (size_t)nd.N * nd.N * 4, cudaMemcpyDeviceToDevice, s);
    else e = cudaMemsetAsync(p.x, 0, (size_t)nd.N * nd.N * 4, s);
    if (e != cudaSuccess) return e;
    init_scalars_kernel<<<1, 1, 0, s>>>(p, lb_const);
    return cudaGetLastError();
}

template <int JC>
static cudaError_t p1_go(const Group &g, cudaStream_t s)
{
    const size_t smem = p1_smem_bytes(g.maxN, JC, g.sym, g.paired);
    auto k = g.sym      ? (g.B == 1 ? p1_sym_kernel<JC, true> : p1_sym_kernel<JC, false>)
             : g.paired ? (g.B == 1 ? p1_pair_kernel<JC, true> : p1_pair_kernel<JC, false>)
                        : (g.B == 1 ? p1_kernel<JC, true> : p1_kernel<JC, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<g.ctas, kP1Threads, smem, s>>>(g);
    return cudaGetLastError();
}

// Spread B -> C, then the fused spread C -> D / complementary D pass.
cudaError_t launch_p1(const Group &g, cudaStream_t s)
{
    cudaError_t e = launch_spread_x(g, s);
    if (e != cudaSuccess) return e;
    switch (g.JC) {
    case 4: return p1_go<4>(g, s);
    case 2: return p1_go<2>(g, s);
    default: return p1_go<1>(g, s);
    }
}

}  // namespace rlt2
