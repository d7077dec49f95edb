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
// JC columns j of rows shared with the CTAs of the other chunks.  The CTA stages
// them in shared memory with 16-byte loads, splits every class, and writes the
// rows back.  With i < k < p the lexicographic ranks of kinds 1..6 are 0..5.
// Full rows move by 1-D bulk copies (cp.async.bulk) completing on one
// mbarrier; the column pieces by 4-byte cp.async; all loads of a CTA are in
// flight at once, and two CTAs per SM overlap one's copies with the other's
// arithmetic.
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

// r-th element of [0, N) without a and b (a != b)
__device__ __forceinline__ int skip2(int r, int a, int b)
{
    const int lo = min(a, b), hi = max(a, b);
    r += (r >= lo);
    r += (r >= hi);
    return r;
}

// Shared-memory layout of one work unit (offsets in ints).  Full tile rows
// (kinds 1, 3, 2, 5) keep the global row stride RS so that they move by bulk
// copies; the JC-column pieces of kinds 4 and 6 use an odd row pitch.
struct P1Layout {
    int n, m, JCp, P4;
    int BAR, A1, A3, A2, A5, A4, A6, H1, H3, H2, H5, H4, H6, total;
};

__host__ __device__ inline P1Layout p1_layout(int N, int JC, int RS)
{
    P1Layout L;
    L.n = N - 2;
    L.m = N - 1;
    L.JCp = JC | 1;
    L.P4 = L.m * L.JCp;
    if (!(L.P4 & 1)) L.P4 += 1;
    int o = 0;
    L.BAR = o; o += 4;  // one mbarrier, 16-byte slot
    L.A1 = o; o += JC * L.m * RS;
    L.A3 = o; o += JC * L.m * RS;
    L.A2 = o; o += JC * L.m * RS;
    L.A5 = o; o += JC * L.m * RS;
    L.A4 = o; o += N * L.P4;
    L.A6 = o; o += N * L.P4;
    L.H1 = o; o += JC * L.m;
    L.H3 = o; o += JC * L.m;
    L.H2 = o; o += JC * L.m;
    L.H5 = o; o += JC * L.m;
    L.H4 = o; o += N * L.m;
    L.H6 = o; o += N * L.m;
    L.total = o;
    return L;
}

size_t p1_smem_bytes(int N, int JC)
{
    const int RS = (N - 2 + 3) & ~3;
    return (size_t)p1_layout(N, JC, RS).total * 4;
}

int p1_chunk(int N)
{
    for (int jc : {4, 2}) if (p1_smem_bytes(N, jc) <= 110 * 1024) return jc;
    return 1;
}

// Tile and tile row of the full rows: kind q (0: kind 1, 1: kind 3, 2: kind 2,
// 3: kind 5), location j of the smallest facility, other location l.
__device__ __forceinline__ void full_row(int q, int N, int i, int k, int pp, int j, int l, int &t,
                                         int &row)
{
    if (q == 0) { t = tidx_n(N, i, j, k, l); row = pp - 2; }        // d_ijklpq: tile (i,j,k,l), row p
    else if (q == 1) { t = tidx_n(N, k, l, i, j); row = pp - 2; }   // d_klijpq: tile (k,l,i,j), row p
    else if (q == 2) { t = tidx_n(N, i, j, pp, l); row = k - 1; }   // d_ijplkn: tile (i,j,p,l), row k
    else { t = tidx_n(N, pp, l, i, j); row = k - 1; }               // d_plijkn: tile (p,l,i,j), row k
}

template <int JC>
__global__ void __launch_bounds__(kP1Threads, 2)
    p1_kernel(PassState p, int N, int RS, const int4 *__restrict__ triples, int nchunks,
              FastDiv fm, FastDiv fn)
// fm divides by N-1, fn by N-2; yS holds c' (C plus the spread of B) per tile
{
    if (*p.stop) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.counter = 0;  // work counter of the D -> C sweep
    extern __shared__ __align__(128) int sm[];
    const P1Layout L = p1_layout(N, JC, RS);
    const int n = L.n, m = L.m;
    const size_t TS = (size_t)n * RS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 tr = triples[blockIdx.x / nchunks];
    const int i = tr.x, k = tr.y, pp = tr.z;
    const int j0 = (blockIdx.x % nchunks) * JC;
    const int jc = min(JC, N - j0);
    const int *__restrict__ yS = p.yS;
    int *__restrict__ z = p.z;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.BAR);
    const unsigned rowBytes = (unsigned)RS * 4u;

    if (threadIdx.x == 0) {
        mbar_init(bar, 4 * 32);
        fence_mbar_init();
    }
    __syncthreads();

    // ---- issue every load: full rows by bulk copies (warps 0-3, one kind
    // each), the JC-column pieces of kinds 4 and 6 by 4-byte cp.async
    if (warp < 4) {
        const int q = warp;
        const int ab = q == 0 ? L.A1 : q == 1 ? L.A3 : q == 2 ? L.A2 : L.A5;
        const int mine = lane < m ? (m - 1 - lane) / 32 + 1 : 0;
        mbar_arrive_expect_tx(bar, (unsigned)(jc * mine) * rowBytes);
        for (int jj = 0; jj < jc; ++jj) {
            const int j = j0 + jj;
            for (int o = lane; o < m; o += 32) {
                const int l = o + (o >= j);
                int t, row;
                full_row(q, N, i, k, pp, j, l, t, row);
                bulk_load_tx(sm + ab + (jj * m + o) * RS, z + t * TS + row * RS, rowBytes, bar);
            }
        }
    } else {
        // one thread per row (a, o): row i of tile (k,a,p,l) (kind 4) or of
        // tile (p,a,k,l) (kind 6); for a fixed a these tiles are consecutive
        const int tw = (warp - 4) * 32 + lane, nt = (kP1Warps - 4) * 32;
        for (int ro = tw; ro < 2 * N * m; ro += nt) {
            const int kind = ro >= N * m;
            const int r2 = ro - kind * N * m;
            const int a = (int)fdiv((unsigned)r2, fm), o = r2 - a * m;
            const int l = o + (o >= a);
            const int t = (kind ? ((pp * N + a) * m + k) * m : ((k * N + a) * m + pp - 1) * m) + o;
            // the share of c' of this tile that row i receives
            sm[(kind ? L.H6 : L.H4) + a * m + o] = share(yS[t], fn, i);
            const int *src = z + t * TS + (size_t)i * RS;
            int *dst = sm + (kind ? L.A6 : L.A4) + a * L.P4 + o * L.JCp;
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const int j = j0 + jj;
                if (jj < jc && j != a && j != l) cp_async4(dst + jj, src + (j - (j > a) - (j > l)));
            }
        }
    }

    // ---- shares of the full rows while the copies fly: c' of the tile (c plus
    // the share of b, computed by the spread kernel into yS) over the tile's rows
    for (int q = warp; q < 4 * JC; q += kP1Warps) {
        const int kind = q / JC, jj = q % JC, j = j0 + jj;
        if (jj >= jc) continue;
        const int hb = kind == 0 ? L.H1 : kind == 1 ? L.H3 : kind == 2 ? L.H2 : L.H5;
        for (int o = lane; o < m; o += 32) {
            const int l = o + (o >= j);
            int t, row;
            full_row(kind, N, i, k, pp, j, l, t, row);
            sm[hb + jj * m + o] = share(yS[t], fn, row);
        }
    }

    cp_async_wait_all();
    const bool ok = __syncthreads_and(mbar_wait(bar, 0));
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(&p.status->err, kDevTimeout);
        mbar_wait(bar, 0);   // let the copies in flight land (bounded), then leave
        return;
    }

    // ---- split every class {(i,j),(k,nn),(p,qq)}, j in the chunk: one warp
    // per (j, nn), lanes over the column s of qq in the kind-1 row
    for (int jj = 0; jj < jc; ++jj) {
        const int j = j0 + jj;
        for (int o = warp; o < m; o += kP1Warps) {
            const int nn = o + (o >= j);
            const int h1 = sm[L.H1 + jj * m + o], h3 = sm[L.H3 + jj * m + o];
            int *r1 = sm + L.A1 + (jj * m + o) * RS;
            int *r3 = sm + L.A3 + (jj * m + o) * RS;
            for (int s = lane; s < n; s += 32) {
                const int qq = skip2(s, j, nn);
                const int q1 = qq - (qq > j);          // rank of qq among locations != j
                const int s2 = o - (nn > qq);          // column of nn in tiles (.,j,.,qq)/(.,qq,.,j)
                const int q4 = qq - (qq > nn);         // rank of qq among locations != nn
                const int n6 = nn - (nn > qq);         // rank of nn among locations != qq
                int *a2 = sm + L.A2 + (jj * m + q1) * RS + s2;
                int *a5 = sm + L.A5 + (jj * m + q1) * RS + s2;
                int *a4 = sm + L.A4 + nn * L.P4 + q4 * L.JCp + jj;
                int *a6 = sm + L.A6 + qq * L.P4 + n6 * L.JCp + jj;
                const int T = r1[s] + h1 + *a2 + sm[L.H2 + jj * m + q1] + r3[s] + h3 +
                              *a4 + sm[L.H4 + nn * m + q4] + *a5 + sm[L.H5 + jj * m + q1] +
                              *a6 + sm[L.H6 + qq * m + n6];
                const int q6 = T / 6, rm = T - 6 * q6;
                r1[s] = q6 + (0 < rm);   // ranks: d_ijknpq 0, d_ijpqkn 1, d_knijpq 2,
                *a2 = q6 + (1 < rm);     //        d_knpqij 3, d_pqijkn 4, d_pqknij 5
                r3[s] = q6 + (2 < rm);
                *a4 = q6 + (3 < rm);
                *a5 = q6 + (4 < rm);
                *a6 = q6 + (5 < rm);
            }
        }
    }
    fence_proxy_async_smem();
    __syncthreads();

    // ---- write back: full rows by bulk stores, column pieces by plain stores
    if (warp < 4) {
        const int q = warp;
        const int ab = q == 0 ? L.A1 : q == 1 ? L.A3 : q == 2 ? L.A2 : L.A5;
        for (int jj = 0; jj < jc; ++jj) {
            const int j = j0 + jj;
            for (int o = lane; o < m; o += 32) {
                const int l = o + (o >= j);
                int t, row;
                full_row(q, N, i, k, pp, j, l, t, row);
                bulk_store(z + t * TS + row * RS, sm + ab + (jj * m + o) * RS, rowBytes);
            }
        }
        bulk_commit();
        bulk_wait_read_all();
    } else {
        const int tw = (warp - 4) * 32 + lane, nt = (kP1Warps - 4) * 32;
        for (int ro = tw; ro < 2 * N * m; ro += nt) {
            const int kind = ro >= N * m;
            const int r2 = ro - kind * N * m;
            const int a = (int)fdiv((unsigned)r2, fm), o = r2 - a * m;
            const int l = o + (o >= a);
            const int t = (kind ? ((pp * N + a) * m + k) * m : ((k * N + a) * m + pp - 1) * m) + o;
            int *dst = z + t * TS + (size_t)i * RS;
            const int *src = sm + (kind ? L.A6 : L.A4) + a * L.P4 + o * L.JCp;
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const int j = j0 + jj;
                if (jj < jc && j != a && j != l) dst[j - (j > a) - (j > l)] = src[jj];
            }
        }
    }
}

// Costs spreading from B to C (Sec. 4.2): c'_ijkn = c_ijkn + the share of b_ij
// of row k (k' = rank of k among the facilities != i), written to yS.  One
// block row per (i, j), threads over the (N-1)^2 entries of C_ij.
__global__ void spread_x_to_y_kernel(PassState p, int N, FastDiv fm)
{
    if (*p.stop) return;
    const int m = N - 1;
    const int ij = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int kk = (int)fdiv((unsigned)e, fm);
    const long long t = (long long)ij * m * m + e;
    p.yS[t] = p.yC[t] + share(p.x[ij], fm, kk);
}

cudaError_t launch_spread_x(const Geom &g, const PassState &p, cudaStream_t s)
{
    const int m = g.N - 1;
    dim3 grid((m * m + 255) / 256, g.N * g.N);
    spread_x_to_y_kernel<<<grid, 256, 0, s>>>(p, g.N, make_fastdiv(m));
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
    DevStatus z = {};
    *p.status = z;
}

cudaError_t launch_init(const Geom &g, const PassState &p, const int32_t *F, const int32_t *D,
                        const int32_t *Blin, long long lb_const, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (p.z) e = cudaMemsetAsync(p.z, 0, (size_t)g.tiles * g.TS * 4, s);
    if (e != cudaSuccess) return e;
    int grid = (int)((g.tiles + 255) / 256);
    if (grid > 8192) grid = 8192;
    init_y_kernel<<<grid, 256, 0, s>>>(p.yC, g.N, F, D);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (Blin) e = cudaMemcpyAsync(p.x, Blin, (size_t)g.N * g.N * 4, cudaMemcpyDeviceToDevice, s);
    else e = cudaMemsetAsync(p.x, 0, (size_t)g.N * g.N * 4, s);
    if (e != cudaSuccess) return e;
    init_scalars_kernel<<<1, 1, 0, s>>>(p, lb_const);
    return cudaGetLastError();
}

template <int JC>
static cudaError_t p1_go(const Geom &g, const PassState &p, const int4 *triples, int ntriples,
                         cudaStream_t s)
{
    const size_t smem = p1_smem_bytes(g.N, JC);
    auto k = p1_kernel<JC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nchunks = (g.N + JC - 1) / JC;
    k<<<ntriples * nchunks, kP1Threads, smem, s>>>(p, g.N, g.RS, triples, nchunks,
                                                    make_fastdiv(g.N - 1), make_fastdiv(g.N - 2));
    return cudaGetLastError();
}

cudaError_t launch_p1(const Geom &g, const PassState &p, const int4 *triples, int ntriples,
                      cudaStream_t s)
{
    cudaError_t e = launch_spread_x(g, p, s);
    if (e != cudaSuccess) return e;
    switch (p1_chunk(g.N)) {
    case 4: return p1_go<4>(g, p, triples, ntriples, s);
    case 2: return p1_go<2>(g, p, triples, ntriples, s);
    default: return p1_go<1>(g, p, triples, ntriples, s);
    }
}

}  // namespace rlt2
