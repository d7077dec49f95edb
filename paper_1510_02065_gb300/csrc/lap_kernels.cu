// lap_kernels.cu -- the cost concentrations of Algorithm 1 (Sec. 4.1) on sm_103a.
//
//   dlap_kernel   concentration D -> C: one Hungarian LAP of size N-2 per tile
//                 D_ijkn; each tile (N-2 rows x W location columns, two of
//                 them without coefficient) comes into shared memory by one
//                 1-D bulk copy (cp.async.bulk completing on an mbarrier), work
//                 is taken from a global counter, the residual tile is written
//                 back in place and S goes to yS.
//   clap_kernel   transfer between complementary costs of C fused with the
//                 concentration C -> B (N^2 LAPs of size N-1).
//   xlap_kernel   concentration B -> LB (one LAP of size N), LB += LB', history,
//                 stopping rule of Algorithm 1.
//   lap_batch_kernel  the same Hungarian on caller-supplied matrices.
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "device.cuh"
#include "kernels.h"

namespace rlt2 {

// D->C LAPs on whole warps use the Hungarian's sentinel column: with packed
// keys the tile's dead column j (and the packed lane words), otherwise lane 31
// with one column slot per lane (a build can turn both off for comparison
// with -DRLT2_NO_SENTINEL)
#ifdef RLT2_NO_SENTINEL
constexpr bool kSentinel = false;
#else
constexpr bool kSentinel = true;
#endif

constexpr int kClapWarps = 4;
constexpr int kDlap16Warps = 4;
constexpr int kXlapWarps = 4;
constexpr int kBatchWarps = 4;

// ------------------------------------------------------------ D -> C sweep

// One tile of D -> C: bring tile t of instance nd into buf with one bulk copy,
// solve its LAP, write the residual tile back in place and S to yS.  Returns
// false if the copy did not complete within the spin limit (recorded in
// status; the copy in flight has landed or been waited for, bounded).
// SEG = 16: the calling half-warp solves the tile (N <= 16), lane = its lane in the half.
// PAIR: t indexes the pair store (tiles with i < k holding the sum of the two
// complementary submatrices); S goes to c_ijkn and c_knij, which receives no
// concentration, is set to 0 (everything it had was spread to D).
template <int NS, bool PACK, int SEG = 32, bool PAIR = false>
__device__ __forceinline__ bool dlap_tile(const NodeDesc &nd, unsigned t, int *buf, uint64_t *bar,
                                          unsigned &parity, int lane, unsigned &steps, unsigned &relax,
                                          DevStatus *status)
{
    const Seg<SEG> sg;
    const int N = nd.N, W = nd.W, n = N - 2, m = N - 1, TS = nd.TS;
    if (lane == 0) {
        fence_proxy_async_smem();
        bulk_load(buf, nd.p.z + (size_t)t * TS, (unsigned)TS * 4u, bar);
    }
    if (!__all_sync(sg.mask, mbar_wait(bar, parity))) {
        if (lane == 0) atomicOr(&status->err, kDevTimeout);
        mbar_wait(bar, parity);
        __syncwarp(sg.mask);
        return false;
    }
    parity ^= 1u;

    // the tile's own locations j and n are the columns without coefficient
    int j, nn;
    unsigned tf = t, tlow = 0;  // tile of C receiving S; PAIR: the complement's
    if constexpr (PAIR) {
        const unsigned pj = fdiv(t, nd.fm);  // t = (pair * N + j) * m + n'
        nn = (int)(t - pj * (unsigned)m);
        const unsigned pr = fdiv(pj, nd.fN);
        j = (int)(pj - pr * (unsigned)N);
        int i, k;
        pair_of((int)pr, i, k);
        const int nl0 = nn + (nn >= j);
        tf = (((unsigned)i * N + j) * m + (k - 1)) * m + nn;                          // (i,j,k,n), k' = k - 1
        tlow = (((unsigned)k * N + nl0) * m + i) * m + (unsigned)(j - (j > nl0));       // (k,n,i,j), i' = i
    } else {
        const unsigned ij = fdiv(t, nd.fmm);
        const unsigned rem = t - ij * (unsigned)(m * m);
        nn = (int)(rem - fdiv(rem, nd.fm) * (unsigned)m);
        j = (int)(ij - fdiv(ij, nd.fN) * (unsigned)N);
    }
    const int nl = nn + (nn >= j);
    int rowOf[NS], uM[NS], v[NS];
    if (!warp_hungarian<NS, PACK, SEG, kSentinel && SEG == 32 && (NS == 1 || PACK)>(buf, W, n, N, j, nl, rowOf, uM, v, steps, relax) &&
        lane == 0)
        atomicOr(&status->err, kDevInternal);
    // u of every row goes to the row's column j, which holds no coefficient
    scatter_rows<NS, SEG>(n, N, j, nl, rowOf, uM, buf + j, nullptr, W);
    __syncwarp(sg.mask);
    int *gz = nd.p.z + (size_t)t * TS;
    for (int r = 0; r < n; ++r) {
        const int ur = buf[r * W + j];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int c = lane + 32 * s;
            if (c < W) gz[r * W + c] = (c < N && c != j && c != nl) ? buf[r * W + c] - ur - v[s] : 0;
        }
    }
    const long long S = lap_value<NS, SEG>(N, j, nl, uM, v);
    if (lane == 0) {
        nd.p.yS[tf] = (int)S;
        if constexpr (PAIR) nd.p.yS[tlow] = 0;
    }
    // the generic writes of column j above precede the next tile's bulk copy
    // into this buffer (async proxy)
    fence_proxy_async_smem();
    __syncwarp(sg.mask);
    return true;
}

// The same for an instance in the class-sum store: the tile is gathered from
// the class sums (one 4-byte asynchronous copy per coefficient, all in flight
// at once), each coefficient becomes its member value in place, and the LAP's
// duals (u of every row, v of every location column) go to du instead of a
// residual tile.
template <int NS, bool PACK, int SEG = 32>
__device__ __forceinline__ bool dlap_tile_sym(const NodeDesc &nd, unsigned t, int *buf, int lane,
                                              unsigned &steps, unsigned &relax, DevStatus *status)
{
    const Seg<SEG> sg;
    const int N = nd.N, W = nd.W, n = N - 2, m = N - 1;
    const unsigned ij = fdiv(t, nd.fmm);
    const unsigned rem = t - ij * (unsigned)(m * m);
    const int kk = (int)fdiv(rem, nd.fm), nn = (int)rem - kk * m;
    const int i = (int)fdiv(ij, nd.fN), j = (int)ij - i * N;
    const int k = kk + (kk >= i), nl = nn + (nn >= j);
    // Rows are the facilities e not in {i,k}, ascending; with a < c the tile's
    // two facilities (at locations la, lc), the rows fall in three ranges whose
    // classes are (e,a,c), (a,e,c), (a,c,e).  Within a range the member rank is
    // fixed and the class index tau = C(z,3) + C(y,2) + x grows by 1, e, C(e,2)
    // from one row to the next, so row addresses advance without division.
    const bool ik = i < k;
    const int a = ik ? i : k, c = ik ? k : i, la = ik ? j : nl, lc = ik ? nl : j;
    const int R0 = ik ? 3 : 5, R1 = ik ? 1 : 4, R2 = ik ? 0 : 2;
    const long long N3 = (long long)N * N * N;
    const int N2 = N * N;
    const int C3c = c * (c - 1) * (c - 2) / 6, C2c = c * (c - 1) / 2, C2a = a * (a - 1) / 2;
    const int *T = nd.p.T;
    bool valid[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int f = lane + 32 * s;
        valid[s] = f < N && f != j && f != nl;
    }
    int r = 0;
    long long base = (long long)(C3c + C2a) * N3 + (long long)la * N + lc;        // e = 0: (e, a, c)
    for (int e = 0; e < a; ++e, ++r, base += N3) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (valid[s]) cp_async4(buf + r * W + lane + 32 * s, T + base + (long long)(lane + 32 * s) * N2);
    }
    base = (long long)(C3c + (a + 1) * a / 2 + a) * N3 + (long long)la * N2 + lc;  // e = a + 1: (a, e, c)
    for (int e = a + 1; e < c; base += (long long)e * N3, ++e, ++r) {  // step C(e+1,2) - C(e,2) = e
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (valid[s]) cp_async4(buf + r * W + lane + 32 * s, T + base + (long long)(lane + 32 * s) * N);
    }
    base = (long long)((c + 1) * c * (c - 1) / 6 + C2c + a) * N3 + (long long)la * N2 + (long long)lc * N;
    for (int e = c + 1; e < N; base += (long long)(e * (e - 1) / 2) * N3, ++e, ++r) {  // (a, c, e); step C(e,2)
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (valid[s]) cp_async4(buf + r * W + lane + 32 * s, T + base + lane + 32 * s);
    }
    cp_async_wait_all();
    __syncwarp(sg.mask);
    for (int rr = 0; rr < n; ++rr) {
        const int rank = rr < a ? R0 : rr < c - 1 ? R1 : R2;
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (valid[s]) buf[rr * W + lane + 32 * s] = sym_member(buf[rr * W + lane + 32 * s], rank);
    }
    __syncwarp(sg.mask);
    int rowOf[NS], uM[NS], v[NS];
    if (!warp_hungarian<NS, PACK, SEG, kSentinel && SEG == 32 && (NS == 1 || PACK)>(buf, W, n, N, j, nl, rowOf, uM, v, steps, relax) &&
        lane == 0)
        atomicOr(&status->err, kDevInternal);
    scatter_rows<NS, SEG>(n, N, j, nl, rowOf, uM, buf + j, nullptr, W);  // u to the free column j
    __syncwarp(sg.mask);
    int *du = nd.p.du + (size_t)t * nd.DS;
    for (int r = lane; r < n; r += SEG) du[r] = buf[r * W + j];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int f = lane + 32 * s;
        if (f < W) du[nd.U0 + f] = (f < N && f != j && f != nl) ? v[s] : 0;
    }
    const long long S = lap_value<NS, SEG>(N, j, nl, uM, v);
    if (lane == 0) nd.p.yS[t] = (int)S;
    __syncwarp(sg.mask);
    return true;
}

// One tile buffer per warp (and one mbarrier: WARPS * (TS * 4 + 8) bytes of
// shared memory per CTA of WARPS warps); a warp takes group-wide tile indices
// from a global counter, finds the tile's instance and solves the tile's LAP.
// Tiles of one instance are consecutive in the group-wide order, so the
// instance found for the previous tile is tried first.  ONE (a group of one
// instance): the instance is the kernel parameter g.first, read from
// parameter space, and the stopping rule is checked once.
// MODE: 0 tile store, 1 class-sum store, 2 pair store (work units: its tiles).
// Resident warps per SM each D->C form is compiled for, i.e. its register
// budget (65536 / 32 / warps).  Two column slots per lane (N >= 32): a tile
// buffer of at least 7.7 KB per warp keeps fewer than 30 warps resident, so
// these forms get 64 registers (32 warps) and never spill.  One slot: a group
// of one reads its instance from kernel parameters and fits 32 registers (64
// warps).  A larger group holds its instances' fields in registers: with the
// tile or pair store it would take 38-43 and spills 40-56 bytes per thread at
// 32, which measured faster at 64 warps than 48 warps without spills (C4
// batch: 28.0 vs 27.5 nodes/s); with the class-sum store's gather it takes up
// to 64 (64 registers, 32 warps; 16 bytes spilled).
template <int NS, bool ONE, int MODE>
constexpr int kDlapWarpsPerSM = NS == 2 ? 32 : ONE ? 64 : MODE == 1 ? 32 : 64;

template <int NS, bool PACK, bool ONE, int MODE, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kDlapWarpsPerSM<NS, ONE, MODE> / WARPS)
    dlap_kernel(Group g, long long lo, long long hi, unsigned *counter, int tsp)
{
    constexpr bool SYM = MODE == 1, PAIR = MODE == 2;
    if (ONE && *g.first.p.stop) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *buf = reinterpret_cast<int *>(smem) + (size_t)warp * tsp;
    unsigned char *tail = smem + (size_t)WARPS * tsp * 4;
    uint64_t *bar = reinterpret_cast<uint64_t *>(tail) + warp;

    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();

    unsigned parity = 0;
    unsigned steps = 0, relax = 0, laps = 0;
    const unsigned ntiles = (unsigned)hi;  // < 2^31 for any group the host accepts
    int b = 0;
    for (;;) {
        unsigned T = 0;
        if (lane == 0) T = atomicAdd(counter, 1u) + (unsigned)lo;
        T = __shfl_sync(kFull, T, 0);
        if (T >= ntiles) break;
        bool ok;
        if constexpr (SYM && ONE) {
            ok = dlap_tile_sym<NS, PACK>(g.first, T, buf, lane, steps, relax, g.status);
        } else if constexpr (SYM) {
            if (T < (unsigned)g.nodes[b].dtile_base || (b + 1 < g.B && T >= (unsigned)g.nodes[b + 1].dtile_base))
                b = find_node(g.nodes, g.B, T, [](const NodeDesc &d) { return d.dtile_base; });
            const NodeDesc &nd = g.nodes[b];
            if (*nd.p.stop) continue;
            ok = dlap_tile_sym<NS, PACK>(nd, T - (unsigned)nd.dtile_base, buf, lane, steps, relax, g.status);
        } else if constexpr (ONE) {
            ok = dlap_tile<NS, PACK, 32, PAIR>(g.first, T, buf, bar, parity, lane, steps, relax, g.status);
        } else {
            if (T < (unsigned)g.nodes[b].dtile_base || (b + 1 < g.B && T >= (unsigned)g.nodes[b + 1].dtile_base))
                b = find_node(g.nodes, g.B, T, [](const NodeDesc &d) { return d.dtile_base; });
            const NodeDesc &nd = g.nodes[b];
            if (*nd.p.stop) continue;
            ok = dlap_tile<NS, PACK, 32, PAIR>(nd, T - (unsigned)nd.dtile_base, buf, bar, parity, lane, steps,
                                               relax, g.status);
        }
        if (!ok) return;
        ++laps;
    }
    if (lane == 0 && laps) {
        atomicAdd(&g.status->laps, (unsigned long long)laps);
        atomicAdd(&g.status->steps, (unsigned long long)steps);
        atomicAdd(&g.status->relax, (unsigned long long)relax);
        atomicAdd(&g.status->dlaps, (unsigned long long)laps);
        atomicAdd(&g.status->dsteps, (unsigned long long)steps);
        atomicAdd(&g.status->drelax, (unsigned long long)relax);
    }
}

// Tiles of instances with N <= 16 (a range [lo, hi) of the group's units,
// from its own counter): two per warp, one per half-warp (LAPs of width <= 16
// on 16 lanes).  Two buffers of tsp ints and two mbarriers per warp; half h
// always uses buffer and barrier h.
// (register budget as above: 39-44 registers with the tile store, more than
// 64 with the class-sum store)
template <bool PACK, bool ONE, bool SYM>
__global__ void __launch_bounds__(kDlap16Warps * 32, (SYM ? 24 : 40) / kDlap16Warps)
    dlap16_kernel(Group g, long long lo, long long hi, unsigned *counter, int tsp)
{
    if (ONE && *g.first.p.stop) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    int *buf = reinterpret_cast<int *>(smem) + ((size_t)warp * 2 + half) * tsp;
    unsigned char *tail = smem + (size_t)kDlap16Warps * 2 * tsp * 4;
    uint64_t *bar = reinterpret_cast<uint64_t *>(tail) + warp * 2 + half;

    if (hl == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();

    unsigned parity = 0;
    unsigned steps = 0, relax = 0, laps = 0;
    const unsigned small = (unsigned)hi, units = (unsigned)((hi - lo + 1) / 2);
    int b = 0;
    for (;;) {
        unsigned U = 0;
        if (lane == 0) U = atomicAdd(counter, 1u);
        U = __shfl_sync(kFull, U, 0);
        if (U >= units) break;
        const unsigned T = (unsigned)lo + 2u * U + (unsigned)half;
        bool ok = true;
        if (T < small) {
            if constexpr (ONE) {
                if constexpr (SYM) ok = dlap_tile_sym<1, PACK, 16>(g.first, T, buf, hl, steps, relax, g.status);
                else ok = dlap_tile<1, PACK, 16>(g.first, T, buf, bar, parity, hl, steps, relax, g.status);
                laps += ok;
            } else {
                if (T < (unsigned)g.nodes[b].dtile_base || (b + 1 < g.B && T >= (unsigned)g.nodes[b + 1].dtile_base))
                    b = find_node(g.nodes, g.B, T, [](const NodeDesc &d) { return d.dtile_base; });
                const NodeDesc &nd = g.nodes[b];
                if (!*nd.p.stop) {
                    const unsigned t = T - (unsigned)nd.dtile_base;
                    if constexpr (SYM) ok = dlap_tile_sym<1, PACK, 16>(nd, t, buf, hl, steps, relax, g.status);
                    else ok = dlap_tile<1, PACK, 16>(nd, t, buf, bar, parity, hl, steps, relax, g.status);
                    laps += ok;
                }
            }
        }
        if (__any_sync(kFull, !ok)) return;  // a half gave up (recorded); leave together
    }
    if (hl == 0 && laps) {
        atomicAdd(&g.status->laps, (unsigned long long)laps);
        atomicAdd(&g.status->steps, (unsigned long long)steps);
        atomicAdd(&g.status->relax, (unsigned long long)relax);
        atomicAdd(&g.status->dlaps, (unsigned long long)laps);
        atomicAdd(&g.status->dsteps, (unsigned long long)steps);
        atomicAdd(&g.status->drelax, (unsigned long long)relax);
    }
}

// -------------------------------------------- complementary C + C -> B

// One warp per C->B problem (instance, i, j) of the group.
template <int NS, bool PACK>
__global__ void __launch_bounds__(kClapWarps * 32) clap_kernel(Group g, int pitch)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *buf = reinterpret_cast<int *>(smem) + (size_t)warp * pitch;
    unsigned steps = 0, relax = 0, laps = 0;
    for (int P = blockIdx.x * kClapWarps + warp; P < g.probs; P += gridDim.x * kClapWarps) {
        const NodeDesc &nd =
            g.nodes[find_node(g.nodes, g.B, P, [](const NodeDesc &d) { return (long long)d.prob_base; })];
        const PassState &p = nd.p;
        if (*p.stop) continue;
        const int N = nd.N, m = N - 1;
        int *uRow = buf + m * m;
        const int prob = P - nd.prob_base;
        const int i = prob / N, j = prob % N;
        const long long base = (long long)prob * m * m;
        // transfer between the complementary pair {c_ijkn, c_knij} (Eq. (10)):
        // the lexicographically first member (i < k) takes the odd unit
        for (int e = lane; e < m * m; e += 32) {
            const int kk = e / m, nn = e % m;
            const int k = kk + (kk >= i), n = nn + (nn >= j);
            const int i2 = i - (i > k), j2 = j - (j > n);
            const long long t2 = ((long long)(k * N + n) * m + i2) * m + j2;
            const int T = p.yS[base + e] + p.yS[t2];
            buf[e] = i < k ? T - T / 2 : T / 2;
        }
        __syncwarp();
        int rowOf[NS], uM[NS], v[NS];
        if (!warp_hungarian_full<NS, PACK>(buf, m, m, rowOf, uM, v, steps, relax) && lane == 0)
            atomicOr(&g.status->err, kDevInternal);
        scatter_rows<NS>(m, m, -1, -1, rowOf, uM, uRow, nullptr);
        __syncwarp();
        for (int r = 0; r < m; ++r) {
            const int ur = uRow[r];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int c = lane + 32 * s;
                if (c < m) p.yC[base + r * m + c] = buf[r * m + c] - ur - v[s];
            }
        }
        const long long S = lap_value<NS>(m, -1, -1, uM, v);
        if (lane == 0) p.x[prob] = (int)S;
        ++laps;
        __syncwarp();
    }
    if (lane == 0 && laps) {
        atomicAdd(&g.status->laps, (unsigned long long)laps);
        atomicAdd(&g.status->steps, (unsigned long long)steps);
        atomicAdd(&g.status->relax, (unsigned long long)relax);
    }
}

// ------------------------------------------------------------- B -> LB

// One warp per instance of the group.
template <int NS, bool PACK>
__global__ void __launch_bounds__(kXlapWarps * 32) xlap_kernel(Group g, int pitch)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kXlapWarps + warp;
    if (b >= g.B) return;
    const NodeDesc &nd = g.nodes[b];
    const PassState &p = nd.p;
    if (*p.stop) return;
    const int N = nd.N;
    int *buf = reinterpret_cast<int *>(smem) + (size_t)warp * pitch;
    int *uRow = buf + N * N;
    for (int e = lane; e < N * N; e += 32) buf[e] = p.x[e];
    __syncwarp();
    unsigned steps = 0, relax = 0;
    int rowOf[NS], uM[NS], v[NS];
    if (!warp_hungarian_full<NS, PACK>(buf, N, N, rowOf, uM, v, steps, relax) && lane == 0)
        atomicOr(&g.status->err, kDevInternal);
    scatter_rows<NS>(N, N, -1, -1, rowOf, uM, uRow, nullptr);
    __syncwarp();
    for (int r = 0; r < N; ++r) {
        const int ur = uRow[r];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int c = lane + 32 * s;
            if (c < N) p.x[r * N + c] = buf[r * N + c] - ur - v[s];
        }
    }
    const long long S = lap_value<NS>(N, -1, -1, uM, v);
    if (lane == 0) {
        const long long lb = *p.LB + S;
        *p.LB = lb;
        const int it = *p.iter;
        if (it < p.hist_cap) p.hist[it] = lb;
        *p.iter = it + 1;
        // stopping rule of Algorithm 1: continue while progress >= K and LB < UB
        if (p.ub > 0.0) {
            if ((double)lb >= p.ub) *p.stop = 1;
            if (p.min_progress > 0.0 && (double)S / p.ub < p.min_progress) *p.stop = 1;
        }
        atomicAdd(&g.status->laps, 1ull);
        atomicAdd(&g.status->steps, (unsigned long long)steps);
        atomicAdd(&g.status->relax, (unsigned long long)relax);
    }
}

// ------------------------------------------------------------- LAP batch

template <int NS>
__global__ void __launch_bounds__(kBatchWarps * 32)
    lap_batch_kernel(const int32_t *__restrict__ M, int n, int count, int64_t *S, int32_t *assign,
                     int32_t *uo, int32_t *vo, int64_t *work, DevStatus *status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *buf = reinterpret_cast<int *>(smem) + (size_t)warp * (n * n + 128);
    int *uRow = buf + n * n;
    int *colOf = uRow + 64;
    for (int prob = blockIdx.x * kBatchWarps + warp; prob < count; prob += gridDim.x * kBatchWarps) {
        const int32_t *src = M + (size_t)prob * n * n;
        int mx = 0, bad = 0;
        for (int e = lane; e < n * n; e += 32) {
            const int a = src[e];
            buf[e] = a;
            mx = max(mx, a);
            bad |= (a < 0) | (a > 536870911);
        }
        bad = __any_sync(kFull, bad);
        mx = __reduce_max_sync(kFull, mx);
        __syncwarp();
        if (bad) {
            if (lane == 0) {
                S[prob] = -1;
                atomicOr(&status->err, kDevRange);
            }
            continue;
        }
        unsigned steps = 0, relax = 0;
        int rowOf[NS], uM[NS], v[NS];
        const bool fine = mx < (1 << 25) / 3
                              ? warp_hungarian_full<NS, true>(buf, n, n, rowOf, uM, v, steps, relax)
                              : warp_hungarian_full<NS, false>(buf, n, n, rowOf, uM, v, steps, relax);
        if (!fine && lane == 0) atomicOr(&status->err, kDevInternal);
        scatter_rows<NS>(n, n, -1, -1, rowOf, uM, uRow, colOf);
        __syncwarp();
        const long long s = lap_value<NS>(n, -1, -1, uM, v);
        for (int e = lane; e < n; e += 32) {
            if (assign) assign[(size_t)prob * n + e] = colOf[e];
            if (uo) uo[(size_t)prob * n + e] = uRow[e];
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int c = lane + 32 * k;
            if (vo && c < n) vo[(size_t)prob * n + c] = v[k];
        }
        if (lane == 0) {
            S[prob] = s;
            if (work) {
                work[2 * (size_t)prob] = steps;
                work[2 * (size_t)prob + 1] = relax;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------ failure detection

// A warp waits on an mbarrier that is never completed (its one arrival is
// expected with bytes no copy will deliver; no copy is issued): the bounded
// wait gives up after `limit` polls and records kDevTimeout, the same path
// every wait of the library takes.  Nothing is in flight, nothing faults.
__global__ void wait_selftest_kernel(DevStatus *status, unsigned limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (!__all_sync(kFull, mbar_wait(&bar, 0, limit)) && threadIdx.x == 0) atomicOr(&status->err, kDevTimeout);
}

cudaError_t launch_wait_selftest(DevStatus *status, unsigned limit, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(status, limit);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- launchers

// Resident CTAs per SM of kernel k with `threads` threads and `smem` bytes of
// dynamic shared memory on the current device, 0 when smem exceeds a CTA's
// opt-in maximum.  The first query for a kernel raises its dynamic
// shared-memory cap to that maximum (a cap only: occupancy follows the bytes
// a launch asks for); answers are cached per kernel, device and size, so a
// launch costs no driver queries after its first one.
static cudaError_t ctas_per_sm(const void *k, int threads, size_t smem, int &per_sm)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> cache;
    static std::set<std::pair<const void *, int>> capped;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(k, dev, threads, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) {
        per_sm = it->second;
        return cudaSuccess;
    }
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    per_sm = 0;
    if (smem <= (size_t)optin) {
        if (!capped.count({k, dev})) {
            if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)) != cudaSuccess)
                return e;
            capped.insert({k, dev});
        }
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem)) != cudaSuccess) return e;
    }
    cache[key] = per_sm;
    return cudaSuccess;
}

// Resident warps per SM of the D->C kernel with CTAs of WARPS warps (0 when its
// tile buffers exceed a CTA's shared memory: 16 warps from N = 61, 32 warps
// from N = 44).
template <int NS, bool PACK, bool ONE, int MODE, int WARPS>
static cudaError_t dlap_fit(const DlapRange &rg, int &warps_per_sm)
{
    const size_t smem = (size_t)WARPS * ((size_t)rg.tsp * 4 + 8);
    int per_sm = 0;
    const cudaError_t e =
        ctas_per_sm(reinterpret_cast<const void *>(dlap_kernel<NS, PACK, ONE, MODE, WARPS>), WARPS * 32, smem, per_sm);
    warps_per_sm = per_sm * WARPS;
    return e;
}

template <int NS, bool PACK, bool ONE, int MODE, int WARPS>
static cudaError_t dlap_run(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s)
{
    const size_t smem = (size_t)WARPS * ((size_t)rg.tsp * 4 + 8);
    int per_sm = 0;
    cudaError_t e = ctas_per_sm(reinterpret_cast<const void *>(dlap_kernel<NS, PACK, ONE, MODE, WARPS>), WARPS * 32,
                                smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sm_count;
    const long long need = (rg.hi - rg.lo + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    dlap_kernel<NS, PACK, ONE, MODE, WARPS><<<(unsigned)grid, WARPS * 32, smem, s>>>(g, rg.lo, rg.hi, rg.counter,
                                                                                   rg.tsp);
    return cudaGetLastError();
}

// CTA size: rg.warps (4, 16 or 32) when given, else the one of those that
// keeps the most warps resident (shared memory decides: at N = 30 two CTAs of
// 32 warps fit where fourteen of 4 do), the smaller on a tie.
// chosen != null: report the CTA size in *chosen and launch nothing.
template <int NS, bool PACK, bool ONE, int MODE>
static cudaError_t dlap_go(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s,
                           int *chosen = nullptr)
{
    int w4 = 0, w16 = 0, w32 = 0;
    cudaError_t e;
    if ((e = dlap_fit<NS, PACK, ONE, MODE, 4>(rg, w4)) != cudaSuccess) return e;
    if ((e = dlap_fit<NS, PACK, ONE, MODE, 16>(rg, w16)) != cudaSuccess) return e;
    if ((e = dlap_fit<NS, PACK, ONE, MODE, 32>(rg, w32)) != cudaSuccess) return e;
    int w = rg.warps;
    if (w == 0) w = (w32 > w4 && w32 > w16) ? 32 : w16 > w4 ? 16 : 4;
    if ((w == 4 && !w4) || (w == 16 && !w16) || (w == 32 && !w32)) return cudaErrorInvalidConfiguration;
    if (chosen) {
        *chosen = w;
        return cudaSuccess;
    }
    if (w == 32) return dlap_run<NS, PACK, ONE, MODE, 32>(g, rg, sm_count, s);
    if (w == 16) return dlap_run<NS, PACK, ONE, MODE, 16>(g, rg, sm_count, s);
    if (w == 4) return dlap_run<NS, PACK, ONE, MODE, 4>(g, rg, sm_count, s);
    return cudaErrorInvalidValue;
}

// One column slot per lane (with the sentinel column in lane 31) up to N = 31,
// two from N = 32.
template <bool ONE, int MODE>
static cudaError_t dlap_pick(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s, int *chosen)
{
    if (rg.maxN <= 31)
        return g.pack ? dlap_go<1, true, ONE, MODE>(g, rg, sm_count, s, chosen)
                      : dlap_go<1, false, ONE, MODE>(g, rg, sm_count, s, chosen);
    return g.pack ? dlap_go<2, true, ONE, MODE>(g, rg, sm_count, s, chosen)
                  : dlap_go<2, false, ONE, MODE>(g, rg, sm_count, s, chosen);
}

static cudaError_t dlap_warp(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s,
                             int *chosen = nullptr)
{
    if (g.sym)
        return g.B == 1 ? dlap_pick<true, 1>(g, rg, sm_count, s, chosen) : dlap_pick<false, 1>(g, rg, sm_count, s, chosen);
    if (g.paired)
        return g.B == 1 ? dlap_pick<true, 2>(g, rg, sm_count, s, chosen) : dlap_pick<false, 2>(g, rg, sm_count, s, chosen);
    return g.B == 1 ? dlap_pick<true, 0>(g, rg, sm_count, s, chosen) : dlap_pick<false, 0>(g, rg, sm_count, s, chosen);
}

template <bool PACK, bool ONE, bool SYM>
static cudaError_t dlap16_go(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s)
{
    const size_t smem = (size_t)kDlap16Warps * ((size_t)rg.tsp * 2 * 4 + 16);
    auto k = dlap16_kernel<PACK, ONE, SYM>;
    int per_sm = 0;
    cudaError_t e = ctas_per_sm(reinterpret_cast<const void *>(k), kDlap16Warps * 32, smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sm_count;
    const long long need = ((rg.hi - rg.lo) / 2 + 1 + kDlap16Warps - 1) / kDlap16Warps;
    if (grid > need) grid = need;
    k<<<(unsigned)grid, kDlap16Warps * 32, smem, s>>>(g, rg.lo, rg.hi, rg.counter, rg.tsp);
    return cudaGetLastError();
}

template <bool ONE, bool SYM>
static cudaError_t dlap16_pick(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s)
{
    return g.pack ? dlap16_go<true, ONE, SYM>(g, rg, sm_count, s) : dlap16_go<false, ONE, SYM>(g, rg, sm_count, s);
}

static cudaError_t dlap_half(const Group &g, const DlapRange &rg, int sm_count, cudaStream_t s)
{
    if (g.paired) return cudaErrorInvalidValue;  // the half-warp form serves the tile and class-sum stores
    if (g.sym) return g.B == 1 ? dlap16_pick<true, true>(g, rg, sm_count, s) : dlap16_pick<false, true>(g, rg, sm_count, s);
    return g.B == 1 ? dlap16_pick<true, false>(g, rg, sm_count, s) : dlap16_pick<false, false>(g, rg, sm_count, s);
}

// The group's two D->C ranges: [small_tiles, dtiles) (counter 0) and the
// small instances' [0, small_tiles) (counter 1), each in its own shape.
static DlapRange dlap_range(const Group &g, int which)
{
    DlapRange rg;
    if (which == 0) {
        rg.lo = g.small_tiles;
        rg.hi = g.dtiles;
        rg.counter = g.counter;
        rg.tsp = g.maxTS;
        rg.maxW = (g.maxN + 3) & ~3;
        rg.maxN = g.maxN;
    } else {
        rg.lo = 0;
        rg.hi = g.small_tiles;
        rg.counter = g.counter + 1;
        rg.tsp = g.smallTS;
        rg.maxW = g.smallW;
        rg.maxN = g.smallW;   // N <= W <= 16
    }
    rg.lanes = g.dshape[which].lanes;
    rg.warps = g.dshape[which].warps;
    return rg;
}

int dlap_cta_warps(const Group &g, int which)
{
    const DlapRange rg = dlap_range(g, which);
    if (rg.hi <= rg.lo) return 0;
    if (rg.lanes == 16) return kDlap16Warps;
    int w = 0;
    return dlap_warp(g, rg, 0, nullptr, &w) == cudaSuccess ? w : 0;
}

cudaError_t launch_dlap_range(const Group &g, int which, int sm_count, cudaStream_t s)
{
    const DlapRange rg = dlap_range(g, which);
    if (rg.hi <= rg.lo) return cudaSuccess;
    if (rg.lanes == 16) {
        if (rg.maxW > 16) return cudaErrorInvalidValue;
        return dlap_half(g, rg, sm_count, s);
    }
    return dlap_warp(g, rg, sm_count, s);
}

cudaError_t launch_dlap(const Group &g, int sm_count, cudaStream_t s, const SideStream *side)
{
    if (g.small_tiles <= 0) return launch_dlap_range(g, 0, sm_count, s);
    cudaError_t e;
    if (!side) {
        if ((e = launch_dlap_range(g, 1, sm_count, s)) != cudaSuccess) return e;
        return launch_dlap_range(g, 0, sm_count, s);
    }
    // fork: the small instances' range on the side stream, the rest here; join
    // before returning
    if ((e = cudaEventRecord(side->fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side->s2, side->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_dlap_range(g, 1, sm_count, side->s2)) != cudaSuccess) return e;
    if ((e = launch_dlap_range(g, 0, sm_count, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(side->join, side->s2)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, side->join, 0);
}

template <int NS, bool PACK>
static cudaError_t clap_go(const Group &g, cudaStream_t s)
{
    const int m = g.maxN - 1;
    const int pitch = m * m + 64;
    const size_t smem = (size_t)kClapWarps * pitch * 4;
    auto k = clap_kernel<NS, PACK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (g.probs + kClapWarps - 1) / kClapWarps;
    k<<<grid, kClapWarps * 32, smem, s>>>(g, pitch);
    return cudaGetLastError();
}

cudaError_t launch_clap(const Group &g, cudaStream_t s)
{
    if (g.rlt1_only) {
        // without D, the input of C -> B is C plus the spread of B
        cudaError_t e = launch_spread_x(g, s);
        if (e != cudaSuccess) return e;
    }
    if (g.maxN - 1 <= 32) return g.pack ? clap_go<1, true>(g, s) : clap_go<1, false>(g, s);
    return g.pack ? clap_go<2, true>(g, s) : clap_go<2, false>(g, s);
}

template <int NS, bool PACK>
static cudaError_t xlap_go(const Group &g, cudaStream_t s)
{
    const int pitch = g.maxN * g.maxN + 64;
    const size_t smem = (size_t)kXlapWarps * pitch * 4;
    auto k = xlap_kernel<NS, PACK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(g.B + kXlapWarps - 1) / kXlapWarps, kXlapWarps * 32, smem, s>>>(g, pitch);
    return cudaGetLastError();
}

cudaError_t launch_xlap(const Group &g, cudaStream_t s)
{
    if (g.maxN <= 32) return g.pack ? xlap_go<1, true>(g, s) : xlap_go<1, false>(g, s);
    return g.pack ? xlap_go<2, true>(g, s) : xlap_go<2, false>(g, s);
}

template <int NS>
static cudaError_t batch_go(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                            int32_t *u, int32_t *v, int64_t *work, DevStatus *status, cudaStream_t s)
{
    const size_t smem = (size_t)kBatchWarps * ((size_t)n * n + 128) * 4;
    auto k = lap_batch_kernel<NS>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = (count + kBatchWarps - 1) / kBatchWarps;
    if (grid > 65535) grid = 65535;
    k<<<grid, kBatchWarps * 32, smem, s>>>(M, n, count, S, assign, u, v, work, status);
    return cudaGetLastError();
}

cudaError_t launch_lap_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                             int32_t *u, int32_t *v, int64_t *work, DevStatus *status,
                             cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    if (n <= 32) return batch_go<1>(M, n, count, S, assign, u, v, work, status, s);
    return batch_go<2>(M, n, count, S, assign, u, v, work, status, s);
}

}  // namespace rlt2
