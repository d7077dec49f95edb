// f64.cu -- the FP64 form of the dual ascent on sm_103a and its C ABI
// (rlt2_f64_*): the paper's real division of a spread cost (Sec. 4.2) and the
// equal re-split T/s of a class of complementary costs (Sec. 4.3), with double
// costs, potentials and bound.
//
// Every floating-point operation is the one the FP64 form defines, in its
// order, so that device and definition agree bit for bit:
//   spread B->C   c_ijkn = c_ijkn + b_ij / (N-1)
//   spread C->D   d_ijknpq = d_ijknpq + c_ijkn / (N-2), c_ijkn = 0
//   complementary D  T = 0 + six members in lexicographic rank order; each = T/6
//                 (spread C->D and this transfer run as one kernel)
//   D->C          c_ijkn = 0 + S; D_ijkn = (M - u) - v      (Hungarian below)
//   complementary C  T = c_ijkn + c_knij (i < k); both = T/2
//   C->B, B->LB   b_ij = b_ij + S, LB = LB + S; residuals (M - u) - v
// One kernel per operation (the two spreads into D fused); the LAP kernels run
// one warp per problem.
//
// Layouts: x = b[i][j] (N*N); y = c in tile order t = ((i*N + j)(N-1) + k')(N-1)
// + n' (C_ij is a contiguous (N-1)^2 block); z = tile t holds N-2 rows (p not
// in {i,k}, ascending) of N location columns (columns j and n hold nothing).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rlt2.h"
#include "device.cuh"

namespace rlt2 {
namespace {

constexpr int kF64Warps = 4;       // warps per CTA of the LAP kernels
constexpr int kF64Threads = 256;   // CTA size of the element-wise kernels

struct F64Dev {
    int N, n, m;          // n = N - 2, m = N - 1
    int TS;               // doubles per tile of z: n * N
    long long tiles;      // N^2 (N-1)^2
    long long classes;    // C(N,3) N (N-1) (N-2)
    const int32_t *F, *D;
    double *x, *y, *z;
    double *LB, *hist;
    int *iter;
    int hist_cap;
    const int4 *triples;  // facility triples a < b < c
    DevStatus *status;
};

// Order-preserving int64 image of a double that is not NaN: comparing images
// as signed integers is comparing the doubles, with -0.0 equal to +0.0.
__device__ __forceinline__ long long okey(double x)
{
    long long b = __double_as_longlong(x);
    b = b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
    return b == -1LL ? 0LL : b;
}

// Warp-wide least (key, column), ties to the smallest column; INT_MAX if no
// lane offers a column (key LLONG_MAX, column INT_MAX).
__device__ __forceinline__ int warp_argmin(long long key, int col)
{
    const int hi = (int)(key >> 32);
    const int mh = __reduce_min_sync(kFull, hi);
    const unsigned lo = hi == mh ? (unsigned)key : 0xffffffffu;
    const unsigned ml = __reduce_min_sync(kFull, lo);
    return __reduce_min_sync(kFull, (hi == mh && (unsigned)key == ml) ? col : INT_MAX);
}

// Hungarian method of the FP64 form, one warp per LAP (shortest augmenting
// paths from u = v = 0, rows inserted in ascending order, argmin ties to the
// smallest column, a label and its predecessor change only on a strict
// improvement; the potentials move by delta after every step).  Column c of
// the matrix lives in lane c % 32, slot c / 32: its potential v, distance
// label, predecessor, labelled flag, the row matched to it and that row's
// potential uM.  The row being inserted keeps its potential in the uM slot of
// column dead0 when there is one (a column without coefficient, which is
// never matched), so that one addition moves it with the rows of the labelled
// columns; else in a register.  The labelled columns' v and the unlabelled
// columns' distance labels move by the same -delta in one addition.  M row r
// at M + r * ld; the LAP's n columns are the indices c < width other than
// dead0 and dead1, in ascending order.
// Out: rowOf, uM, v per column slot; S = the sum over the columns in ascending
// order of M[row][column], from 0; steps, relax += the work (as the int form
// counts it).  Returns false if an invariant fails (not for finite entries).
template <int NS>
__device__ bool hungarian_f64(const double *M, int ld, int n, int width, int dead0, int dead1,
                              int (&rowOf)[NS], double (&uM)[NS], double (&v)[NS], double &S,
                              unsigned &steps, unsigned &relax)
{
    const int lane = threadIdx.x & 31;
    const double kInfD = __longlong_as_double(0x7ff0000000000000LL);
    const bool rootInLane = dead0 >= 0;
    const int rl = dead0 & 31, rs = dead0 >> 5;
    bool valid[NS], root[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int c = lane + 32 * s;
        valid[s] = c < width && c != dead0 && c != dead1;
        root[s] = c == dead0;
        rowOf[s] = -1;
        uM[s] = 0.0;
        v[s] = 0.0;
    }
    for (int r = 0; r < n; ++r) {
        double dist[NS];
        int way[NS];
        bool lab[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            dist[s] = kInfD;
            way[s] = -1;
            lab[s] = false;
            if (root[s]) uM[s] = 0.0;  // u of row r before its insertion
        }
        double ur = 0.0, ui0 = 0.0;
        int col = -1, i0 = r, next = -1, K = 0;
        for (;;) {
            if (++K > n + 1) return false;
            const double *Mr = M + (size_t)i0 * ld + lane;
            long long best = LLONG_MAX;
            int bc = INT_MAX;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (valid[s] && !lab[s]) {
                    const double red = (Mr[32 * s] - ui0) - v[s];
                    long long kd = okey(dist[s]);
                    const long long kr = okey(red);
                    if (kr < kd) {
                        dist[s] = red;
                        way[s] = col;
                        kd = kr;
                    }
                    if (kd < best) {
                        best = kd;
                        bc = lane + 32 * s;
                    }
                }
            }
            next = warp_argmin(best, bc);
            if (next == INT_MAX) return false;
            // one slot per lane: the column is the lane itself
            const int src = NS == 1 ? next : next & 31, sl = NS == 1 ? 0 : next >> 5;
            const double delta = __shfl_sync(kFull, pick<NS>(dist, sl), src);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (valid[s]) {
                    const double moved = (lab[s] ? v[s] : dist[s]) - delta;
                    if (lab[s]) v[s] = moved;
                    else dist[s] = moved;
                }
                if (lab[s] || root[s]) uM[s] += delta;
            }
            if (!rootInLane) ur += delta;
            const int rj = __shfl_sync(kFull, pick<NS>(rowOf, sl), src);
            const double uj = __shfl_sync(kFull, pick<NS>(uM, sl), src);
            if (rj < 0) break;  // free column: augmenting path found
            if (lane == src) put<NS>(lab, sl, true);
            col = next;
            i0 = rj;
            ui0 = uj;
        }
        steps += (unsigned)K;
        relax += (unsigned)(n * K - K * (K - 1) / 2);
        if (rootInLane) ur = __shfl_sync(kFull, pick<NS>(uM, rs), rl);
        // augment: each column on the path takes the row (and its potential)
        // of its predecessor; the first takes row r
        int c = next;
        for (int hop = 0;; ++hop) {
            if (hop > n) return false;
            // (one slot per lane: columns are lanes; a shuffle from lane -1
            // reads lane 31, whose values a predecessor -1 ignores)
            const int cs = NS == 1 ? 0 : c >> 5, cl = NS == 1 ? c : c & 31;
            const int w = __shfl_sync(kFull, pick<NS>(way, cs), cl);
            const int ws = NS == 1 ? 0 : (w < 0 ? 0 : w) >> 5, wl = NS == 1 ? w : (w < 0 ? 0 : w) & 31;
            const int pr = __shfl_sync(kFull, pick<NS>(rowOf, ws), wl);
            const double pu = __shfl_sync(kFull, pick<NS>(uM, ws), wl);
            if (lane == cl) {
                put<NS>(rowOf, cs, w < 0 ? r : pr);
                put<NS>(uM, cs, w < 0 ? ur : pu);
            }
            if (w < 0) break;
            c = w;
        }
    }
    double xs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) xs[s] = valid[s] && rowOf[s] >= 0 ? M[(size_t)rowOf[s] * ld + lane + 32 * s] : 0.0;
    double sum = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
        for (int l = 0; l < 32; ++l) {
            const double xv = __shfl_sync(kFull, xs[s], l);
            const int c = l + 32 * s;
            if (c < width && c != dead0 && c != dead1) sum += xv;
        }
    S = sum;
    return true;
}

__device__ __forceinline__ void decode_tile(const F64Dev &d, long long t, int &i, int &j, int &k, int &n)
{
    const int m = d.m;
    const int nn = (int)(t % m);
    const long long q = t / m;
    const int kk = (int)(q % m);
    const int ij = (int)(q / m);
    i = ij / d.N;
    j = ij - i * d.N;
    k = kk + (kk >= i);
    n = nn + (nn >= j);
}

__global__ void f64_init_kernel(F64Dev d)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d.tiles;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k, n;
        decode_tile(d, t, i, j, k, n);
        d.y[t] = (double)((long long)d.F[i * d.N + k] * (long long)d.D[j * d.N + n]);
    }
}

// spread B -> C: every c_ijkn += b_ij / (N-1)  (b is cleared afterwards)
__global__ void f64_spread_x_kernel(F64Dev d)
{
    const long long mm = (long long)d.m * d.m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d.tiles;
         t += (long long)gridDim.x * blockDim.x)
        d.y[t] += d.x[t / mm] / (double)(d.N - 1);
}

// Spread C -> D fused with the transfer between complementary costs of D: one
// CTA per facility triple a < b < c and location la, i.e. the classes
// {(a,la),(b,lb),(c,lc)} for every lb != la and lc not in {la, lb}.  Their
// members, in lexicographic rank order, are
//   m0 = d(a la, b lb, c lc)  row c of tile (a,la,b,lb), column lc
//   m1 = d(a la, c lc, b lb)  row b of tile (a,la,c,lc), column lb
//   m2 = d(b lb, a la, c lc)  row c of tile (b,lb,a,la), column lc
//   m3 = d(b lb, c lc, a la)  row a of tile (b,lb,c,lc), column la
//   m4 = d(c lc, a la, b lb)  row b of tile (c,lc,a,la), column lb
//   m5 = d(c lc, b lb, a la)  row a of tile (c,lc,b,lb), column la
// Kinds 0, 1, 2, 4 fill whole tile rows (every coefficient of such a row
// belongs to one of the CTA's classes), so they move as contiguous rows
// through shared memory; kinds 3 and 5 are single coefficients.  Each
// coefficient first takes its tile's share (z + c/(N-2): spread C -> D), then
// T = 0 + m0 + ... + m5 and every member becomes T/6.  On entry y holds the
// shares (f64_share_kernel); it is not cleared here (other CTAs read it):
// D -> C writes c = 0 + S.
__global__ void __launch_bounds__(kF64Threads) f64_p1_kernel(F64Dev d)
{
    extern __shared__ double f64_smem[];
    const int N = d.N, m = d.m, TS = d.TS, NN = N * N;
    const int4 tr = d.triples[blockIdx.x / N];
    const int la = (int)(blockIdx.x % N);
    const int a = tr.x, b = tr.y, c = tr.z;
    double *A[4] = {f64_smem, f64_smem + NN, f64_smem + 2 * NN, f64_smem + 3 * NN};
    auto tile = [&](int i, int j, int k, int n) -> long long {
        return ((long long)(i * N + j) * m + (k - (k > i))) * m + (n - (n > j));
    };
    // row source of kind slot s (0: m0, 1: m1, 2: m2, 3: m4) for the row's own location x
    auto row_tile = [&](int s, int x) -> long long {
        return s == 0 ? tile(a, la, b, x) : s == 1 ? tile(a, la, c, x) : s == 2 ? tile(b, x, a, la) : tile(c, x, a, la);
    };
    auto row_of = [&](int s) -> int { return (s == 0 || s == 2) ? c - 2 : b - 1; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int sr = warp; sr < 4 * N; sr += nw) {
        const int s = sr / N, x = sr - s * N;
        if (x == la) continue;
        const long long t = row_tile(s, x);
        const double sh = d.y[t];  // the tile's share c/(N-2)
        const double *src = d.z + (size_t)t * TS + (size_t)row_of(s) * N;
        double *dst = A[s] + x * N;
        for (int q = lane; q < N; q += 32) {
            double v = src[q];
            if (q != la && q != x) v = v + sh;
            dst[q] = v;
        }
    }
    __syncthreads();
    const int cls = (N - 1) * (N - 2);
    for (int e = threadIdx.x; e < cls; e += blockDim.x) {
        const int lbp = e / (N - 2), lcp = e - lbp * (N - 2);
        const int lb = lbp + (lbp >= la);
        const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
        int lc = lcp + (lcp >= lo);
        lc += (lc >= hi);
        const long long t3 = tile(b, lb, c, lc), t5 = tile(c, lc, b, lb);
        double *p3 = d.z + (size_t)t3 * TS + (size_t)a * N + la;
        double *p5 = d.z + (size_t)t5 * TS + (size_t)a * N + la;
        const double m3 = *p3 + d.y[t3];
        const double m5 = *p5 + d.y[t5];
        double T = 0.0;
        T += A[0][lb * N + lc];
        T += A[1][lc * N + lb];
        T += A[2][lb * N + lc];
        T += m3;
        T += A[3][lc * N + lb];
        T += m5;
        const double each = T / 6.0;
        A[0][lb * N + lc] = each;
        A[1][lc * N + lb] = each;
        A[2][lb * N + lc] = each;
        A[3][lc * N + lb] = each;
        *p3 = each;
        *p5 = each;
    }
    __syncthreads();
    for (int sr = warp; sr < 4 * N; sr += nw) {
        const int s = sr / N, x = sr - s * N;
        if (x == la) continue;
        double *dst = d.z + (size_t)row_tile(s, x) * TS + (size_t)row_of(s) * N;
        const double *src = A[s] + x * N;
        for (int q = lane; q < N; q += 32)
            if (q != la && q != x) dst[q] = src[q];
    }
}

// c_ijkn <- c_ijkn / (N-2): the share of every coefficient of tile D_ijkn in
// spread C -> D, formed once per tile (f64_p1_kernel adds it)
__global__ void f64_share_kernel(F64Dev d)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d.tiles;
         t += (long long)gridDim.x * blockDim.x)
        d.y[t] = d.y[t] / (double)(d.N - 2);
}

// concentration D -> C, one warp per tile (tile and u of its rows in shared memory)
template <int NS>
__global__ void __launch_bounds__(kF64Warps * 32) f64_dlap_kernel(F64Dev d)
{
    extern __shared__ double f64_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int TS = d.TS, n = d.n, N = d.N;
    double *buf = f64_smem + (size_t)warp * (TS + n);
    double *uRow = buf + TS;
    unsigned steps = 0, relax = 0, laps = 0;
    bool ok = true;
    const long long nw = (long long)gridDim.x * kF64Warps;
    for (long long t = blockIdx.x * (long long)kF64Warps + warp; t < d.tiles; t += nw) {
        int i, j, k, nl;
        decode_tile(d, t, i, j, k, nl);
        double *zt = d.z + (size_t)t * TS;
        for (int e = lane; e < TS; e += 32) buf[e] = zt[e];
        __syncwarp();
        int rowOf[NS];
        double uM[NS], v[NS], S;
        ok &= hungarian_f64<NS>(buf, N, n, N, j, nl, rowOf, uM, v, S, steps, relax);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int c = lane + 32 * s;
            if (c < N && c != j && c != nl && rowOf[s] >= 0 && rowOf[s] < n) uRow[rowOf[s]] = uM[s];
        }
        __syncwarp();
        for (int r = 0; r < n; ++r) {
            const double ur = uRow[r];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int c = lane + 32 * s;
                if (c < N && c != j && c != nl) zt[r * N + c] = (buf[r * N + c] - ur) - v[s];
            }
        }
        if (lane == 0) d.y[t] = 0.0 + S;  // c was spread to D (cleared), then += S
        ++laps;
        __syncwarp();
    }
    if (lane == 0) {
        if (!ok) atomicOr(&d.status->err, kDevInternal);
        if (laps) {
            atomicAdd(&d.status->laps, (unsigned long long)laps);
            atomicAdd(&d.status->steps, (unsigned long long)steps);
            atomicAdd(&d.status->relax, (unsigned long long)relax);
            atomicAdd(&d.status->dlaps, (unsigned long long)laps);
            atomicAdd(&d.status->dsteps, (unsigned long long)steps);
            atomicAdd(&d.status->drelax, (unsigned long long)relax);
        }
    }
}

// transfer between complementary costs of C: T = c_ijkn + c_knij (i < k), both T/2
__global__ void f64_complementary_C_kernel(F64Dev d)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < d.tiles;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k, n;
        decode_tile(d, t, i, j, k, n);
        if (i >= k) continue;
        const long long t2 = ((long long)(k * d.N + n) * d.m + i) * d.m + (j - (j > n));
        const double T = d.y[t] + d.y[t2];
        d.y[t] = T / 2.0;
        d.y[t2] = T / 2.0;
    }
}

// One warp per LAP of count problems of size n (matrix p at M + p * n * n,
// row-major), in shared memory; S[p] = the LAP value; optional residual
// written back in place, row potentials, column potentials, assignment, work.
// Used by the concentrations C -> B (add = x: b_ij += S) and B -> LB, and by
// rlt2_f64_lap_batch.
template <int NS>
__global__ void __launch_bounds__(kF64Warps * 32)
f64_lap_kernel(double *M, int n, long long count, double *Sout, double *addTo, int32_t *assign, double *uOut,
               double *vOut, int64_t *work, bool residual, DevStatus *status, bool dsum)
{
    extern __shared__ double f64_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nn = n * n;
    double *buf = f64_smem + (size_t)warp * (nn + n);
    double *uRow = buf + nn;
    unsigned steps = 0, relax = 0, laps = 0;
    bool ok = true;
    const long long nw = (long long)gridDim.x * kF64Warps;
    for (long long p = blockIdx.x * (long long)kF64Warps + warp; p < count; p += nw) {
        double *Mp = M + (size_t)p * nn;
        for (int e = lane; e < nn; e += 32) buf[e] = Mp[e];
        __syncwarp();
        int rowOf[NS];
        double uM[NS], v[NS], S;
        unsigned st0 = steps, rl0 = relax;
        ok &= hungarian_f64<NS>(buf, n, n, n, -1, -1, rowOf, uM, v, S, steps, relax);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int c = lane + 32 * s;
            if (c < n && rowOf[s] >= 0 && rowOf[s] < n) {
                uRow[rowOf[s]] = uM[s];
                if (assign) assign[(size_t)p * n + rowOf[s]] = c;
                if (vOut) vOut[(size_t)p * n + c] = v[s];
            }
        }
        __syncwarp();
        if (uOut)
            for (int r = lane; r < n; r += 32) uOut[(size_t)p * n + r] = uRow[r];
        if (residual)
            for (int r = 0; r < n; ++r) {
                const double ur = uRow[r];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int c = lane + 32 * s;
                    if (c < n) Mp[r * n + c] = (buf[r * n + c] - ur) - v[s];
                }
            }
        if (lane == 0) {
            if (Sout) Sout[p] = S;
            if (addTo) addTo[p] = addTo[p] + S;
            if (work) {
                work[2 * p] = (int64_t)(steps - st0);
                work[2 * p + 1] = (int64_t)(relax - rl0);
            }
        }
        ++laps;
        __syncwarp();
    }
    if (lane == 0 && status) {
        if (!ok) atomicOr(&status->err, kDevInternal);
        if (laps && dsum) {
            atomicAdd(&status->laps, (unsigned long long)laps);
            atomicAdd(&status->steps, (unsigned long long)steps);
            atomicAdd(&status->relax, (unsigned long long)relax);
        }
    }
}

// LB <- LB + S, the history entry of the pass, pass count
__global__ void f64_lb_kernel(F64Dev d, const double *S)
{
    const double lb = d.LB[0] + S[0];
    d.LB[0] = lb;
    const int it = d.iter[0];
    if (it < d.hist_cap) d.hist[it] = lb;
    d.iter[0] = it + 1;
}

int grid_for(long long items, int per_cta)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (items + per_cta - 1) / per_cta;
    const long long cap = (long long)sms * 16;
    return (int)(need < 1 ? 1 : need < cap ? need : cap);
}

size_t lap_smem(int n) { return (size_t)kF64Warps * ((size_t)n * n + n) * sizeof(double); }

cudaError_t launch_f64_lap(double *M, int n, long long count, double *Sout, double *addTo, int32_t *assign,
                           double *uOut, double *vOut, int64_t *work, bool residual, DevStatus *status,
                           bool dsum, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const size_t sm = lap_smem(n);
    const int grid = grid_for(count, kF64Warps);
    if (n <= 32) {
        cudaError_t e = cudaFuncSetAttribute(f64_lap_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        f64_lap_kernel<1><<<grid, kF64Warps * 32, sm, s>>>(M, n, count, Sout, addTo, assign, uOut, vOut, work,
                                                           residual, status, dsum);
    } else {
        cudaError_t e = cudaFuncSetAttribute(f64_lap_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        f64_lap_kernel<2><<<grid, kF64Warps * 32, sm, s>>>(M, n, count, Sout, addTo, assign, uOut, vOut, work,
                                                           residual, status, dsum);
    }
    return cudaGetLastError();
}

cudaError_t launch_f64_dlap(const F64Dev &d, cudaStream_t s)
{
    const size_t sm = (size_t)kF64Warps * (d.TS + d.n) * sizeof(double);
    const int grid = grid_for(d.tiles, kF64Warps);
    if (d.N <= 32) {
        cudaError_t e = cudaFuncSetAttribute(f64_dlap_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        f64_dlap_kernel<1><<<grid, kF64Warps * 32, sm, s>>>(d);
    } else {
        cudaError_t e = cudaFuncSetAttribute(f64_dlap_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        f64_dlap_kernel<2><<<grid, kF64Warps * 32, sm, s>>>(d);
    }
    return cudaGetLastError();
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return RLT2_OK;
    if (e == cudaErrorMemoryAllocation) return RLT2_E_OOM;
    return RLT2_E_CUDA;
}

#define CKF(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_rc(e_); \
    } while (0)

}  // namespace
}  // namespace rlt2

using namespace rlt2;

struct rlt2_f64_ctx {
    F64Dev d{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int rlt1_only = 0, profile = 0, enqueued = 0;
    double *Sx = nullptr;        // the B -> LB LAP value of the pass
    int32_t *Fd = nullptr, *Dd = nullptr;
    int4 *tri = nullptr;
    cudaEvent_t ev[5] = {};
    double stage_ms[4] = {0, 0, 0, 0};
    int profiled = 0;
};

static void f64_free(rlt2_f64_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->d.x);
    cudaFree(c->d.y);
    cudaFree(c->d.z);
    cudaFree(c->d.LB);
    cudaFree(c->Fd);
    cudaFree(c->Dd);
    cudaFree(c->tri);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// one pass of Algorithm 1 in the FP64 form
static int f64_pass(rlt2_f64_ctx *c)
{
    const F64Dev &d = c->d;
    cudaStream_t s = c->stream;
    const int ew = grid_for(d.tiles, kF64Threads);
    auto mark = [&](int k) -> cudaError_t { return c->profile ? cudaEventRecord(c->ev[k], s) : cudaSuccess; };
    CKF(mark(0));
    f64_spread_x_kernel<<<ew, kF64Threads, 0, s>>>(d);
    CKF(cudaGetLastError());
    CKF(cudaMemsetAsync(d.x, 0, (size_t)d.N * d.N * sizeof(double), s));
    if (!c->rlt1_only) {
        const size_t sm = 4 * (size_t)d.N * d.N * sizeof(double);
        CKF(cudaFuncSetAttribute(f64_p1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        f64_share_kernel<<<ew, kF64Threads, 0, s>>>(d);
        CKF(cudaGetLastError());
        f64_p1_kernel<<<(unsigned)(d.classes / ((long long)(d.N - 1) * (d.N - 2))), kF64Threads, sm, s>>>(d);
        CKF(cudaGetLastError());
        CKF(mark(1));
        CKF(launch_f64_dlap(d, s));
    } else {
        CKF(mark(1));
    }
    CKF(mark(2));
    f64_complementary_C_kernel<<<ew, kF64Threads, 0, s>>>(d);
    CKF(cudaGetLastError());
    CKF(launch_f64_lap(d.y, d.m, (long long)d.N * d.N, nullptr, d.x, nullptr, nullptr, nullptr, nullptr, true,
                       d.status, true, s));
    CKF(mark(3));
    CKF(launch_f64_lap(d.x, d.N, 1, c->Sx, nullptr, nullptr, nullptr, nullptr, nullptr, true, d.status, true, s));
    f64_lb_kernel<<<1, 1, 0, s>>>(d, c->Sx);
    CKF(cudaGetLastError());
    CKF(mark(4));
    if (c->profile) {
        CKF(cudaEventSynchronize(c->ev[4]));
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            // stage 0: spreads and complementary D; 1: D->C; 2: complementary C + C->B; 3: B->LB
            CKF(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
            c->stage_ms[k] += ms;
        }
        c->profiled++;
    }
    return RLT2_OK;
}

extern "C" {

int rlt2_f64_create(const int32_t *F, const int32_t *D, int N, const double *B_lin, double lb_const,
                    const rlt2_opts *opts, rlt2_f64_ctx **out)
{
    if (!out) return RLT2_E_INVAL;
    *out = nullptr;
    if (!F || !D || N < RLT2_MIN_N || N > RLT2_MAX_N) return RLT2_E_INVAL;
    for (int e = 0; e < N * N; e++)
        if (F[e] < 0 || D[e] < 0 || (B_lin && !(B_lin[e] >= 0.0 && std::isfinite(B_lin[e])))) return RLT2_E_INVAL;
    if (!std::isfinite(lb_const)) return RLT2_E_INVAL;
    rlt2_opts o;
    rlt2_default_opts(&o);
    if (opts) o = *opts;
    if (o.max_iters < 1) return RLT2_E_INVAL;
    rlt2_f64_ctx *c = new (std::nothrow) rlt2_f64_ctx;
    if (!c) return RLT2_E_OOM;
    F64Dev &d = c->d;
    d.N = N;
    d.n = N - 2;
    d.m = N - 1;
    d.TS = d.n * N;
    d.tiles = (long long)N * N * d.m * d.m;
    const long long ntri = (long long)N * (N - 1) * (N - 2) / 6;
    d.classes = ntri * N * (N - 1) * (N - 2);
    d.hist_cap = o.max_iters;
    c->rlt1_only = o.rlt1_only;
    c->profile = o.profile;
    auto fail = [&](int rc) {
        f64_free(c);
        return rc;
    };
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RLT2_E_CUDA);
        c->own_stream = true;
    }
    // small scalars in one allocation: LB, Sx, iter, status, history
    const size_t small = 64 + sizeof(DevStatus) + 64 + (size_t)d.hist_cap * sizeof(double);
    cudaError_t e = cudaMalloc((void **)&d.LB, small);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.x, (size_t)N * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.y, (size_t)d.tiles * sizeof(double));
    if (e == cudaSuccess && !c->rlt1_only) e = cudaMalloc((void **)&d.z, (size_t)d.tiles * d.TS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->Fd, (size_t)N * N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->Dd, (size_t)N * N * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->tri, (size_t)(ntri > 0 ? ntri : 1) * sizeof(int4));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(cuda_rc(e));
    }
    char *base = reinterpret_cast<char *>(d.LB);
    c->Sx = reinterpret_cast<double *>(base + 8);
    d.iter = reinterpret_cast<int *>(base + 16);
    d.status = reinterpret_cast<DevStatus *>(base + 64);
    d.hist = reinterpret_cast<double *>(base + 64 + sizeof(DevStatus) + 64);
    d.F = c->Fd;
    d.D = c->Dd;
    d.triples = c->tri;
    std::vector<int4> tri;
    for (int a = 0; a < N; a++)
        for (int b = a + 1; b < N; b++)
            for (int cc = b + 1; cc < N; cc++) tri.push_back(make_int4(a, b, cc, 0));
    std::vector<double> x0((size_t)N * N, 0.0);
    if (B_lin) std::memcpy(x0.data(), B_lin, x0.size() * sizeof(double));
    cudaStream_t s = c->stream;
    e = cudaMemsetAsync(d.LB, 0, small, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.LB, &lb_const, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->Fd, F, (size_t)N * N * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->Dd, D, (size_t)N * N * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !tri.empty())
        e = cudaMemcpyAsync(c->tri, tri.data(), tri.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.x, x0.data(), x0.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d.z) e = cudaMemsetAsync(d.z, 0, (size_t)d.tiles * d.TS * sizeof(double), s);
    if (e == cudaSuccess) {
        f64_init_kernel<<<grid_for(d.tiles, kF64Threads), kF64Threads, 0, s>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && c->profile)
        for (auto &ev : c->ev)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffers go out of scope
    if (e != cudaSuccess) return fail(cuda_rc(e));
    *out = c;
    return RLT2_OK;
}

void rlt2_f64_destroy(rlt2_f64_ctx *ctx) { f64_free(ctx); }

int rlt2_f64_iterate(rlt2_f64_ctx *c, int k)
{
    if (!c || k < 0) return RLT2_E_INVAL;
    if ((long long)c->enqueued + k > c->d.hist_cap) return RLT2_E_STATE;
    for (int p = 0; p < k; ++p) {
        const int rc = f64_pass(c);
        if (rc != RLT2_OK) return rc;
        c->enqueued++;
    }
    return RLT2_OK;
}

static int f64_status(rlt2_f64_ctx *c)
{
    int err = 0;
    CKF(cudaMemcpyAsync(&err, &c->d.status->err, 4, cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaStreamSynchronize(c->stream));
    return (err & kDevInternal) ? RLT2_E_INTERNAL : RLT2_OK;
}

int rlt2_f64_bound(rlt2_f64_ctx *c, double *lb, int *iters)
{
    if (!c) return RLT2_E_INVAL;
    double v = 0;
    int it = 0;
    CKF(cudaMemcpyAsync(&v, c->d.LB, 8, cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaMemcpyAsync(&it, c->d.iter, 4, cudaMemcpyDeviceToHost, c->stream));
    const int rc = f64_status(c);
    if (rc != RLT2_OK) return rc;
    if (lb) *lb = v;
    if (iters) *iters = it;
    return RLT2_OK;
}

int rlt2_f64_bound_history(rlt2_f64_ctx *c, double *out, int cap, int *count)
{
    if (!c || cap < 0 || (cap > 0 && !out)) return RLT2_E_INVAL;
    int it = 0;
    CKF(cudaMemcpyAsync(&it, c->d.iter, 4, cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaStreamSynchronize(c->stream));
    const int nrec = it < c->d.hist_cap ? it : c->d.hist_cap;
    const int ncopy = nrec < cap ? nrec : cap;
    if (ncopy > 0) CKF(cudaMemcpyAsync(out, c->d.hist, (size_t)ncopy * 8, cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaStreamSynchronize(c->stream));
    if (count) *count = ncopy;
    return f64_status(c);
}

int rlt2_f64_get_state(rlt2_f64_ctx *c, int level, double *host, size_t count)
{
    if (!c || !host) return RLT2_E_INVAL;
    const F64Dev &d = c->d;
    const int N = d.N, n = d.n;
    if (level == 0) {
        if (count != (size_t)N * N) return RLT2_E_INVAL;
        CKF(cudaMemcpyAsync(host, d.x, count * 8, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 1) {
        if (count != (size_t)d.tiles) return RLT2_E_INVAL;
        CKF(cudaMemcpyAsync(host, d.y, count * 8, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 2) {
        if (!d.z || count != (size_t)d.tiles * n * n) return RLT2_E_INVAL;
        std::vector<double> tmp;
        try {
            tmp.resize((size_t)d.tiles * d.TS);
        } catch (...) {
            return RLT2_E_OOM;
        }
        CKF(cudaMemcpyAsync(tmp.data(), d.z, tmp.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CKF(cudaStreamSynchronize(c->stream));
        const int m = d.m;
        size_t o = 0;
        for (long long t = 0; t < d.tiles; t++) {
            const int nn = (int)(t % m), j = (int)((t / ((long long)m * m)) % N);
            const int nl = nn + (nn >= j);
            const double *src = tmp.data() + (size_t)t * d.TS;
            for (int r = 0; r < n; r++)
                for (int q = 0; q < N; q++)
                    if (q != j && q != nl) host[o++] = src[r * N + q];
        }
    } else {
        return RLT2_E_INVAL;
    }
    CKF(cudaStreamSynchronize(c->stream));
    return f64_status(c);
}

void *rlt2_f64_device_state(rlt2_f64_ctx *c, int which)
{
    if (!c) return nullptr;
    return which == 0 ? (void *)c->d.x : which == 1 ? (void *)c->d.y : which == 2 ? (void *)c->d.z : nullptr;
}

int rlt2_f64_work(rlt2_f64_ctx *c, int64_t out[6])
{
    if (!c || !out) return RLT2_E_INVAL;
    DevStatus st;
    CKF(cudaMemcpyAsync(&st, c->d.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    CKF(cudaStreamSynchronize(c->stream));
    out[0] = (int64_t)st.laps;
    out[1] = (int64_t)st.steps;
    out[2] = (int64_t)st.relax;
    out[3] = (int64_t)st.dlaps;
    out[4] = (int64_t)st.dsteps;
    out[5] = (int64_t)st.drelax;
    return RLT2_OK;
}

int rlt2_f64_stage_times(rlt2_f64_ctx *c, double out[4], int *passes)
{
    if (!c || !out) return RLT2_E_INVAL;
    CKF(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 4; ++k) out[k] = c->stage_ms[k];
    if (passes) *passes = c->profiled;
    return RLT2_OK;
}

int rlt2_f64_lap_batch(const double *M, int n, int count, double *S, int32_t *assign, double *u, double *v,
                       int64_t *work, void *stream)
{
    if (n < 1 || n > 64 || count < 0 || (count > 0 && (!M || !S))) return RLT2_E_INVAL;
    if (count == 0) return RLT2_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus *st = nullptr;
    CKF(cudaMallocAsync((void **)&st, sizeof(DevStatus), s));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    // residual = false: the kernel only reads M
    if (e == cudaSuccess)
        e = launch_f64_lap(const_cast<double *>(M), n, count, S, nullptr, assign, u, v, work, false, st, false, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_rc(e);
    return (err & kDevInternal) ? RLT2_E_INTERNAL : RLT2_OK;
}

}  // extern "C"
