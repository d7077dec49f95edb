// sweep_kernels.cu -- initialisation and the fused pass over D (sm_103a).
//
// p1_kernel performs the first three operations of the loop of Algorithm 1 in
// one read and one write of D:
//   spread B -> C   (Sec. 4.2): c'_ijkn = c_ijkn + the share of b_ij of row k,
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
#include "device.cuh"
#include "kernels.h"

namespace rlt2 {

constexpr int kP1Threads = 512;

__device__ __forceinline__ int tidx_n(int N, int a, int b, int c, int d)
{
    const int m = N - 1;
    return ((a * N + b) * m + (c - (c > a))) * m + (d - (d > b));
}

// t-th of m shares of x (reading of Sec. 4.2 in integers)
__device__ __forceinline__ int share(int x, int m, int t)
{
    const int q = x / m;
    return q + (t < x - q * m ? 1 : 0);
}

// r-th element of [0, N) without a and b (a != b)
__device__ __forceinline__ int skip2(int r, int a, int b)
{
    const int lo = min(a, b), hi = max(a, b);
    r += (r >= lo);
    r += (r >= hi);
    return r;
}

struct P1Layout {
    int n, m, n2, JCp, P4;
    int A1, A3, A2, A5, A4, A6, H1, H2, H3, H5, H4, H6, total;
};

__host__ __device__ inline P1Layout p1_layout(int N, int JC)
{
    P1Layout L;
    L.n = N - 2;
    L.m = N - 1;
    L.n2 = L.n | 1;
    L.JCp = JC | 1;
    L.P4 = L.m * L.JCp;
    if (!(L.P4 & 1)) L.P4 += 1;
    int o = 0;
    L.A1 = o; o += JC * L.m * L.n;
    L.A3 = o; o += JC * L.m * L.n;
    L.A2 = o; o += JC * L.m * L.n2;
    L.A5 = o; o += JC * L.m * L.n2;
    L.A4 = o; o += N * L.P4;
    L.A6 = o; o += N * L.P4;
    L.H1 = o; o += JC * L.m;
    L.H2 = o; o += JC * L.m;
    L.H3 = o; o += JC * L.m;
    L.H5 = o; o += JC * L.m;
    L.H4 = o; o += N * L.m;
    L.H6 = o; o += N * L.m;
    L.total = o;
    return L;
}

size_t p1_smem_bytes(int N, int JC) { return (size_t)p1_layout(N, JC).total * 4; }

int p1_chunk(int N)
{
    for (int jc : {4, 2}) if (p1_smem_bytes(N, jc) <= 110 * 1024) return jc;
    return 1;
}

template <int JC>
__global__ void __launch_bounds__(kP1Threads)
    p1_kernel(PassState p, int N, int RS, const int4 *__restrict__ triples, int nchunks)
{
    if (*p.stop) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.counter = 0;  // work counter of the D -> C sweep
    extern __shared__ __align__(16) int sm[];
    const P1Layout L = p1_layout(N, JC);
    const int n = L.n, m = L.m;
    const int TS = n * RS;
    const int4 tr = triples[blockIdx.x / nchunks];
    const int i = tr.x, k = tr.y, pp = tr.z;
    const int j0 = (blockIdx.x % nchunks) * JC;
    const int jc = min(JC, N - j0);
    const int *__restrict__ yC = p.yC;
    const int *__restrict__ xb = p.x;
    int *__restrict__ z = p.z;
    const int RV = RS >> 2;  // int4 per tile row

    // ---- shares of the staged rows (c' of the tile, spread over its rows)
    // kinds 1,3,2,5: jc*m rows each
    for (int e = threadIdx.x; e < 4 * jc * m; e += blockDim.x) {
        const int kind = e / (jc * m), rr = e % (jc * m);
        const int jj = rr / m, o = rr % m, j = j0 + jj;
        const int l = o + (o >= j);  // n (kinds 1,3) or q (kinds 2,5)
        int t, b, bk, row, h;
        if (kind == 0) {         // kind 1: tile (i,j,k,l) row p
            t = tidx_n(N, i, j, k, l); b = xb[i * N + j]; bk = k - 1; row = pp - 2; h = L.H1;
        } else if (kind == 1) {  // kind 3: tile (k,l,i,j) row p
            t = tidx_n(N, k, l, i, j); b = xb[k * N + l]; bk = i; row = pp - 2; h = L.H3;
        } else if (kind == 2) {  // kind 2: tile (i,j,p,l) row k
            t = tidx_n(N, i, j, pp, l); b = xb[i * N + j]; bk = pp - 1; row = k - 1; h = L.H2;
        } else {                 // kind 5: tile (p,l,i,j) row k
            t = tidx_n(N, pp, l, i, j); b = xb[pp * N + l]; bk = i; row = k - 1; h = L.H5;
        }
        const int c1 = yC[t] + share(b, m, bk);
        sm[h + rr] = share(c1, n, row);
    }
    // kinds 4,6: N*m rows each
    for (int e = threadIdx.x; e < 2 * N * m; e += blockDim.x) {
        const int kind = e / (N * m), rr = e % (N * m);
        const int a = rr / m, o = rr % m;
        const int l = o + (o >= a);
        int t, c1;
        if (kind == 0) {  // kind 4: tile (k,a,p,l) row i
            t = tidx_n(N, k, a, pp, l);
            c1 = yC[t] + share(xb[k * N + a], m, pp - 1);
            sm[L.H4 + rr] = share(c1, n, i);
        } else {          // kind 6: tile (p,a,k,l) row i
            t = tidx_n(N, pp, a, k, l);
            c1 = yC[t] + share(xb[pp * N + a], m, k);
            sm[L.H6 + rr] = share(c1, n, i);
        }
    }

    // ---- stage the tile rows
    for (int e = threadIdx.x; e < 4 * jc * m * RV; e += blockDim.x) {
        const int kind = e / (jc * m * RV), rem = e % (jc * m * RV);
        const int rr = rem / RV, part = rem % RV;
        const int jj = rr / m, o = rr % m, j = j0 + jj;
        const int l = o + (o >= j);
        int t, row, base, ld;
        if (kind == 0) { t = tidx_n(N, i, j, k, l); row = pp - 2; base = L.A1; ld = n; }
        else if (kind == 1) { t = tidx_n(N, k, l, i, j); row = pp - 2; base = L.A3; ld = n; }
        else if (kind == 2) { t = tidx_n(N, i, j, pp, l); row = k - 1; base = L.A2; ld = L.n2; }
        else { t = tidx_n(N, pp, l, i, j); row = k - 1; base = L.A5; ld = L.n2; }
        const int4 w = *reinterpret_cast<const int4 *>(z + (size_t)t * TS + row * RS + 4 * part);
        int *dst = sm + base + rr * ld + 4 * part;
        const int c = 4 * part;
        if (c + 0 < n) dst[0] = w.x;
        if (c + 1 < n) dst[1] = w.y;
        if (c + 2 < n) dst[2] = w.z;
        if (c + 3 < n) dst[3] = w.w;
    }
    for (int e = threadIdx.x; e < 2 * N * m * jc; e += blockDim.x) {
        const int kind = e / (N * m * jc), rem = e % (N * m * jc);
        const int a = rem / (m * jc), o = (rem / jc) % m, jj = rem % jc, j = j0 + jj;
        const int l = o + (o >= a);
        if (j == a || j == l) continue;
        const int col = j - (j > a) - (j > l);
        int t, base;
        if (kind == 0) { t = tidx_n(N, k, a, pp, l); base = L.A4; }
        else { t = tidx_n(N, pp, a, k, l); base = L.A6; }
        sm[base + a * L.P4 + o * L.JCp + jj] = z[(size_t)t * TS + i * RS + col];
    }
    __syncthreads();

    // ---- split every class {(i,j),(k,nn),(p,qq)}, j in the chunk
    for (int e = threadIdx.x; e < jc * m * n; e += blockDim.x) {
        const int jj = e / (m * n), o = (e / n) % m, s = e % n;
        const int j = j0 + jj;
        const int nn = o + (o >= j);
        const int qq = skip2(s, j, nn);
        const int q1 = qq - (qq > j);
        const int s2 = nn - (nn > j) - (nn > qq);
        const int q4 = qq - (qq > nn);
        const int n6 = nn - (nn > qq);
        int *a1 = sm + L.A1 + (jj * m + o) * n + s;
        int *a3 = sm + L.A3 + (jj * m + o) * n + s;
        int *a2 = sm + L.A2 + (jj * m + q1) * L.n2 + s2;
        int *a5 = sm + L.A5 + (jj * m + q1) * L.n2 + s2;
        int *a4 = sm + L.A4 + nn * L.P4 + q4 * L.JCp + jj;
        int *a6 = sm + L.A6 + qq * L.P4 + n6 * L.JCp + jj;
        const int T = *a1 + sm[L.H1 + jj * m + o] + *a2 + sm[L.H2 + jj * m + q1] +
                      *a3 + sm[L.H3 + jj * m + o] + *a4 + sm[L.H4 + nn * m + q4] +
                      *a5 + sm[L.H5 + jj * m + q1] + *a6 + sm[L.H6 + qq * m + n6];
        const int q6 = T / 6, rm = T - 6 * q6;
        *a1 = q6 + (0 < rm);
        *a2 = q6 + (1 < rm);
        *a3 = q6 + (2 < rm);
        *a4 = q6 + (3 < rm);
        *a5 = q6 + (4 < rm);
        *a6 = q6 + (5 < rm);
    }
    __syncthreads();

    // ---- write back
    for (int e = threadIdx.x; e < 4 * jc * m * RV; e += blockDim.x) {
        const int kind = e / (jc * m * RV), rem = e % (jc * m * RV);
        const int rr = rem / RV, part = rem % RV;
        const int jj = rr / m, o = rr % m, j = j0 + jj;
        const int l = o + (o >= j);
        int t, row, base, ld;
        if (kind == 0) { t = tidx_n(N, i, j, k, l); row = pp - 2; base = L.A1; ld = n; }
        else if (kind == 1) { t = tidx_n(N, k, l, i, j); row = pp - 2; base = L.A3; ld = n; }
        else if (kind == 2) { t = tidx_n(N, i, j, pp, l); row = k - 1; base = L.A2; ld = L.n2; }
        else { t = tidx_n(N, pp, l, i, j); row = k - 1; base = L.A5; ld = L.n2; }
        const int *src = sm + base + rr * ld + 4 * part;
        const int c = 4 * part;
        int4 w;
        w.x = c + 0 < n ? src[0] : 0;
        w.y = c + 1 < n ? src[1] : 0;
        w.z = c + 2 < n ? src[2] : 0;
        w.w = c + 3 < n ? src[3] : 0;
        *reinterpret_cast<int4 *>(z + (size_t)t * TS + row * RS + c) = w;
    }
    for (int e = threadIdx.x; e < 2 * N * m * jc; e += blockDim.x) {
        const int kind = e / (N * m * jc), rem = e % (N * m * jc);
        const int a = rem / (m * jc), o = (rem / jc) % m, jj = rem % jc, j = j0 + jj;
        const int l = o + (o >= a);
        if (j == a || j == l) continue;
        const int col = j - (j > a) - (j > l);
        int t, base;
        if (kind == 0) { t = tidx_n(N, k, a, pp, l); base = L.A4; }
        else { t = tidx_n(N, pp, a, k, l); base = L.A6; }
        z[(size_t)t * TS + i * RS + col] = sm[base + a * L.P4 + o * L.JCp + jj];
    }
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
    k<<<ntriples * nchunks, kP1Threads, smem, s>>>(p, g.N, g.RS, triples, nchunks);
    return cudaGetLastError();
}

cudaError_t launch_p1(const Geom &g, const PassState &p, const int4 *triples, int ntriples,
                      cudaStream_t s)
{
    switch (p1_chunk(g.N)) {
    case 4: return p1_go<4>(g, p, triples, ntriples, s);
    case 2: return p1_go<2>(g, p, triples, ntriples, s);
    default: return p1_go<1>(g, p, triples, ntriples, s);
    }
}

}  // namespace rlt2
