// auction.cu -- the auction method for the linear assignment problem on
// sm_103a, the LAP method the paper runs on its GPU (Sec. 6), for comparison
// with the Hungarian method of the dual ascent.
//
// One warp per LAP (min-cost, integer costs >= 0), lane c % 32 slot c / 32
// holding object (column) c's price and owner.  Gauss-Seidel bidding: the
// lowest-indexed unassigned person bids for its best object j1 (least cost +
// price, ties to the smallest column) and raises its price by the gap to the
// second best plus eps; the object's previous owner becomes unassigned.
// eps-scaling: costs are multiplied by K = n + 1 and eps falls by a factor 4
// per phase down to 1; with eps = 1 < K / n the final assignment is optimal
// (eps-complementary slackness for integer costs), so S equals the optimum
// the Hungarian method finds.  Prices and costs are 64-bit.  Every phase is
// bounded: past 64 n^2 + 64 bids it records an internal error and stops.
#include "device.cuh"
#include "kernels.h"

namespace rlt2 {

constexpr int kAucWarps = 4;

__device__ __forceinline__ long long warp_min64(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
}

template <int NS>
__global__ void __launch_bounds__(kAucWarps * 32)
    auction_kernel(const int32_t *__restrict__ M, int n, int count, int64_t *S, int32_t *assign,
                   int64_t *work, DevStatus *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *a = reinterpret_cast<int *>(smem) + (size_t)warp * (n * n + 64);
    int *objOf = a + n * n;  // person -> object (-1: unassigned)
    constexpr long long kBig = 0x3fffffffffffffffLL;
    for (int prob = blockIdx.x * kAucWarps + warp; prob < count; prob += gridDim.x * kAucWarps) {
        const int32_t *src = M + (size_t)prob * n * n;
        int mx = 0, bad = 0;
        for (int e = lane; e < n * n; e += 32) {
            const int x = src[e];
            a[e] = x;
            mx = max(mx, x);
            bad |= (x < 0) | (x > 536870911);
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
        const long long K = n + 1;
        long long price[NS];
        int own[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) price[s] = 0;
        long long eps = (long long)mx * K / 4;
        if (eps < 1) eps = 1;
        long long bids = 0;
        bool fine = true;
        for (;;) {  // one eps phase
#pragma unroll
            for (int s = 0; s < NS; ++s) own[s] = -1;
            for (int e = lane; e < n; e += 32) objOf[e] = -1;
            __syncwarp();
            long long phaseBids = 0;
            const long long limit = 64LL * n * n + 64;
            for (;;) {
                // lowest-indexed unassigned person
                unsigned b0 = __ballot_sync(kFull, lane < n && objOf[lane] < 0);
                unsigned b1 = NS == 2 ? __ballot_sync(kFull, lane + 32 < n && objOf[lane + 32] < 0) : 0u;
                if (!b0 && !b1) break;
                const int i = b0 ? __ffs(b0) - 1 : 31 + __ffs(b1);
                if (++phaseBids > limit) {
                    fine = false;
                    break;
                }
                // best and second best object: key = (cost K + price) << 7 | column
                long long k1 = kBig, k2 = kBig;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int c = lane + 32 * s;
                    if (c < n) {
                        const long long key = (((long long)a[i * n + c] * K + price[s]) << 7) | c;
                        if (key < k1) {
                            k2 = k1;
                            k1 = key;
                        } else if (key < k2) {
                            k2 = key;
                        }
                    }
                }
                const long long best = warp_min64(k1);
                // second best: the least key other than best over all lanes
                const long long mine = k1 == best ? k2 : k1;
                const long long second = warp_min64(mine);
                const int j1 = (int)(best & 127);
                const long long w1 = best >> 7;
                const long long w2 = second >= kBig ? w1 : (second >> 7);
                const long long raise = w2 - w1 + eps;
                const int ls = j1 & 31, ss = j1 >> 5;
                const int prev = __shfl_sync(kFull, pick<NS>(own, ss), ls);
                if (lane == ls) {
                    put<NS>(price, ss, pick<NS>(price, ss) + raise);
                    put<NS>(own, ss, i);
                }
                if (lane == 0) {
                    objOf[i] = j1;
                    if (prev >= 0) objOf[prev] = -1;
                }
                __syncwarp();
            }
            bids += phaseBids;
            if (!fine || eps == 1) break;
            eps = eps / 4 > 1 ? eps / 4 : 1;
        }
        if (!fine && lane == 0) atomicOr(&status->err, kDevInternal);
        long long s = 0;
        for (int e = lane; e < n; e += 32) {
            const int j = objOf[e];
            s += j >= 0 ? a[e * n + j] : 0;
            if (assign) assign[(size_t)prob * n + e] = j;
        }
        s = warp_sum64(s);
        if (lane == 0) {
            S[prob] = fine ? s : -1;
            if (work) work[prob] = bids;
        }
        __syncwarp();
    }
}

cudaError_t launch_auction_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                                 int64_t *work, DevStatus *status, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const size_t smem = (size_t)kAucWarps * ((size_t)n * n + 64) * 4;
    int grid = (count + kAucWarps - 1) / kAucWarps;
    if (grid > 65535) grid = 65535;
    cudaError_t e;
    if (n <= 32) {
        if ((e = cudaFuncSetAttribute(auction_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        auction_kernel<1><<<grid, kAucWarps * 32, smem, s>>>(M, n, count, S, assign, work, status);
    } else {
        if ((e = cudaFuncSetAttribute(auction_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        auction_kernel<2><<<grid, kAucWarps * 32, smem, s>>>(M, n, count, S, assign, work, status);
    }
    return cudaGetLastError();
}

}  // namespace rlt2
