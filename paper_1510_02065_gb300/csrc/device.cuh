// device.cuh -- device-side building blocks of the RLT2 library (sm_103a).
//
//  * bounded mbarrier waits and 1-D bulk copies global -> shared (the TMA
//    engine's cp.async.bulk), used to stage LAP tiles;
//  * warp_hungarian<NS, PACK>: the Hungarian method of the cost concentration
//    (Sec. 4.1), one warp per linear assignment problem.
#pragma once
#include <climits>
#include <cstdint>

namespace rlt2 {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kInf = INT_MAX;

// bits of the device status word
constexpr int kDevTimeout = 1;
constexpr int kDevRange = 2;
constexpr int kDevInternal = 4;   // an invariant of the Hungarian method failed

// Iteration bound of every spin on an mbarrier.  try_wait suspends the thread
// for a while on each call, so the bound is far above any real wait.
constexpr unsigned kSpinLimit = 1u << 22;

struct DevStatus {
    int err;                     // kDev* bits
    int pad;
    unsigned long long laps;     // LAPs solved
    unsigned long long steps;    // columns labelled (all concentrations)
    unsigned long long relax;    // reduced distances evaluated
    unsigned long long dlaps;    // LAPs of the D->C concentrations
    unsigned long long dsteps;   // their steps
    unsigned long long drelax;   // their relaxations
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on bar expecting `bytes` of asynchronous transactions, then start a
// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, unsigned bytes,
                                          uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Arrive on bar (count 1 of its expected arrivals) announcing `bytes` of
// asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy (no arrive) of `bytes` global -> shared, completing on bar.
__device__ __forceinline__ void bulk_load_tx(void *dst_smem, const void *src_gmem, unsigned bytes,
                                             uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Tiled 5-D tensor copy global -> shared through tensor map `map` (generic
// address of a map in parameter, constant or global space), box origin
// c0..c4 (c0 x 4 bytes a multiple of 16), completing its bytes on bar.
__device__ __forceinline__ void tensor_load5(void *dst_smem, const void *map, int c0, int c1, int c2,
                                             int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst_smem)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}

// Tiled 5-D tensor copy shared -> global (bulk-group completion); elements
// outside the tensor are not written.
__device__ __forceinline__ void tensor_store5(const void *map, int c0, int c1, int c2, int c3, int c4,
                                              const void *src_smem)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
            map),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(src_smem))
        : "memory");
}

// Order this thread's later tensor copies after the (host-written) map in global memory.
__device__ __forceinline__ void tensormap_acquire(const void *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// 4-byte asynchronous copy global -> shared (cp.async), and its completion.
__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src_gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Exact unsigned division of x < 2^31 by a runtime divisor d >= 1:
// q = (umulhi(x, mul) + x) >> shift with shift = ceil(log2 d) and
// mul = ceil(2^(32+shift) / d) - 2^32 (0 when d is a power of two).
struct FastDiv {
    unsigned mul, shift, d;
};

inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    unsigned l = 0;
    while ((1ull << l) < d) l++;
    f.shift = l;
    f.mul = ((1ull << l) == d) ? 0u
                               : (unsigned)((1ull << (32 + l)) / d + 1 - (1ull << 32));
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv &f)
{
    return (__umulhi(x, f.mul) + x) >> f.shift;
}

// Wait for the phase of parity `parity` of bar to complete; false after
// kSpinLimit unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit = kSpinLimit)
{
    const uint32_t a = smem_addr(bar);
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ------------------------------------------------------------ register slots
// A column c of a LAP lives in lane c % 32, slot c / 32 (NS slots per lane).
// Slot selection by a warp-uniform runtime index without local memory.

template <int NS, typename T>
__device__ __forceinline__ T pick(const T (&a)[NS], int s)
{
    if constexpr (NS == 1) return a[0];
    else return s ? a[1] : a[0];
}

template <int NS, typename T>
__device__ __forceinline__ void put(T (&a)[NS], int s, T x)
{
    if constexpr (NS == 1) a[0] = x;
    else {
        if (s) a[1] = x;
        else a[0] = x;
    }
}

__device__ __forceinline__ long long warp_sum64(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Lane segments: SEG = 32 (a warp per LAP) or 16 (two LAPs per warp, one per
// half).  sl = lane within the segment, mask = the segment's lanes.
template <int SEG>
struct Seg {
    int sl, base;
    unsigned mask;
    __device__ __forceinline__ Seg()
    {
        const int lane = threadIdx.x & 31;
        sl = SEG == 32 ? lane : (lane & (SEG - 1));
        base = lane - sl;
        mask = SEG == 32 ? kFull : (((1u << SEG) - 1u) << base);
    }
};

template <int SEG>
__device__ __forceinline__ long long seg_sum64(long long x, unsigned mask)
{
#pragma unroll
    for (int o = SEG / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

// ------------------------------------------------------- Hungarian method
//
// Shortest-augmenting-path Hungarian method with row and column potentials,
// rows inserted in ascending order from u = v = 0; the next column labelled is
// the unlabelled one of least reduced distance, ties to the smallest column;
// a distance label and its predecessor change only on a strict improvement.
//
// Warp mapping: lane c % 32, slot c / 32 owns column c: its potential v, the
// row matched to it (rowOf) and that row's potential (uM), its distance label
// and predecessor column (way).  Each step relaxes the newly reached row
// against every column at once and takes the argmin with one warp reduction.
//
// Potentials are updated lazily.  Within the insertion of one row, let D be
// the running sum of the step minima.  A column labelled when the sum was
// dlab ends the phase with v -= Dend - dlab and its row with u += Dend - dlab;
// unlabelled columns keep v; the new row gets u = Dend.  Distance labels are
// stored plus the D of their last update, so the per-step update of every
// label disappears.  In exact integer arithmetic this takes the same decisions
// and ends with the same (u, v, assignment) as updating every potential at
// every step.
//
// PACK: when every key is below 2^25 the key and its column are packed into
// one 32-bit value (key * 64 + column) and one reduction yields both the
// minimum and the smallest column attaining it.
//
// Value range: with entries in [0, A], |u|, |v| <= A and every key <= 3A, so
// A <= 2^29 - 1 fits int32 (PACK needs 3A < 2^25).
//
// steps_out / relax_out accumulate the LAP's work (32-bit: a caller sums at
// most one launch's LAPs of one warp, far below 2^32 for n <= 64).
//
// SEG = 16 runs the same method on a half-warp (width <= 16, NS = 1): each
// half of a warp solves its own LAP, every warp-wide primitive restricted to
// the half's lanes; the halves may diverge and reconverge freely.
//
// M: shared memory, row r at M + r * ld (rows 0..n-1).  The n columns are the
// indices c < width other than dead0 and dead1 (width <= 32 * NS); a column's
// lane and slot follow its index, so ties still go to the smallest column.
//
// Every loop is bounded for any input, valid or not: a phase ends at the
// latest when every column is labelled, and an augmenting path is at most as
// long as the phase.  If an invariant fails (it cannot for entries in range)
// the function stops and returns false instead of spinning.
//
// SENT: with packed keys (PACK) on a whole warp, see warp_hungarian_lane
// below (dead0 must be a column < width).  Otherwise (width <= 32 NS - 1) the
// last column slot, lane 31 of slot NS - 1,
// holds no column and serves as a sentinel: never matched (its row stays -1),
// its key above every key a column can have (PACK: the largest distance a
// packed key allows; keys of real columns are below it or tie with a smaller
// column) yet below a labelled column's.  A phase in which every real column
// got labelled then also ends on a free column -- the sentinel -- so a step
// tests only for a free column, and reaching the sentinel reports the
// invariant failure.
//
// A whole warp with packed keys and a sentinel (SEG = 32, PACK, SENT) goes to
// warp_hungarian_lane: the same method in a representation that takes fewer
// instructions per step, with the LAP's dead column dead0 as its sentinel.
//
// warp_hungarian_lane: lane c % 32, slot c / 32 owns column c.  Each column
// keeps two words, both modulo 2^32:
//   ruM = 64 uM + rowOf + 1   (its matched row and that row's potential)
//   wv  = c - 64 v            (its potential)
// A relaxation forms the packed key 64 x + wv - q = 64 (x - v - c0) + c
// directly (q = 64 c0), which is, modulo 2^32, the value the general form
// gets by shifting the candidate, so every comparison and every result is the
// same.  The winning column's lane hands over the next row and offset in one
// word, z = ruM - key + c = 64 (uM - Dk) + rowOf + 1: its low six bits are the
// row + 1 (0: a free column, the augmenting path's end), the rest is q.
// Labelling sets the key's top bit and keeps its value (64 Dk + c) for the
// lazy update, which moves ruM and wv by 64 (Dend - Dk); augmenting moves one
// word per column.  (rowOf + 1 < 64: n <= 62.)
//
// The sentinel is column sent, one outside the LAP (dead0, or a slot c >=
// width, c < 32 NS): its key is the largest distance a packed key allows (real
// keys stay at least one below it) and it is never matched, so a phase in
// which every real column got labelled ends on it and reports the invariant
// failure.
// Columns outside the LAP are never relaxed and keep the key 0x7fffffff,
// above the sentinel's.
//
// Bounded on any data: a labelled key is negative as a signed value and a
// relaxation only replaces a key by a smaller one, so it stays labelled (on
// data in range no relaxation reaches it: a labelled column's candidate is its
// reduced cost plus its label, >= 0); every step that does not end the phase
// labels the least unlabelled key, so after at most one step per column the
// sentinel is the least key and ends the phase.
template <int NS>
__device__ __forceinline__ bool warp_hungarian_lane(const int *__restrict__ M, int ld, int n, int width,
                                                    int dead0, int dead1, int sent, int (&rowOf)[NS],
                                                    int (&uM)[NS], int (&v)[NS], unsigned &steps_out,
                                                    unsigned &relax_out)
{
    constexpr unsigned kLab = 0x80000000u;   // set on the key of a labelled column
    constexpr unsigned kNone = 0x7fffffffu;  // key of a column outside the LAP
    constexpr unsigned kSentBase = ((1u << 25) - 1u) << 6;
    const int lane = threadIdx.x & 31;
    bool valid[NS];
    unsigned key0[NS], key[NS], ruM[NS], wv[NS];
    int way[NS];  // packed key of the column through which the column was reached (-1: the new row)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int c = lane + 32 * s;
        valid[s] = c < width && c != dead0 && c != dead1;
        key0[s] = c == sent ? kSentBase | (unsigned)c : kNone;
        ruM[s] = 0u;
        wv[s] = (unsigned)c;
        way[s] = -1;
    }
    int sumK = 0, sumK2 = 0;
    const int off = lane - ld;  // row i at M + (i + 1) * ld + off

    for (int r = 0; r < n; ++r) {
#pragma unroll
        for (int s = 0; s < NS; ++s) key[s] = key0[s];
        unsigned r1 = (unsigned)r + 1u, q = 0u, mm;
        int j0 = -1;
        for (;;) {
            const int *row = M + ((int)r1 * ld + off);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (valid[s]) {
                    const unsigned ck = (unsigned)row[32 * s] * 64u + (wv[s] - q);
                    if ((int)ck < (int)key[s]) {
                        key[s] = ck;
                        way[s] = j0;
                    }
                }
            }
            unsigned lmin, z;
            if constexpr (NS == 1) {
                lmin = key[0];
                z = ruM[0] - key[0] + (unsigned)lane;
            } else {
                const bool hi = key[1] < key[0];
                lmin = hi ? key[1] : key[0];
                z = (hi ? ruM[1] : ruM[0]) - lmin + (unsigned)(hi ? lane + 32 : lane);
            }
            mm = __reduce_min_sync(kFull, lmin);
            const unsigned zw = __shfl_sync(kFull, z, (int)mm);  // from the lane of column mm % 64
            r1 = zw & 63u;
            if (r1 == 0u) break;  // free column (or the sentinel): augmenting path found
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (key[s] == mm) key[s] |= kLab;
            q = zw & ~63u;
            j0 = (int)mm;
        }
        const int jf = (int)(mm & 63u);
        if (jf == sent) return false;  // the sentinel: every column labelled, cannot happen
        const unsigned Dend6 = mm & ~63u;

        // lazy potential updates of the columns labelled in this phase
        int K = 1;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const bool lab = (int)key[s] < 0;
            K += __popc(__ballot_sync(kFull, lab));
            if (lab) {
                const unsigned dd = Dend6 - (key[s] & (kLab - 64u));
                wv[s] += dd;
                ruM[s] += dd;
            }
        }
        sumK += K;
        sumK2 += K * K;

        // augment: each column on the path takes the row (and its potential)
        // of its predecessor, the first one the new row with u = Dend (a
        // shuffle from lane -1 reads lane 31, whose word a predecessor -1 ignores)
        const unsigned root = Dend6 + (unsigned)r + 1u;
        int c = jf;
        for (int hop = 0;; ++hop) {
            if (hop > K) return false;
            const int w = __shfl_sync(kFull, pick<NS>(way, NS == 1 ? 0 : c >> 5), c);
            const unsigned p = __shfl_sync(kFull, pick<NS>(ruM, NS == 1 ? 0 : (w >> 5) & 1), w);
            if (NS == 1 ? lane == c : lane == (c & 31)) put<NS>(ruM, NS == 1 ? 0 : c >> 5, w >= 0 ? p : root);
            if (w < 0) break;
            c = w & 63;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        rowOf[s] = (int)(ruM[s] & 63u) - 1;
        uM[s] = (int)(ruM[s] & ~63u) >> 6;
        v[s] = (int)((unsigned)(lane + 32 * s) - wv[s]) >> 6;
    }
    steps_out += (unsigned)sumK;
    relax_out += (unsigned)(n * sumK - (sumK2 - sumK) / 2);
    return true;
}

template <int NS, bool PACK, int SEG = 32, bool SENT = false>
__device__ __forceinline__ bool warp_hungarian(const int *__restrict__ M, int ld, int n, int width,
                                               int dead0, int dead1, int (&rowOf)[NS],
                                               int (&uM)[NS], int (&v)[NS],
                                               unsigned &steps_out, unsigned &relax_out)
{
    static_assert(SEG == 32 || (SEG == 16 && NS == 1), "a half-warp LAP has one column per lane");
    static_assert(!SENT || SEG == 32, "the sentinel is lane 31 of a whole warp");
    if constexpr (SEG == 32 && PACK && SENT)
        return warp_hungarian_lane<NS>(M, ld, n, width, dead0, dead1, dead0, rowOf, uM, v, steps_out,
                                       relax_out);
    // A labelled column's key is kDone = INT_MIN: as a signed value no
    // candidate is below it, so no relaxation touches it (whatever the data),
    // and as an unsigned value it is above every unlabelled key, so no
    // reduction picks it while an unlabelled column remains.  Each step
    // therefore labels a new column or ends the phase: at most n + 1 steps.
    // A column outside the LAP has key kNone (never relaxed, never picked
    // before kDone, told apart from a labelled column).
    constexpr unsigned kDone = 0x80000000u;  // key of a labelled column
    constexpr unsigned kNone = 0xffffffffu;  // key of a column outside the LAP
    constexpr int kSentCol = 32 * NS - 1;
    constexpr unsigned kSentKey = PACK ? ((((1u << 25) - 1u) << 6) | (unsigned)kSentCol) : 0x7fffffffu;
    const Seg<SEG> g;
    const int lane = g.sl;  // the lane's place in its segment
    bool valid[NS];
    int way[NS], dlab[NS];
    unsigned key[NS], key0[NS];  // key0: the key a column starts every row with
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int c = lane + 32 * s;
        valid[s] = c < width && c != dead0 && c != dead1;
        key0[s] = valid[s] ? 0x7fffffffu : (SENT && c == kSentCol) ? kSentKey : kNone;
        rowOf[s] = -1;
        uM[s] = 0;
        v[s] = 0;
        way[s] = -1;
        dlab[s] = 0;
    }
    int sumK = 0, sumK2 = 0;

    for (int r = 0; r < n; ++r) {
        // key = distance label (+ D of its last update), packed with the column
        // when PACK
#pragma unroll
        for (int s = 0; s < NS; ++s) key[s] = key0[s];
        int i0 = r;   // row scanned at this step
        int j0 = -1;  // column through which i0 was reached (-1: the new row)
        int c0 = 0;   // u(i0) - D before this step
        unsigned mm;
        int Dk, j1;
        for (;;) {
            const int *Mrow = M + i0 * ld + lane;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (valid[s]) {
                    const int cand = Mrow[32 * s] - v[s] - c0;
                    const unsigned ck = PACK ? ((unsigned)cand << 6) | (unsigned)(lane + 32 * s)
                                             : (unsigned)cand;
                    if ((int)ck < (int)key[s]) {
                        key[s] = ck;
                        way[s] = j0;
                    }
                }
            }
            unsigned lmin = key[0];
            if constexpr (NS == 2) lmin = min(lmin, key[1]);
            mm = __reduce_min_sync(g.mask, lmin);
            if constexpr (PACK) {
                Dk = (int)(mm >> 6);
                j1 = (int)(mm & 63u);
            } else {
                Dk = (int)mm;
                const unsigned b0 = __ballot_sync(g.mask, key[0] == mm) >> g.base;
                if constexpr (NS == 1) {
                    j1 = __ffs(b0) - 1;
                } else {
                    const unsigned b1 = __ballot_sync(g.mask, key[1] == mm);
                    j1 = b0 ? __ffs(b0) - 1 : 31 + __ffs(b1);
                }
            }
            // one slot per lane on a whole warp: j1 < 32 is the lane itself
            constexpr bool kOne = NS == 1 && SEG == 32;
            const int src = kOne ? j1 : j1 & 31, sl = kOne ? 0 : j1 >> 5;
            const int rj = __shfl_sync(g.mask, pick<NS>(rowOf, sl), g.base + src);
            const int uj = __shfl_sync(g.mask, pick<NS>(uM, sl), g.base + src);
            if constexpr (SENT) {
                if (rj < 0) break;  // free column (or the sentinel): augmenting path found
            } else {
                if (rj < 0 || mm == kDone) break;  // free column: augmenting path found
            }
            if (lane == src) {
                put<NS>(key, sl, kDone);
                put<NS>(dlab, sl, Dk);
            }
            i0 = rj;
            j0 = j1;
            c0 = uj - Dk;
        }
        if (SENT ? j1 == kSentCol : mm == kDone) return false;  // every column labelled: cannot happen
        const int jf = j1, Dend = Dk;

        // lazy potential updates of the columns labelled in this phase
        int K = 1;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const bool lab = key[s] == kDone;
            K += __popc(__ballot_sync(g.mask, lab));
            if (lab) {
                const int dd = Dend - dlab[s];
                v[s] -= dd;
                uM[s] += dd;
            }
        }
        sumK += K;
        sumK2 += K * K;

        // augment: each column on the path takes the row of its predecessor
        // (one slot per lane on a whole warp: columns are lanes, and a shuffle
        // from lane -1 reads lane 31, whose values a predecessor -1 ignores)
        constexpr bool kOne = NS == 1 && SEG == 32;
        int c = jf;
        for (int hop = 0;; ++hop) {
            if (hop > K) return false;
            const int cs = kOne ? 0 : c >> 5, cl = kOne ? c : c & 31;
            const int w = __shfl_sync(g.mask, pick<NS>(way, cs), g.base + cl);
            int nr = r, nu = Dend;
            const int ws = kOne ? 0 : (w < 0 ? 0 : w) >> 5, wl = kOne ? w : (w < 0 ? 0 : w) & 31;
            const int pr = __shfl_sync(g.mask, pick<NS>(rowOf, ws), g.base + wl);
            const int pu = __shfl_sync(g.mask, pick<NS>(uM, ws), g.base + wl);
            if (w >= 0) {
                nr = pr;
                nu = pu;
            }
            if (lane == cl) {
                put<NS>(rowOf, cs, nr);
                put<NS>(uM, cs, nu);
            }
            if (w < 0) break;
            c = w;
        }
    }
    steps_out += (unsigned)sumK;
    relax_out += (unsigned)(n * sumK - (sumK2 - sumK) / 2);
    return true;
}

// A full n x n LAP (no dead columns, width n): the lane words when keys pack
// and a column slot is free for the sentinel (n < 32 NS), else the general form.
template <int NS, bool PACK>
__device__ __forceinline__ bool warp_hungarian_full(const int *__restrict__ M, int ld, int n, int (&rowOf)[NS],
                                                    int (&uM)[NS], int (&v)[NS], unsigned &steps_out,
                                                    unsigned &relax_out)
{
    if constexpr (PACK) {
        if (n < 32 * NS)
            return warp_hungarian_lane<NS>(M, ld, n, n, -1, -1, 32 * NS - 1, rowOf, uM, v, steps_out, relax_out);
    }
    return warp_hungarian<NS, PACK>(M, ld, n, n, -1, -1, rowOf, uM, v, steps_out, relax_out);
}

// S = sum of the row and column potentials = cost of the assignment.
template <int NS, int SEG = 32>
__device__ __forceinline__ long long lap_value(int width, int dead0, int dead1, const int (&uM)[NS],
                                               const int (&v)[NS])
{
    const Seg<SEG> g;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int c = g.sl + 32 * k;
        if (c < width && c != dead0 && c != dead1) s += (long long)uM[k] + v[k];
    }
    return seg_sum64<SEG>(s, g.mask);
}

// Row potentials by row index into shared uRow[n] (and the column of each row
// into colOf[n] when non-null); the caller syncs the warp afterwards.
template <int NS, int SEG = 32>
__device__ __forceinline__ void scatter_rows(int n, int width, int dead0, int dead1,
                                             const int (&rowOf)[NS], const int (&uM)[NS],
                                             int *uRow, int *colOf, int ustride = 1)
{
    const Seg<SEG> g;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int c = g.sl + 32 * k;
        if (c < width && c != dead0 && c != dead1 && rowOf[k] >= 0 && rowOf[k] < n) {
            uRow[rowOf[k] * ustride] = uM[k];
            if (colOf) colOf[rowOf[k]] = c;
        }
    }
}

}  // namespace rlt2
