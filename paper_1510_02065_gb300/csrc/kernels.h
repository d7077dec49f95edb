// kernels.h -- internal interface between the C ABI and the device kernels.
//
// Every stage kernel advances a *group* of RLT2 instances at once: a table of
// per-instance descriptors, each work item (CTA, warp or thread) finding its
// instance by binary search over prefix counts.  A single dual ascent is a
// group of one; a batch of branch-and-bound nodes of different residual sizes
// is a larger group advanced by the same launches.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace rlt2 {

// Geometry of the tile store of D.  Tile t = ((i*N + j)*(N-1) + k')*(N-1) + n'
// holds the submatrix D_ijkn: its N-2 rows are the facilities p not in {i,k}
// (ascending) and its columns are indexed by the location q itself, W =
// round_up(N, 4) of them; columns j and n (and q >= N) carry no coefficient.
// Every row starts on a 16-byte boundary and any 4 consecutive locations
// 4c..4c+3 form one aligned 16-byte piece of a row.
struct Geom {
    int N;
    int n;            // N - 2: rows (and coefficients per row) of a tile
    int W;            // row width in ints, round_up(N, 4)
    int TS;           // tile stride, ints (n * W)
    int U0;           // class-sum store: offset of v in a tile's duals, round_up(n, 4)
    int DS;           // class-sum store: ints of duals per tile, U0 + W
    long long tiles;  // N^2 (N-1)^2
    long long classes_ints;  // class-sum store: C(N,3) N^3 ints
    long long htiles;        // pair store: the tiles with i < k, N (N-1)/2 * N (N-1)
};

inline Geom make_geom(int N)
{
    Geom g;
    g.N = N;
    g.n = N - 2;
    g.W = (N + 3) & ~3;
    g.TS = g.n * g.W;
    g.U0 = (g.n + 3) & ~3;
    g.DS = g.U0 + g.W;
    g.tiles = (long long)N * N * (N - 1) * (N - 1);
    g.classes_ints = (long long)N * (N - 1) * (N - 2) / 6 * N * N * N;
    g.htiles = g.tiles / 2;
    return g;
}

// Class-sum store of D (the alternative to the tile store): the six members
// of a class {(x,lx),(y,ly),(z,lz)}, facilities x < y < z, hold after the
// transfer between complementary costs floor(T/6) + [rank < T mod 6] of its
// sum T (rank = lexicographic rank of the member, Eq. (11)), so one int per
// class, T[tri_index(x,y,z) N^3 + lx N^2 + ly N + lz], and the duals (u, v) of
// each tile's last LAP determine every reduced cost of D: d = member - u_r - v_q.
__host__ __device__ inline long long tri_index(int x, int y, int z)
{
    return (long long)z * (z - 1) * (z - 2) / 6 + y * (y - 1) / 2 + x;
}

// Row of tile (i,j,k,n) held by facility e (e not in {i,k}) in the class-sum
// store: the member at column (location) f is T[base + f * stride]; rank is
// the lexicographic rank of the member ordering (i, k, e) of its class.
struct SymRow {
    long long base;
    int stride, rank;
};

__host__ __device__ inline SymRow sym_row(int N, int i, int j, int k, int n, int e)
{
    const int a = i < k ? i : k, c = i < k ? k : i, la = i < k ? j : n, lc = i < k ? n : j;
    const long long N2 = (long long)N * N, N3 = N2 * N;
    SymRow s;
    if (e < a) {
        s.base = tri_index(e, a, c) * N3 + (long long)la * N + lc;
        s.stride = (int)N2;
    } else if (e < c) {
        s.base = tri_index(a, e, c) * N3 + (long long)la * N2 + lc;
        s.stride = N;
    } else {
        s.base = tri_index(a, c, e) * N3 + (long long)la * N2 + (long long)lc * N;
        s.stride = 1;
    }
    // positions of i, k, e among the sorted three; orderings of (x, y, z) in
    // lexicographic order have ranks 2 * (position of the first) + [second > third]
    const int pi = (i > k) + (i > e), pk = (k > i) + (k > e), pe = (e > i) + (e > k);
    s.rank = 2 * pi + (pk > pe ? 1 : 0);
    return s;
}

// Member of rank `rank` of a class with sum T >= 0 (Eq. (11), equal split).
__host__ __device__ inline int sym_member(int T, int rank)
{
    const int q = (int)((unsigned)T / 6u);
    return q + (rank < T - 6 * q ? 1 : 0);
}

// Pair store (the complementary submatrices of Sec. 6 kept as one): the tile
// D_ijkn with i < k holds the sum of D_ijkn and D_knij; its index is
// th = (pair(i,k) N + j)(N-1) + n' with n' = n - (n > j) and pair(i,k) = C(k,2) + i.
__host__ __device__ inline int pair_index(int i, int k) { return k * (k - 1) / 2 + i; }

__host__ __device__ inline void pair_of(int idx, int &i, int &k)
{
    k = 1;
    while ((k + 1) * k / 2 <= idx) ++k;  // k <= 63: at most 63 steps
    i = idx - k * (k - 1) / 2;
}

// Device state of one instance.
struct PassState {
    int *z;            // tile store of D (null without D or with the class-sum store)
    int *T;            // class-sum store (null unless it is used)
    int *du;           // per tile: u of its N-2 rows (padded to U0), then v of its W location columns
    int *yS;           // per tile: c' before D->C, then S of the tile's LAP
    int *yC;           // reduced C after concentration C->B
    int *x;            // reduced B
    long long *LB;     // bound
    long long *hist;   // LB after each pass
    int *iter;         // passes completed
    int *stop;         // stopping rule fired
    int hist_cap;
    double ub, min_progress;
};

// One instance as the kernels see it.
struct NodeDesc {
    // The tile store as a 5-D tensor of ints: (column q, row, n', k', i*N + j),
    // box (4, 1, m|1, 1, N): the location-chunk pieces of one facility row
    // across all tiles of a fixed facility pair, as the fused pass over D
    // moves them (valid when zmap_ok; m = N - 1, the box overhang m|1 > m only
    // pads the shared-memory pitch and is out of bounds, zero-filled on load
    // and skipped on store).
    CUtensorMap zmap;     // class-sum store: the same box over the v part of the tile duals
    int zmap_ok;
    int paired;           // D in the pair store (z holds the tiles with i < k)
    PassState p;
    int N, W, TS;
    int U0, DS;           // class-sum store: dual offsets (Geom)
    int nchunks;          // location chunks of the fused pass over D
    long long tiles;      // tiles of C (all (i,j,k,n))
    long long tile_base;  // first group-wide tile index of this instance
    long long dtiles;     // D->C work units: tiles, or the pair store's htiles
    long long dtile_base; // first group-wide D->C unit of this instance
    int cta_base;         // first fused-pass CTA of this instance
    int prob_base;        // first C->B problem of this instance
    FastDiv fN, fm, fmm, fn;
};

inline void fill_node(NodeDesc &d, int N, int JC)
{
    const Geom g = make_geom(N);
    d.N = N;
    d.W = g.W;
    d.TS = g.TS;
    d.U0 = g.U0;
    d.DS = g.DS;
    d.tiles = g.tiles;
    d.dtiles = d.paired ? g.htiles : g.tiles;  // d.paired is set by the caller first
    d.nchunks = (N + JC - 1) / JC;
    d.fN = make_fastdiv(N);
    d.fm = make_fastdiv(N - 1);
    d.fmm = make_fastdiv((N - 1) * (N - 1));
    d.fn = make_fastdiv(N - 2);
}

// How the D->C concentration solves a range of tiles: `lanes` lanes per tile
// (32: a warp per tile, in CTAs of `warps` = 4, 16 or 32 warps, 0 for the
// size that keeps the most warps resident; 16: two tiles per warp, one per
// half-warp, for rows of at most 16 columns in the tile and class-sum
// stores).  Every shape gives identical results.
struct DlapShape {
    int lanes, warps;
};

// A group of instances advanced together.
struct Group {
    const NodeDesc *nodes;  // device array [B]
    int B;
    long long tiles;        // total tiles
    int ctas;               // total fused-pass CTAs
    int probs;              // total C->B problems
    int maxN, maxTS;        // largest instance
    int JC;                 // locations per fused-pass CTA (one value for the group)
    bool pack;              // every instance's keys fit the packed reduction
    bool rlt1_only;
    bool sym;               // D in the class-sum store (every instance of the group)
    bool paired;            // D in the pair store (every instance of the group)
    long long dtiles;       // total D->C work units
    int small_tiles;        // D->C: the first small_tiles units (instances with N <= 16, which
                            // come first in the group) form a range of their own
    int smallTS, smallW;    // largest tile stride (ints) and row width among those instances
    DlapShape dshape[2];    // D->C shape of the other units [0] and of the small ones [1]
    unsigned *counter;      // D->C work counters: [0] the other units, [1] the small ones
    DevStatus *status;      // error bits and work counters of the group
    DevStatus *snap;        // [3] copies of *status taken inside a tuning pass
    const int4 *triples;    // facility triples i<k<p ordered by p: the first C(N,3) serve N
    NodeDesc first;         // copy of nodes[0]: kernels of a group of one read it as a parameter
};

int p1_chunk(int N, bool sym, bool paired);  // locations per CTA of the fused pass over D
// Encode nd.zmap for the fused pass with location chunk JC (sets zmap_ok;
// false leaves the pieces to per-piece copies).  nd.p.z (or du), nd.paired
// and the geometry must be set.
bool encode_zmap(NodeDesc &nd, int JC);
size_t p1_smem_bytes(int N, int JC, bool sym, bool paired);  // its dynamic shared memory

// Initialise instance `node` of the group (index b) from device copies of its
// F, D and linear costs (Blin may be null).
cudaError_t launch_init(const NodeDesc &node, const int32_t *F, const int32_t *D,
                        const int32_t *Blin, long long lb_const, cudaStream_t s);
cudaError_t launch_spread_x(const Group &g, cudaStream_t s);
// State of the warm-started child ch (N - 1) of instance par fixing facility f
// to location l (tile or pair store): B, C, D and LB derived on the device.
cudaError_t launch_child(const NodeDesc &par, const NodeDesc &ch, int f, int l, cudaStream_t s);
// Reduced costs of D of a class-sum-store instance in the tile-store layout
// (tiles x (N-2) x W ints at out; columns without coefficient 0).
cudaError_t launch_materialize(const NodeDesc &nd, int *out, cudaStream_t s);
cudaError_t launch_p1(const Group &g, cudaStream_t s);
// A second stream and fork/join events: with them, the half-warp D->C kernel
// of a group that has both small and larger instances runs beside the
// whole-warp one (in eager launches and in captured graphs alike).
struct SideStream {
    cudaStream_t s2;
    cudaEvent_t fork, join;
};
cudaError_t launch_dlap(const Group &g, int sm_count, cudaStream_t s, const SideStream *side = nullptr);
// One range [lo, hi) of the group's D->C units, taken from *counter (reset to
// 0 by the fused pass), tiles of at most tsp ints and maxW columns.
struct DlapRange {
    long long lo, hi;
    unsigned *counter;
    int tsp, maxW, maxN, lanes, warps;
};
// One of the group's two D->C ranges (0: the units from small_tiles on, 1:
// the small instances' units) in its shape g.dshape[which].
cudaError_t launch_dlap_range(const Group &g, int which, int sm_count, cudaStream_t s);
// Warps per CTA that range `which` launches with (0 if it is empty).
int dlap_cta_warps(const Group &g, int which);
// Whether a shape can solve rows of width W (paired: the pair store).
inline bool dlap_shape_fits(const DlapShape &d, int W, bool paired)
{
    if (d.lanes == 16) return W <= 16 && !paired && d.warps == 0;
    return d.lanes == 32 && (d.warps == 0 || d.warps == 4 || d.warps == 16 || d.warps == 32);
}
cudaError_t launch_clap(const Group &g, cudaStream_t s);
cudaError_t launch_xlap(const Group &g, cudaStream_t s);
cudaError_t launch_lap_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                             int32_t *u, int32_t *v, int64_t *work, DevStatus *status,
                             cudaStream_t s);

// Failure-detection self-test: a bounded wait on an mbarrier nothing completes.
cudaError_t launch_wait_selftest(DevStatus *status, unsigned limit, cudaStream_t s);

// The auction method on caller matrices (comparison with the Hungarian method).
cudaError_t launch_auction_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                                 int64_t *work, DevStatus *status, cudaStream_t s);

// Index of the instance owning group-wide item x; base(node) is its first item.
template <typename F>
__device__ __forceinline__ int find_node(const NodeDesc *nodes, int B, long long x, F base)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(nodes[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace rlt2
