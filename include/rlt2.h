/*
 * rlt2.h -- C ABI of the GB300 (sm_103a) level-2 RLT dual-ascent library.
 *
 * The library computes the RLT2 dual-ascent lower bound of the Koopmans-
 * Beckmann quadratic assignment problem (QAP), Algorithm 1 of Goncalves,
 * Pessoa, Drummond, Bentes, Farias, "Solving the Quadratic Assignment Problem
 * on heterogeneous environment (CPUs and GPUs) with the application of Level 2
 * Reformulation and Linearization Technique" (arXiv:1510.02065).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns RLT2_OK (0) or a negative RLT2_E_* code;
 *    rlt2_strerror() names it.  No function aborts the process.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory on the current device.  Inputs are copied or only read;
 *    the caller keeps ownership of every buffer it passes.  A context owns
 *    all the device memory it allocates and frees it in rlt2_destroy().
 *  - Indices are 0-based.  Matrices are row-major int32.
 *  - A context is not thread-safe; distinct contexts are independent and
 *    may run on distinct streams concurrently.
 *  - Arithmetic is exact: reduced costs, potentials and LAP values are
 *    integers (int32 on the device, guarded against overflow at creation);
 *    the bound LB is carried in int64 and also reported as a double.  The
 *    rlt2_f64_* calls at the end are the FP64 form (the paper's real
 *    division), in doubles.
 *
 * Notation (Sec. 3, Eq. (5)): x_ij / b_ij is the assignment variable and its
 * reduced cost (matrix B, N x N); x'_ijkn / c_ijkn the pair variable and its
 * reduced cost (matrix C); x''_ijknpq / d_ijknpq the triple variable and its
 * reduced cost (matrix D).  The exported layouts are compact:
 *   x: b[i][j]                          N*N entries
 *   y: c[i][j][k'][n']                  N*N*(N-1)*(N-1) entries, k' = rank of k
 *                                       among the facilities != i, n' = rank of n
 *                                       among the locations != j
 *   z: d[i][j][k'][n'][r][s]            y's count * (N-2)*(N-2) entries, r = rank
 *                                       of p among the facilities not in {i,k},
 *                                       s = rank of q among the locations not in {j,n}
 * A "tile" is the (N-2) x (N-2) submatrix D_ijkn of Sec. 4.1; tile index
 * t = ((i*N + j)*(N-1) + k')*(N-1) + n'.
 */
#ifndef RLT2_H
#define RLT2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RLT2_OK            0
#define RLT2_E_INVAL      -1   /* bad argument: null pointer, N out of range, negative entry */
#define RLT2_E_OOM        -2   /* device or host allocation failed                            */
#define RLT2_E_OVERFLOW   -3   /* costs too large for exact int32 arithmetic (see rlt2_create) */
#define RLT2_E_CUDA       -4   /* a CUDA runtime call failed                                  */
#define RLT2_E_TIMEOUT    -5   /* a bounded device-side wait gave up                          */
#define RLT2_E_STATE      -6   /* call out of order (e.g. history capacity exhausted)         */
#define RLT2_E_INTERNAL   -7   /* a kernel's internal consistency check failed (a bug)        */
#define RLT2_E_IO         -8   /* checkpoint file not writable / readable, or not a checkpoint */

#define RLT2_MIN_N         3
#define RLT2_MAX_N        64   /* the LAP kernels hold at most 64 columns per warp */
#define RLT2_LAP_MAX_ENTRY 536870911  /* 2^29 - 1: largest LAP cost the int32 kernels accept */

/* Options of a dual-ascent context.  Zero-initialise, or call rlt2_default_opts. */
typedef struct {
    int rlt1_only;        /* 1: Algorithm 1 without the three operations on D
                             (the strong-branching dual of Sec. 6); default 0 */
    int use_graph;        /* 1 (default): each pass is one captured CUDA graph   */
    int profile;          /* 1: launch every stage of every pass directly on the
                             stream with CUDA events between the stages (no
                             graph; see rlt2_stage_times); default 0          */
    int max_iters;        /* capacity of the on-device LB history; default 65536 */
    double ub;            /* UB of Algorithm 1 (stop once LB >= UB); <= 0: none  */
    double min_progress;  /* K of Algorithm 1: stop once LB'/UB < K; 0: never     */
    void *stream;         /* cudaStream_t to run on; NULL = a non-blocking stream
                             created for (and owned by) the context              */
    int store;            /* how D is kept: RLT2_STORE_TILES (default),
                             RLT2_STORE_CLASSES (identical results) or
                             RLT2_STORE_PAIRS (the paired dual ascent)          */
    int lanes;            /* lanes per D->C LAP (Sec. 4.1's concentration of D):
                             32 (a warp per tile) or 16 (two tiles per warp, one
                             per half-warp; needs N <= 16, tile or class-sum
                             store); 0 (default): chosen (see "Autotuning"
                             below).  Results are identical in every shape    */
    int cta_warps;        /* warps per CTA of the whole-warp D->C kernel: 4, 16
                             or 32 (it must fit the CTA's shared memory: 32 warps
                             up to N = 43, 16 up to N = 60); 0 (default): chosen */
} rlt2_opts;

/*
 * Autotuning of the D->C shape (opts.lanes = opts.cta_warps = 0).  The first
 * passes of a context or batch are tuning passes: one unmeasured pass
 * in the default shape (whole warps in the CTA size that keeps the most warps
 * resident), then one pass per candidate -- the default, half-warps where the
 * rows have at most 16 columns, whole warps in CTAs of 4, 16 and 32 warps
 * where they fit (up to six passes in all) -- each timed by CUDA events and
 * measured by the Hungarian's step counter.  A candidate replaces the default
 * only if its time per step is at least 3% lower (a pass's time per step
 * drifts by a percent or two from one pass to the next).  In a group or
 * batch that holds instances with N <= 16 and larger ones, the two kinds form
 * separate D->C ranges, each with its own shape (a batch tunes each; after
 * tuning the small one runs on a second stream beside the other).  Tuning
 * passes are ordinary passes (every shape gives the same results), launched
 * directly rather than from a graph, and each synchronises the stream.  The
 * choice is remembered for the process per device, store and row width: later
 * contexts, groups and batches with the same key start with it and do not
 * tune.  A group (rlt2_group_create) takes the remembered shape of its key,
 * else the default, and never tunes (a server rebuilds its group whenever its
 * membership changes, often sooner than tuning would end).
 */

/*
 * Stores of D.  RLT2_STORE_TILES keeps every reduced cost d_ijknpq in the tile
 * layout of rlt2_device_state (about 4 B N^2 (N-1)^2 (N-2)^2; 2.7 GB at N =
 * 30, 6.7 GB at N = 35).  RLT2_STORE_CLASSES keeps one int per class
 * {(i,j),(k,n),(p,q)} -- the class sum T after the transfer between
 * complementary costs, whose six members are floor(T/6) + [rank < T mod 6]
 * (Eq. (11)) -- plus the duals (u, v) of every tile's last LAP, from which
 * every reduced cost follows as member - u_p - v_q (about 4 B C(N,3) N^3 +
 * 4 B N^2 (N-1)^2 (2N); 0.6 GB at N = 30, 1.5 GB at N = 35, 52 GB at N = 64).
 */
#define RLT2_STORE_TILES   0
#define RLT2_STORE_CLASSES 1
/*
 * RLT2_STORE_PAIRS: the complementary submatrices of Sec. 6.  Each
 * coefficient (d_ijkn)_pq has the complementary coefficient (d_knij)_pq (the
 * same variable), so the pair is kept as one sum in D_ijkn with i < k: half
 * of D and half of the D->C LAPs per pass.  This is a different dual ascent:
 * spreading C->D adds the shares of c_knij to D_ijkn, the transfer between
 * complementary costs of D splits a class sum equally over its three members
 * d_ijknpq, d_ijpqkn, d_knpqij (i < k < p), and D->C concentrates D_ijkn
 * (i < k) into c_ijkn.  Its bounds differ from the other two stores' (same
 * for both of those); the oracle has the same form.  Exported D (level 2):
 * the pair sums in the tiles with i < k, the others 0.
 */
#define RLT2_STORE_PAIRS   2

typedef struct rlt2_ctx rlt2_ctx;

void rlt2_default_opts(rlt2_opts *opts);
const char *rlt2_strerror(int code);

/*
 * Create a dual-ascent context for one QAP instance and initialise it as
 * Algorithm 1 does: LB <- lb_const, b_ij <- B_lin[i][j] (or 0), c_ijkn <- F_ik
 * * D_jn for i != k and j != n, d <- 0.
 *   F, D      host, N x N int32 flow and distance matrices (Eq. (1)); entries
 *             must be >= 0; the diagonals are ignored (only i != k enters).
 *   N         RLT2_MIN_N .. RLT2_MAX_N.
 *   B_lin     host, N x N int32 linear costs b_ij (a branch-and-bound node's
 *             residual instance), or NULL for none.  Entries >= 0.
 *   lb_const  constant part of the objective (0 at the root).
 *   opts      options, or NULL for the defaults.
 *   out       receives the context.
 * Errors: RLT2_E_INVAL, RLT2_E_OVERFLOW when U = sum_{i!=k} F_ik * max_{j!=n}
 * D_jn + sum_i max_j B_lin[i][j] exceeds RLT2_LAP_MAX_ENTRY (every reduced
 * cost, class sum and Hungarian potential is then bounded by 3U and fits
 * int32), RLT2_E_OOM, RLT2_E_CUDA; RLT2_E_INVAL also for an unknown
 * opts->store.  Device memory: D in the chosen store (see RLT2_STORE_*) plus
 * 12 B * N^2 (N-1)^2; rlt2_state_bytes() gives the exact figure.
 */
int rlt2_create(const int32_t *F, const int32_t *D, int N, const int32_t *B_lin,
                int64_t lb_const, const rlt2_opts *opts, rlt2_ctx **out);

/* Release every resource of ctx (NULL is allowed). */
void rlt2_destroy(rlt2_ctx *ctx);

/*
 * Enqueue k passes of the loop of Algorithm 1 on the context's stream:
 * spread B->C (a pass over C), spread C->D with the transfer between
 * complementary costs of D (one fused pass over D), concentration D->C (N^2 (N-1)^2 Hungarian LAPs of
 * size N-2, Sec. 4.1), transfer between complementary costs of C fused into
 * concentration C->B (N^2 LAPs of size N-1), concentration B->LB (one LAP of
 * size N) and LB <- LB + LB'.  Returns without waiting for the GPU.  Passes
 * after the stopping rule of Algorithm 1 fired (opts.ub / opts.min_progress)
 * do nothing.  Errors: RLT2_E_INVAL (k < 0), RLT2_E_STATE (history full),
 * RLT2_E_CUDA.
 */
int rlt2_iterate(rlt2_ctx *ctx, int k);

/*
 * Wait for the context's stream and read the bound.
 *   lb        (may be NULL) LB as a double
 *   lb_exact  (may be NULL) LB as an exact int64
 *   iters     (may be NULL) passes completed so far
 * Errors: RLT2_E_TIMEOUT if a device-side wait gave up, RLT2_E_CUDA.
 */
int rlt2_bound(rlt2_ctx *ctx, double *lb, int64_t *lb_exact, int *iters);

/* LB after each completed pass, oldest first: up to cap values into host
 * buffer out; *count receives the number written. */
int rlt2_bound_history(rlt2_ctx *ctx, int64_t *out, int cap, int *count);

/*
 * Copy the current reduced costs to host memory in the compact layouts above.
 *   level 0: x (B), count N*N;  1: y (C), count N^2 (N-1)^2;
 *   2: z (D), count N^2 (N-1)^2 (N-2)^2.
 * Synchronises the context's stream.  Errors: RLT2_E_INVAL on a wrong count.
 */
int rlt2_get_state(rlt2_ctx *ctx, int level, int32_t *host_buf, size_t count);

/*
 * Cumulative work of the Hungarian method in this context (synchronises):
 * out[0] LAPs solved, out[1] steps (columns labelled), out[2] relaxations
 * (reduced distances evaluated for unlabelled columns), out[3..5] the same
 * three counts for the D->C concentrations alone.
 */
int rlt2_work(rlt2_ctx *ctx, int64_t out[6]);

/*
 * The context's D->C shape (see rlt2_opts.lanes and "Autotuning"): out[0]
 * lanes per LAP, out[1] warps per CTA of its launches, out[2] 1 while tuning
 * passes are still to come, else 0.  All 0 without D (RLT1 mode).
 */
int rlt2_dlap_shape(rlt2_ctx *ctx, int out[3]);

/*
 * Stage times recorded while opts.profile was set (synchronises): out[s] =
 * total milliseconds of stage s over all profiled passes, s = 0 spread B->C
 * and the fused spread/complementary pass over D, 1 concentration D->C, 2 complementary C +
 * concentration C->B, 3 concentration B->LB; *passes = passes recorded.
 * rlt2_reset_stage_times() clears the totals.
 */
int rlt2_stage_times(rlt2_ctx *ctx, double out[4], int *passes);
int rlt2_reset_stage_times(rlt2_ctx *ctx);

/* Device pointer of the context's state: which 0 = x, 1 = y (C), 2 = z, 3 =
 * the tile duals of the class-sum store.  In the tile store, tile t of z
 * holds N-2 rows (facilities p not in {i,k}) of rlt2_row_stride(N) =
 * round_up(N, 4) ints indexed by the location q itself; columns j and n of
 * the tile and q >= N hold no coefficient.  In the class-sum store, which 2
 * is the class sums T[tau(x,y,z) N^3 + lx N^2 + ly N + lz] (facilities x < y
 * < z at locations lx, ly, lz; tau = C(z,3) + C(y,2) + x) and which 3 the
 * duals, per tile round_up(N-2, 4) ints of u then round_up(N, 4) of v by
 * location.  Returns NULL on error or for a part the context does not have. */
void *rlt2_device_state(rlt2_ctx *ctx, int which);
int rlt2_row_stride(int N);

/*
 * Warm-started child of a branch-and-bound node (the paper does not say how a
 * node's bound starts; this is the warm form of the cold start rlt2_subproblem
 * gives).  The child fixes the parent's facility f to its location l (parent
 * indices); its facilities and locations are the parent's others, renumbered
 * in ascending order, and its state is the parent's dual state restricted to
 * the permutations with pi(f) = l:
 *   LB' = LB + b_fl,  b'_kn = b_kn + c_flkn + c_knfl,
 *   c'_knpq = c_knpq + d_flknpq + d_knflpq + d_knpqfl,  d' = d restricted,
 * all reduced costs >= 0 and LB' >= LB; further passes continue from there.
 * The child is a new context (N - 1) with the parent's store (tiles or pairs;
 * the class-sum store is refused) and RLT1 mode, opts for the rest; it is
 * derived on the device after every pass enqueued on the parent (its stream
 * waits for the parent's), and the call synchronises the child.
 * Errors: RLT2_E_INVAL (N - 1 < RLT2_MIN_N, f or l out of range, class-sum
 * store, bad opts), RLT2_E_OOM, RLT2_E_CUDA, RLT2_E_TIMEOUT / RLT2_E_INTERNAL
 * (a pending error of the parent's passes; no child).
 */
int rlt2_child(rlt2_ctx *parent, int f, int l, const rlt2_opts *opts, rlt2_ctx **out);

/*
 * Checkpoint and resume of a dual ascent (no counterpart in the paper, whose
 * runs are not interrupted; it serves long branch-and-bound runs).
 *
 * rlt2_save waits for the context's stream and writes its whole state to the
 * file `path` (created or truncated): LB, passes done, the stopping flag, the
 * LB history, B, C and the tile store of D as laid out on the device (about
 * the device memory of the context: 2.7 GB at N = 30).  Errors:
 * RLT2_E_INVAL, RLT2_E_IO (cannot write), RLT2_E_TIMEOUT / RLT2_E_INTERNAL
 * (a pending device error; nothing written), RLT2_E_CUDA.
 *
 * rlt2_load creates a new context from such a file; opts as for rlt2_create
 * (ub, min_progress, stream, graph and profile settings are taken from opts;
 * rlt1_only and the instance come from the file; opts->max_iters must be at
 * least the passes already done).  Passes after the load continue exactly as
 * the saved context would have.  Errors: RLT2_E_INVAL, RLT2_E_IO (unreadable,
 * truncated or not a checkpoint), RLT2_E_OOM, RLT2_E_CUDA.
 */
int rlt2_save(rlt2_ctx *ctx, const char *path);
int rlt2_load(const char *path, const rlt2_opts *opts, rlt2_ctx **out);

/* Bytes of device memory rlt2_create allocates for an instance of size N
 * with D in `store` (0 for N out of range); max_iters <= 0 means the default. */
size_t rlt2_state_bytes(int N, int rlt1_only, int max_iters, int store);

/*
 * Groups: several live contexts advanced together, every stage of every pass
 * one kernel launch for all of them (continuous batching: a server forms a new
 * group whenever contexts join or leave).  The group only references the
 * contexts' device state; each context's results are exactly those of
 * rlt2_iterate on it alone.
 *   rlt2_group_create   ctxs[count] (all RLT2 or all RLT1 mode); stream NULL:
 *                       a stream created for the group.  The group's launches
 *                       start after every context's pending work.
 *   rlt2_group_iterate  enqueue k passes of every member (returns at once);
 *                       every member's later calls wait for them.
 *   rlt2_group_sync     wait; RLT2_E_TIMEOUT / RLT2_E_INTERNAL if a kernel of
 *                       the group reported one.
 *   rlt2_group_destroy  waits, then releases the group (not the contexts).
 * A context may belong to one group at a time; destroy the group before its
 * contexts.
 */
typedef struct rlt2_group rlt2_group;
int rlt2_group_create(rlt2_ctx *const *ctxs, int count, void *stream, rlt2_group **out);
int rlt2_group_iterate(rlt2_group *group, int k);
int rlt2_group_sync(rlt2_group *group);
void rlt2_group_destroy(rlt2_group *group);

/* A branch-and-bound node (Sec. 6): facility fac[t] is fixed to location
 * loc[t], t < k; the facilities and locations are distinct. */
typedef struct {
    int k;
    const int32_t *fac;
    const int32_t *loc;
} rlt2_node;

/*
 * Residual instance of a node (host only, no GPU): free facilities and free
 * locations renumbered in ascending order (N' = N - k), and for any completion
 * pi' of the node
 *   Q(full pi) = lb_const + sum_x Blin[x][pi'(x)] + sum_{x!=y} Fp[x][y] Dp[pi'(x)][pi'(y)],
 *   Blin[x][y] = sum_t F[fx][fac t] D[ly][loc t] + F[fac t][fx] D[loc t][ly],
 *   lb_const   = sum_{t!=t'} F[fac t][fac t'] D[loc t][loc t'].
 * Fp, Dp, Blin: caller buffers of N'*N' int32.  Errors: RLT2_E_INVAL (bad or
 * repeated indices), RLT2_E_OVERFLOW (a linear cost beyond int32).  Bounding
 * (Fp, Dp, Blin, lb_const) with rlt2_create bounds the node.
 */
int rlt2_subproblem(const int32_t *F, const int32_t *D, int N, int k, const int32_t *fac,
                    const int32_t *loc, int32_t *Fp, int32_t *Dp, int32_t *Blin, int64_t *lb_const);

/*
 * Bound B nodes of one instance together: `iters` passes of Algorithm 1 on
 * each node's residual instance (cold start), every stage of every pass one
 * kernel launch for all nodes, all passes captured into one CUDA graph and
 * launched once.  Each node's result equals rlt2_create + rlt2_iterate(iters)
 * on its residual instance, bit for bit.
 *   F, D      host, N x N (the instance); nodes[B] (host); every N - k >= 3
 *   lb_out    host, B int64: each node's LB (lb_const included)
 *   ms_out    (may be NULL) milliseconds of device work from the first
 *             initialisation to the last pass (CUDA events)
 *   opts      stream (NULL: a stream created for the call), store, lanes,
 *             cta_warps; rlt1_only must be 0
 *   shape_out (may be NULL) int[4]: the D->C shape used after tuning, as
 *             (lanes per LAP, warps per CTA) for the nodes with N - k > 16,
 *             then for those with N - k <= 16 (0, 0 where there are none)
 * opts->lanes = 0: the first passes are tuning passes (see "Autotuning"),
 * the rest one captured graph.  Nodes of N' <= 16 are placed first
 * internally; lb_out keeps the caller's order.
 * One device allocation holds every node's state (about 4 B * N'^2 (N'-1)^2
 * (N'-2) * round_up(N',4) each) and is freed before returning; synchronises.
 * Errors: as rlt2_create, per node.
 */
int rlt2_batch_bound(const int32_t *F, const int32_t *D, int N, const rlt2_node *nodes, int B,
                     int iters, const rlt2_opts *opts, int64_t *lb_out, double *ms_out,
                     int *shape_out);

/*
 * Batched linear assignment with the library's Hungarian kernel (the LAP of
 * Sec. 4.1, solved by the method the dual ascent uses).  count independent
 * n x n problems, one warp each.
 *   M       device, count * n * n int32, row-major, entries in
 *           [0, RLT2_LAP_MAX_ENTRY]
 *   n       1 .. 64;  count >= 0
 *   S       device, count int64: optimal cost (-1 for a matrix with an entry
 *           out of range)
 *   assign  device, count * n int32: column of each row (may be NULL)
 *   u, v    device, count * n int32: row and column potentials; M - u - v
 *           is >= 0 and 0 on the assignment (each may be NULL)
 *   work    device, count * 2 int64: steps, relaxations (may be NULL)
 *   stream  cudaStream_t or NULL.
 * Synchronises the stream.  Errors: RLT2_E_INVAL (bad n/count/pointer or an
 * entry out of range: every other problem is still solved), RLT2_E_CUDA.
 */
int rlt2_lap_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                   int32_t *u, int32_t *v, int64_t *work, void *stream);

/*
 * Failure-detection self-test (no counterpart in the paper): one warp waits on
 * an mbarrier that nothing completes, through the same bounded wait every
 * device-side wait of the library uses, giving up after `polls` polls.
 * Nothing is in flight and nothing faults; the device stays usable.
 * Returns RLT2_E_TIMEOUT (the expected outcome), RLT2_E_INVAL (polls = 0) or
 * RLT2_E_CUDA.  Synchronises the stream.
 */
int rlt2_selftest_timeout(unsigned polls, void *stream);

/*
 * The same problems solved by the auction method, the LAP method the paper
 * uses on its GPU (Sec. 6; Bertsekas' auction), for comparison with the
 * Hungarian kernel.  One warp per problem, Gauss-Seidel bidding with
 * eps-scaling on costs scaled by n + 1 down to eps = 1, which makes the final
 * assignment optimal: S equals rlt2_lap_batch's S (the assignment may differ
 * where optima tie).  No potentials are returned (the auction's prices are not
 * the Hungarian method's duals).
 *   M, n, count, S, assign, stream: as rlt2_lap_batch
 *   work    device, count int64: bids placed (may be NULL)
 * Synchronises the stream.  Errors: as rlt2_lap_batch; RLT2_E_INTERNAL if a
 * problem needed more than 64 n^2 + 64 bids in one eps phase (S = -1 there).
 */
int rlt2_lap_batch_auction(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                           int64_t *work, void *stream);

/*
 * rlt2_lap_batch_static -- rlt2_lap_batch for callers that must not let a
 * library allocate device memory (the paper has no counterpart to this call).
 * Such callers hand all device memory to one owning allocator, run under a
 * hard memory budget, or cannot afford an allocation's latency or failure in
 * the middle of their work; rlt2_lap_batch would allocate a small status block
 * on every call.  This variant keeps that block (48 bytes: the kernel's error
 * bits and work counters) in a fixed array of the library's own device memory,
 * one per GPU, held from the library's loading until the process exits.
 *
 * Arguments, results and errors are those of rlt2_lap_batch; n beyond
 * RLT2_LAP_STATIC_MAX_N is rejected with RLT2_E_INVAL.  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) for that device and keeps it until the process
 *     exits; make that call before any stream capture on the device, and do
 *     not call this entry point on a device after cudaDeviceReset of it (the
 *     reset unloads the library's device code, and the array may move).
 *   - Every call on a device reuses the same block and clears it first; two
 *     calls whose work overlaps on the GPU (different streams, or host threads
 *     calling at once) race on it, so serialise them.
 *   - Synchronises the stream, like rlt2_lap_batch.
 */
#define RLT2_LAP_STATIC_MAX_N 64
int rlt2_lap_batch_static(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                          int32_t *u, int32_t *v, int64_t *work, void *stream);

/* ------------------------------------------------------------------------
 * FP64 form (the paper's real division).
 *
 * The same seven operations of Algorithm 1 with double costs, potentials and
 * bound: a cost x spread over m rows (Sec. 4.2) adds x/m (one IEEE division)
 * to every coefficient of the submatrix; a class of s complementary costs
 * (Sec. 4.3) is summed (from 0, in lexicographic rank order of its members)
 * and each member becomes T/s; the Hungarian method is that of the integer
 * form with every reduced distance formed as (M - u) - v and the potentials
 * moved after every step; S sums the LAP's columns in ascending order.  Every
 * double operation is defined in this order, so results are reproducible bit
 * for bit.  D is kept as tiles of N-2 rows by N location columns (8 B
 * N^3 (N-1)^2 (N-2); 5.1 GB at N = 30); no class or pair store, no groups,
 * batches, checkpoints or stopping rule.
 * ------------------------------------------------------------------------ */
typedef struct rlt2_f64_ctx rlt2_f64_ctx;

/*
 * Create an FP64 context, initialised as rlt2_create's (c_ijkn = F_ik * D_jn,
 * converted to double once).
 *   F, D, N   as rlt2_create (host int32, entries >= 0, N in 3..64)
 *   B_lin     host, N x N doubles >= 0 (finite), or NULL for 0
 *   lb_const  constant part of the objective (finite)
 *   opts      NULL or options: rlt1_only, profile, max_iters and stream are
 *             used; the rest are ignored
 * Errors: RLT2_E_INVAL, RLT2_E_OOM, RLT2_E_CUDA.
 */
int rlt2_f64_create(const int32_t *F, const int32_t *D, int N, const double *B_lin, double lb_const,
                    const rlt2_opts *opts, rlt2_f64_ctx **out);
void rlt2_f64_destroy(rlt2_f64_ctx *ctx);

/* Enqueue k passes (stream-ordered, no wait).  Errors: RLT2_E_INVAL (k < 0),
 * RLT2_E_STATE (more passes than opts.max_iters), RLT2_E_CUDA. */
int rlt2_f64_iterate(rlt2_f64_ctx *ctx, int k);

/* LB and the number of completed passes (synchronises).  Errors: RLT2_E_INTERNAL
 * if a Hungarian invariant failed (not for finite inputs), RLT2_E_CUDA. */
int rlt2_f64_bound(rlt2_f64_ctx *ctx, double *lb, int *iters);

/* LB after each completed pass, oldest first, up to cap into host out. */
int rlt2_f64_bound_history(rlt2_f64_ctx *ctx, double *out, int cap, int *count);

/* Reduced costs into host doubles, in the compact layouts of the integer form
 * (level 0 x: N*N, 1 y: N^2 (N-1)^2, 2 z: N^2 (N-1)^2 (N-2)^2).  Synchronises.
 * Errors: RLT2_E_INVAL on a wrong count (or level 2 in RLT1 mode). */
int rlt2_f64_get_state(rlt2_f64_ctx *ctx, int level, double *host_buf, size_t count);

/* Device pointer of x (which 0), y (1) or z (2: tile t at t * (N-2) * N doubles,
 * row r = rank of p among the facilities not in {i,k}, column = location q;
 * columns j and n hold 0), or NULL. */
void *rlt2_f64_device_state(rlt2_f64_ctx *ctx, int which);

/* Hungarian work as rlt2_work; stage times (opts.profile) as rlt2_stage_times. */
int rlt2_f64_work(rlt2_f64_ctx *ctx, int64_t out[6]);
int rlt2_f64_stage_times(rlt2_f64_ctx *ctx, double out[4], int *passes);

/*
 * The FP64 Hungarian method on count n x n problems, one warp each:
 *   M       device, count * n * n doubles, finite, row-major (left unchanged)
 *   S       device, count doubles: the assignment cost (columns summed in order)
 *   assign  device, count * n int32: column of each row (may be NULL)
 *   u, v    device, count * n doubles: row and column potentials (may be NULL)
 *   work    device, count * 2 int64: steps, relaxations (may be NULL)
 * n in 1..64.  Synchronises the stream.  Errors: RLT2_E_INVAL, RLT2_E_INTERNAL
 * (an invariant failed: a non-finite entry), RLT2_E_CUDA.
 */
int rlt2_f64_lap_batch(const double *M, int n, int count, double *S, int32_t *assign, double *u, double *v,
                       int64_t *work, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RLT2_H */
