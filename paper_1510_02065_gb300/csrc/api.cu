// api.cu -- the C ABI declared in include/rlt2.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/rlt2.h"
#include "device.cuh"
#include "kernels.h"

using namespace rlt2;

namespace {

int cuda_code(cudaError_t e)
{
    if (e == cudaSuccess) return RLT2_OK;
    if (e == cudaErrorMemoryAllocation) return RLT2_E_OOM;
    return RLT2_E_CUDA;
}

#define CK(call)                                     \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_code(e_); \
    } while (0)

// U bounds Q(pi) - LB for every permutation pi; every reduced cost lies on some
// pi and all are >= 0, so every cost and every class sum is <= U.
long long guard_U(const int32_t *F, const int32_t *D, int N, const int32_t *B)
{
    long long sf = 0, md = 0, sb = 0;
    for (int i = 0; i < N; i++)
        for (int k = 0; k < N; k++)
            if (i != k) {
                sf += F[i * N + k];
                md = std::max<long long>(md, D[i * N + k]);
            }
    if (B)
        for (int i = 0; i < N; i++) {
            long long mb = 0;
            for (int j = 0; j < N; j++) mb = std::max<long long>(mb, B[i * N + j]);
            sb += mb;
        }
    return sf * md + sb;
}

int check_instance(const int32_t *F, const int32_t *D, int N, const int32_t *B_lin, long long *U)
{
    if (!F || !D || N < RLT2_MIN_N || N > RLT2_MAX_N) return RLT2_E_INVAL;
    for (int e = 0; e < N * N; e++)
        if (F[e] < 0 || D[e] < 0 || (B_lin && B_lin[e] < 0)) return RLT2_E_INVAL;
    *U = guard_U(F, D, N, B_lin);
    return *U > RLT2_LAP_MAX_ENTRY ? RLT2_E_OVERFLOW : RLT2_OK;
}

long long n_triples(int N) { return (long long)N * (N - 1) * (N - 2) / 6; }

// Instances with N <= kSmallN (rows of at most 16 location columns) form a
// D->C range of their own in a group that also has larger ones, so that each
// range gets the lanes per tile that suit its width.
constexpr int kSmallN = 16;

bool lanes_opt_ok(const rlt2_opts &o)
{
    return (o.lanes == 0 || o.lanes == 16 || o.lanes == 32) &&
           (o.cta_warps == 0 || o.cta_warps == 4 || o.cta_warps == 16 || o.cta_warps == 32) &&
           !(o.lanes == 16 && o.cta_warps != 0);
}

// D->C shapes that can solve rows of width W with tiles of tsp ints, in the
// order the autotuner tries them, the default first (whole warps in the CTA
// size that keeps the most warps resident): a CTA of whole warps needs warps
// x (4 tsp + 8) bytes of shared memory, at most `optin` (a CTA of 32 warps
// stops fitting at N = 44, one of 16 at N = 61).
std::vector<DlapShape> shape_candidates(int W, bool paired, int tsp, int optin)
{
    std::vector<DlapShape> v;
    for (DlapShape d : {DlapShape{32, 0}, DlapShape{16, 0}, DlapShape{32, 4}, DlapShape{32, 16}, DlapShape{32, 32}})
        if (dlap_shape_fits(d, W, paired) && (d.warps == 0 || (long long)d.warps * (4LL * tsp + 8) <= optin))
            v.push_back(d);
    return v;
}

// Autotuner of a group's D->C shapes.  While active, each pass of the group is
// a tuning pass: the D->C ranges run one after the other, each in its next
// candidate shape, timed by CUDA events and measured by the device's
// relaxation counter; after the last candidate, the fastest per relaxation of
// each range becomes the group's shape (every shape gives identical results,
// so the tuning passes are ordinary passes).  The choice is remembered per
// device, store and row width, and later groups with the same key start with
// it and skip tuning.  A candidate that does not fit in shared memory (a CTA
// of many warps at large N) is skipped.
struct DlapTuner {
    std::vector<DlapShape> cand[2];
    int W[2] = {0, 0};
    int tried = -1, total = 0;  // tried = -1: the unmeasured first pass is still to come
    double best[2] = {0.0, 0.0};
    DlapShape bestS[2] = {{0, 0}, {0, 0}};
    int key_store = 0;
    bool active() const { return total > 0 && tried < total; }
};

constexpr int kMaxDev = 64;
std::mutex g_tuned_mutex;
DlapShape g_tuned[kMaxDev][3][65];  // per device, store kind, row width ({0, 0}: not yet)

int store_kind(const Group &g) { return g.sym ? 1 : g.paired ? 2 : 0; }

DlapShape tuned_shape(int store, int W)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || W < 0 || W > 64) return {0, 0};
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    return g_tuned[dev][store][W];
}

void remember_shape(int store, int W, DlapShape d)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev || W < 0 || W > 64) return;
    std::lock_guard<std::mutex> lock(g_tuned_mutex);
    g_tuned[dev][store][W] = d;
}

int range_width(const Group &g, int which) { return which == 0 ? (g.maxN + 3) & ~3 : g.smallW; }

bool range_empty(const Group &g, int which)
{
    return which == 0 ? g.dtiles <= g.small_tiles : g.small_tiles <= 0;
}

// The D->C shapes of a group from the options: forced (RLT2_E_INVAL if a
// forced shape cannot solve a range's rows), or remembered, or the default
// (whole warps in the CTA size that keeps the most warps resident) with the
// tuner armed.  Without D there is no D->C.
int setup_dshape(Group &g, const rlt2_opts &o, DlapTuner *tuner)
{
    if (tuner) *tuner = DlapTuner{};
    for (int r = 0; r < 2; r++) {
        g.dshape[r] = DlapShape{32, 0};
        if (g.rlt1_only || range_empty(g, r)) continue;
        const int W = range_width(g, r);
        if (o.lanes != 0 || o.cta_warps != 0) {
            DlapShape d{o.lanes ? o.lanes : 32, o.cta_warps};
            if (o.lanes == 0 && W <= 16 && !g.paired && o.cta_warps == 0) d.lanes = 16;
            if (!dlap_shape_fits(d, W, g.paired)) return RLT2_E_INVAL;
            int dev = 0, optin = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
                return RLT2_E_CUDA;
            if ((long long)d.warps * (4LL * (r == 0 ? g.maxTS : g.smallTS) + 8) > optin) return RLT2_E_INVAL;
            g.dshape[r] = d;
            continue;
        }
        const DlapShape known = tuned_shape(store_kind(g), W);
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return RLT2_E_CUDA;
        const std::vector<DlapShape> cand =
            shape_candidates(W, g.paired, r == 0 ? g.maxTS : g.smallTS, optin);
        g.dshape[r] = known.lanes ? known : DlapShape{32, 0};
        if (!known.lanes && tuner) {
            tuner->cand[r] = cand;
            tuner->W[r] = W;
            tuner->total = std::max(tuner->total, (int)cand.size());
        }
    }
    if (tuner) tuner->key_store = store_kind(g);
    return RLT2_OK;
}

// Facility triples i < k < p ordered by p, then k, then i: the first C(N,3)
// of the table for any larger N are exactly the triples of N.
std::vector<int4> triple_table(int N)
{
    std::vector<int4> t;
    for (int p = 2; p < N; p++)
        for (int k = 1; k < p; k++)
            for (int i = 0; i < k; i++) t.push_back(make_int4(i, k, p, 0));
    return t;
}

// Device memory carved from one allocation (256-byte aligned pieces).
struct Arena {
    size_t used = 0;
    size_t take(size_t bytes)
    {
        const size_t off = used;
        used += (bytes + 255) & ~size_t(255);
        return off;
    }
};

// One instance's state inside an arena (byte offsets).
struct NodeOffsets {
    size_t z, T, du, yS, yC, x, LB, hist, iter, stop;
};

constexpr size_t kNone = (size_t)-1;

// D (with_d) in the tile store, the class-sum store or the pair store (RLT2_STORE_*).
NodeOffsets plan_node(Arena &a, int N, bool with_d, int store, int hist_cap)
{
    const Geom g = make_geom(N);
    const bool sym = store == RLT2_STORE_CLASSES;
    NodeOffsets o;
    o.z = with_d && !sym ? a.take((size_t)(store == RLT2_STORE_PAIRS ? g.htiles : g.tiles) * g.TS * 4) : kNone;
    o.T = with_d && sym ? a.take((size_t)g.classes_ints * 4) : kNone;
    o.du = with_d && sym ? a.take((size_t)g.tiles * g.DS * 4) : kNone;
    o.yS = a.take((size_t)g.tiles * 4);
    o.yC = a.take((size_t)g.tiles * 4);
    o.x = a.take((size_t)N * N * 4);
    o.LB = a.take(8);
    o.hist = a.take((size_t)hist_cap * 8);
    o.iter = a.take(4);
    o.stop = a.take(4);
    return o;
}

PassState node_state(char *base, const NodeOffsets &o, int hist_cap, const rlt2_opts &opts)
{
    PassState p{};
    p.z = o.z == kNone ? nullptr : reinterpret_cast<int *>(base + o.z);
    p.T = o.T == kNone ? nullptr : reinterpret_cast<int *>(base + o.T);
    p.du = o.du == kNone ? nullptr : reinterpret_cast<int *>(base + o.du);
    p.yS = reinterpret_cast<int *>(base + o.yS);
    p.yC = reinterpret_cast<int *>(base + o.yC);
    p.x = reinterpret_cast<int *>(base + o.x);
    p.LB = reinterpret_cast<long long *>(base + o.LB);
    p.hist = reinterpret_cast<long long *>(base + o.hist);
    p.iter = reinterpret_cast<int *>(base + o.iter);
    p.stop = reinterpret_cast<int *>(base + o.stop);
    p.hist_cap = hist_cap;
    p.ub = opts.ub;
    p.min_progress = opts.min_progress;
    return p;
}

// Copy F, D (and B_lin) of one instance to the device and run the
// initialisation of Algorithm 1 on it.
cudaError_t init_node(const NodeDesc &nd, const int32_t *F, const int32_t *D, const int32_t *B_lin,
                      long long lb_const, int32_t *staging, cudaStream_t s)
{
    const size_t nn = (size_t)nd.N * nd.N;
    cudaError_t e = cudaMemcpyAsync(staging, F, nn * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(staging + nn, D, nn * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && B_lin)
        e = cudaMemcpyAsync(staging + 2 * nn, B_lin, nn * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_init(nd, staging, staging + nn, B_lin ? staging + 2 * nn : nullptr, lb_const, s);
    return e;
}

// One pass of Algorithm 1 for the whole group.  ev: 5 events around the stages.
// NVTX range around the host-side enqueue of one stage (visible in timeline
// profilers; no cost without a tool attached).
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
};

// A tuning pass's events before, between and after the two D->C ranges
// (small instances first); the device work counters at those points are
// copied to g.snap on the device, so the pass enqueues without waiting.
struct TunePass {
    cudaEvent_t te[3];
};

cudaError_t enqueue_pass(const Group &g, int sm_count, cudaStream_t s, cudaEvent_t *ev,
                         const SideStream *side = nullptr, TunePass *tp = nullptr)
{
    cudaError_t e;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    if (!g.rlt1_only) {
        {
            StageRange r("rlt2: spread B->C, C->D + complementary D");
            if ((e = launch_p1(g, s)) != cudaSuccess) return e;
        }
        if ((e = mark(1)) != cudaSuccess) return e;
        StageRange r("rlt2: concentration D->C");
        if (!tp) {
            if ((e = launch_dlap(g, sm_count, s, side)) != cudaSuccess) return e;
        } else {
            // the two ranges one after the other, measured
            for (int k = 0; k < 3; k++) {
                if ((e = cudaMemcpyAsync(g.snap + k, g.status, sizeof(DevStatus), cudaMemcpyDeviceToDevice, s)) !=
                        cudaSuccess ||
                    (e = cudaEventRecord(tp->te[k], s)) != cudaSuccess)
                    return e;
                if (k < 2 && (e = launch_dlap_range(g, 1 - k, sm_count, s)) != cudaSuccess) return e;
            }
        }
    } else if ((e = mark(1)) != cudaSuccess) {
        return e;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    {
        StageRange r("rlt2: complementary C + concentration C->B");
        if ((e = launch_clap(g, s)) != cudaSuccess) return e;
    }
    if ((e = mark(3)) != cudaSuccess) return e;
    {
        StageRange r("rlt2: concentration B->LB");
        if ((e = launch_xlap(g, s)) != cudaSuccess) return e;
    }
    return mark(4);
}

cudaError_t capture_passes(const Group &g, int sm_count, cudaStream_t s, int passes,
                           cudaGraph_t *graph, cudaGraphExec_t *exec, const SideStream *side = nullptr)
{
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = cudaSuccess;
    for (int t = 0; t < passes && e2 == cudaSuccess; t++) e2 = enqueue_pass(g, sm_count, s, nullptr, side);
    e = cudaStreamEndCapture(s, graph);
    if (e2 != cudaSuccess) return e2;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(exec, *graph, 0);
}

// One pass of group g as a tuning pass of t (see DlapTuner); synchronises s.
// The first is a plain pass in the group's default shape, unmeasured: pass 1
// of a dual ascent does other work than later ones, and it loads the kernels.
int tune_step(Group &g, DlapTuner &t, int sm_count, cudaStream_t s, cudaEvent_t *ev)
{
    if (t.tried < 0) {
        CK(enqueue_pass(g, sm_count, s, ev));
        t.tried = 0;
        return RLT2_OK;
    }
    Group gt = g;
    DlapShape tried[2] = {{0, 0}, {0, 0}};
    for (int r = 0; r < 2; r++)
        if (!t.cand[r].empty()) gt.dshape[r] = tried[r] = t.cand[r][t.tried % t.cand[r].size()];
    TunePass tp{};
    DevStatus st[3];
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; k++) e = cudaEventCreate(&tp.te[k]);
    if (e == cudaSuccess) e = enqueue_pass(gt, sm_count, s, ev, nullptr, &tp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st, g.snap, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms[2] = {0.f, 0.f};
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[1], tp.te[0], tp.te[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[0], tp.te[1], tp.te[2]);
    for (cudaEvent_t ev2 : tp.te)
        if (ev2) cudaEventDestroy(ev2);
    if (e != cudaSuccess) return cuda_code(e);
    // work of each range: Hungarian steps (a step costs the same instructions
    // in every pass, while the relaxations per step change from pass to pass)
    const double work[2] = {(double)(st[2].dsteps - st[1].dsteps), (double)(st[1].dsteps - st[0].dsteps)};
    // the default (measured first) stays unless a candidate is clearly faster:
    // one pass's time per step drifts by a percent or two from pass to pass
    constexpr double kMargin = 0.97;
    for (int r = 0; r < 2; r++) {
        if (!tried[r].lanes || work[r] <= 0) continue;
        const double per = ms[r] / work[r];
        if (!t.bestS[r].lanes || per < kMargin * t.best[r]) {
            t.best[r] = per;
            t.bestS[r] = tried[r];
        }
    }
    if (++t.tried == t.total)
        for (int r = 0; r < 2; r++)
            if (t.bestS[r].lanes) {
                g.dshape[r] = t.bestS[r];
                remember_shape(t.key_store, t.W[r], t.bestS[r]);
            }
    return RLT2_OK;
}

int group_status(const Group &g, cudaStream_t s)
{
    int err = 0;
    CK(cudaMemcpyAsync(&err, &g.status->err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err & kDevTimeout) return RLT2_E_TIMEOUT;
    if (err & kDevInternal) return RLT2_E_INTERNAL;
    return RLT2_OK;
}

}  // namespace

struct rlt2_ctx {
    rlt2_opts opts;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    char *mem = nullptr;   // all device state of the context, one allocation
    Group g{};             // a group of one instance
    NodeDesc node{};       // host copy of that instance's descriptor
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int enqueued = 0;
    long long U = 0;       // the int32 guard's bound of the instance (kept for checkpoints)
    // profiling: 5 events per pass, recorded on the stream between the stages
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    DlapTuner tuner;       // D->C shape tuning on the first passes (opts.lanes = 0)
};

static void free_ctx(rlt2_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    cudaFree(c->mem);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

extern "C" {

void rlt2_default_opts(rlt2_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->use_graph = 1;
    o->max_iters = 65536;
}

const char *rlt2_strerror(int code)
{
    switch (code) {
    case RLT2_OK: return "ok";
    case RLT2_E_INVAL: return "invalid argument";
    case RLT2_E_OOM: return "out of memory";
    case RLT2_E_OVERFLOW: return "costs too large for exact int32 arithmetic";
    case RLT2_E_CUDA: return "CUDA runtime error";
    case RLT2_E_TIMEOUT: return "a bounded device-side wait gave up";
    case RLT2_E_STATE: return "call out of order or capacity exhausted";
    case RLT2_E_INTERNAL: return "an internal consistency check of a kernel failed";
    case RLT2_E_IO: return "checkpoint file could not be written or read, or is not a checkpoint";
    default: return "unknown error";
    }
}

int rlt2_row_stride(int N) { return (N + 3) & ~3; }

void rlt2_destroy(rlt2_ctx *c) { free_ctx(c); }

}  // extern "C"

// Allocate and describe the device state of a context of size N (no
// initialisation of the costs): stream, one arena, the instance descriptor,
// the group of one, the triple table, zeroed status and work counter.
// *stage receives 3 N^2 ints of device staging memory.
static int setup_ctx(rlt2_ctx *c, int N, bool with_d, int store, long long U, int32_t **stage)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RLT2_E_CUDA;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RLT2_E_CUDA;
    if (c->opts.stream) {
        c->stream = (cudaStream_t)c->opts.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return RLT2_E_CUDA;
        c->own_stream = true;
    }
    const bool sym = with_d && store == RLT2_STORE_CLASSES, paired = with_d && store == RLT2_STORE_PAIRS;
    const int JC = p1_chunk(N, sym, paired);
    const std::vector<int4> tri = triple_table(N);
    Arena a;
    const NodeOffsets no = plan_node(a, N, with_d, store, c->opts.max_iters);
    const size_t o_node = a.take(sizeof(NodeDesc));
    const size_t o_tri = a.take(tri.size() * sizeof(int4));
    const size_t o_cnt = a.take(8);
    const size_t o_st = a.take(sizeof(DevStatus));
    const size_t o_snap = a.take(3 * sizeof(DevStatus));
    const size_t o_stage = a.take((size_t)3 * N * N * 4);
    cudaError_t e = cudaMalloc((void **)&c->mem, a.used);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->mem = nullptr;
        return cuda_code(e);
    }
    char *base = c->mem;
    NodeDesc &nd = c->node;
    nd.paired = paired;
    fill_node(nd, N, JC);
    nd.p = node_state(base, no, c->opts.max_iters, c->opts);
    encode_zmap(nd, JC);
    nd.tile_base = 0;
    nd.dtile_base = 0;
    nd.cta_base = 0;
    nd.prob_base = 0;

    Group &g = c->g;
    g.nodes = reinterpret_cast<const NodeDesc *>(base + o_node);
    g.B = 1;
    g.tiles = nd.tiles;
    g.ctas = (int)(n_triples(N) * nd.nchunks);
    g.probs = N * N;
    g.maxN = N;
    g.maxTS = nd.TS;
    g.JC = JC;
    g.pack = 3 * U < (1LL << 25);
    g.rlt1_only = !with_d;
    g.sym = sym;
    g.paired = paired;
    g.dtiles = nd.dtiles;
    // one instance: one D->C range, its shape forced, remembered or tuned
    g.small_tiles = 0;
    g.smallTS = nd.TS;
    g.smallW = nd.W;
    const int rc_shape = setup_dshape(g, c->opts, &c->tuner);
    if (rc_shape != RLT2_OK) return rc_shape;
    g.counter = reinterpret_cast<unsigned *>(base + o_cnt);
    g.status = reinterpret_cast<DevStatus *>(base + o_st);
    g.snap = reinterpret_cast<DevStatus *>(base + o_snap);
    g.triples = reinterpret_cast<const int4 *>(base + o_tri);
    g.first = nd;
    c->U = U;

    e = cudaMemcpyAsync(base + o_node, &nd, sizeof(NodeDesc), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_tri, tri.data(), tri.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.status, 0, sizeof(DevStatus), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.counter, 0, 8, c->stream);
    // the table must outlive its asynchronous copy
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_code(e);
    *stage = reinterpret_cast<int32_t *>(base + o_stage);
    return RLT2_OK;
}

static rlt2_ctx *new_ctx(const rlt2_opts *opts)
{
    rlt2_ctx *c = new (std::nothrow) rlt2_ctx();
    if (!c) return nullptr;
    if (opts) c->opts = *opts;
    else rlt2_default_opts(&c->opts);
    if (c->opts.max_iters <= 0) c->opts.max_iters = 65536;
    return c;
}

// Checkpoint file: this header, then the LB history (iter int64), B (N^2
// int32), C after its last concentration (tiles int32) and, with D, the tile
// store as laid out on the device (tiles x (N-2) x round_up(N,4) int32) or
// the class sums (C(N,3) N^3 int32) and the tile duals (tiles x DS int32).
struct CkptHeader {
    char magic[8];
    int32_t version, N, with_d, iter, stop, store;
    int64_t LB, U, tiles, z_ints;
};
static const char kCkptMagic[8] = {'R', 'L', 'T', '2', 'C', 'K', 'P', 'T'};

// Move `bytes` between a FILE and device memory through a bounded host buffer.
static int file_device(FILE *f, char *dev, size_t bytes, bool to_file, cudaStream_t s)
{
    const size_t chunk = (size_t)64 << 20;
    std::vector<char> buf(std::min(bytes, chunk));
    for (size_t off = 0; off < bytes; off += chunk) {
        const size_t n = std::min(chunk, bytes - off);
        if (to_file) {
            if (cudaMemcpyAsync(buf.data(), dev + off, n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RLT2_E_CUDA;
            if (std::fwrite(buf.data(), 1, n, f) != n) return RLT2_E_IO;
        } else {
            if (std::fread(buf.data(), 1, n, f) != n) return RLT2_E_IO;
            if (cudaMemcpyAsync(dev + off, buf.data(), n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RLT2_E_CUDA;
        }
    }
    return RLT2_OK;
}

extern "C" {

int rlt2_create(const int32_t *F, const int32_t *D, int N, const int32_t *B_lin, int64_t lb_const,
                const rlt2_opts *opts, rlt2_ctx **out)
{
    if (!out) return RLT2_E_INVAL;
    *out = nullptr;
    long long U = 0;
    int rc = check_instance(F, D, N, B_lin, &U);
    if (rc != RLT2_OK) return rc;
    rlt2_ctx *c = new_ctx(opts);
    if (!c) return RLT2_E_OOM;
    int32_t *stage = nullptr;
    if ((c->opts.store != RLT2_STORE_TILES && c->opts.store != RLT2_STORE_CLASSES &&
         c->opts.store != RLT2_STORE_PAIRS) ||
        !lanes_opt_ok(c->opts)) {
        free_ctx(c);
        return RLT2_E_INVAL;
    }
    rc = setup_ctx(c, N, !c->opts.rlt1_only, c->opts.store, U, &stage);
    if (rc != RLT2_OK) {
        free_ctx(c);
        return rc;
    }
    cudaError_t e = init_node(c->node, F, D, B_lin, lb_const, stage, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_code(e);
    }
    *out = c;
    return RLT2_OK;
}

int rlt2_child(rlt2_ctx *par, int f, int l, const rlt2_opts *opts, rlt2_ctx **out)
{
    if (!par || !out) return RLT2_E_INVAL;
    *out = nullptr;
    const NodeDesc &pn = par->node;
    const int N = pn.N;
    if (N - 1 < RLT2_MIN_N || f < 0 || f >= N || l < 0 || l >= N || pn.p.T) return RLT2_E_INVAL;
    rlt2_ctx *c = new_ctx(opts);
    if (!c) return RLT2_E_OOM;
    c->opts.rlt1_only = pn.p.z == nullptr;
    c->opts.store = pn.paired ? RLT2_STORE_PAIRS : RLT2_STORE_TILES;
    if (!lanes_opt_ok(c->opts)) {
        free_ctx(c);
        return RLT2_E_INVAL;
    }
    int32_t *stage = nullptr;
    int rc = setup_ctx(c, N - 1, pn.p.z != nullptr, c->opts.store, par->U, &stage);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaSuccess;
    if (rc == RLT2_OK) {
        // after every pass enqueued on the parent
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, par->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, ev, 0);
        if (e == cudaSuccess) e = launch_child(pn, c->node, f, l, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (ev) cudaEventDestroy(ev);
        if (e != cudaSuccess) rc = cuda_code(e);
    }
    if (rc == RLT2_OK) rc = group_status(par->g, par->stream);  // the parent's passes were sound
    if (rc != RLT2_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return RLT2_OK;
}

int rlt2_save(rlt2_ctx *c, const char *path)
{
    if (!c || !path) return RLT2_E_INVAL;
    int64_t lb = 0;
    int it = 0;
    int rc = rlt2_bound(c, nullptr, &lb, &it);  // synchronises; reports device errors
    if (rc != RLT2_OK) return rc;
    const NodeDesc &nd = c->node;
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.N = nd.N;
    h.with_d = nd.p.z != nullptr || nd.p.T != nullptr;
    h.store = nd.p.T ? RLT2_STORE_CLASSES : nd.paired ? RLT2_STORE_PAIRS : RLT2_STORE_TILES;
    h.iter = it;
    CK(cudaMemcpy(&h.stop, nd.p.stop, 4, cudaMemcpyDeviceToHost));
    h.LB = lb;
    h.U = c->U;
    h.tiles = nd.tiles;
    h.z_ints = !h.with_d                     ? 0
               : h.store == RLT2_STORE_CLASSES ? make_geom(nd.N).classes_ints + nd.tiles * nd.DS
                                               : nd.dtiles * nd.TS;
    FILE *f = std::fopen(path, "wb");
    if (!f) return RLT2_E_IO;
    const int nh = std::min(it, c->opts.max_iters);
    rc = std::fwrite(&h, sizeof(h), 1, f) == 1 ? RLT2_OK : RLT2_E_IO;
    if (rc == RLT2_OK) rc = file_device(f, (char *)nd.p.hist, (size_t)nh * 8, true, c->stream);
    if (rc == RLT2_OK) rc = file_device(f, (char *)nd.p.x, (size_t)nd.N * nd.N * 4, true, c->stream);
    if (rc == RLT2_OK) rc = file_device(f, (char *)nd.p.yC, (size_t)nd.tiles * 4, true, c->stream);
    const bool hsym = h.store == RLT2_STORE_CLASSES;
    if (rc == RLT2_OK && h.with_d && !hsym)
        rc = file_device(f, (char *)nd.p.z, (size_t)h.z_ints * 4, true, c->stream);
    if (rc == RLT2_OK && hsym)
        rc = file_device(f, (char *)nd.p.T, (size_t)make_geom(nd.N).classes_ints * 4, true, c->stream);
    if (rc == RLT2_OK && hsym) rc = file_device(f, (char *)nd.p.du, (size_t)nd.tiles * nd.DS * 4, true, c->stream);
    if (std::fclose(f) != 0 && rc == RLT2_OK) rc = RLT2_E_IO;
    return rc;
}

int rlt2_load(const char *path, const rlt2_opts *opts, rlt2_ctx **out)
{
    if (!path || !out) return RLT2_E_INVAL;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return RLT2_E_IO;
    CkptHeader h{};
    int rc = RLT2_OK;
    rlt2_ctx *c = nullptr;
    do {
        if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1 ||
            h.N < RLT2_MIN_N || h.N > RLT2_MAX_N || h.iter < 0 || h.U < 0 || h.U > RLT2_LAP_MAX_ENTRY ||
            h.tiles != make_geom(h.N).tiles || h.store < RLT2_STORE_TILES || h.store > RLT2_STORE_PAIRS ||
            (h.store != RLT2_STORE_TILES && !h.with_d) ||
            h.z_ints != (!h.with_d ? 0
                         : h.store == RLT2_STORE_CLASSES
                             ? make_geom(h.N).classes_ints + h.tiles * (long long)make_geom(h.N).DS
                         : h.store == RLT2_STORE_PAIRS ? make_geom(h.N).htiles * (long long)make_geom(h.N).TS
                                                       : h.tiles * (long long)make_geom(h.N).TS)) {
            rc = RLT2_E_IO;
            break;
        }
        c = new_ctx(opts);
        if (!c) {
            rc = RLT2_E_OOM;
            break;
        }
        c->opts.rlt1_only = !h.with_d;
        c->opts.store = h.store;
        if (h.iter > c->opts.max_iters || !lanes_opt_ok(c->opts)) {  // the history must fit
            rc = RLT2_E_INVAL;
            break;
        }
        int32_t *stage = nullptr;
        if ((rc = setup_ctx(c, h.N, h.with_d != 0, h.store, h.U, &stage)) != RLT2_OK) break;
        const bool hsym = h.store == RLT2_STORE_CLASSES;
        const NodeDesc &nd = c->node;
        if ((rc = file_device(f, (char *)nd.p.hist, (size_t)h.iter * 8, false, c->stream)) != RLT2_OK) break;
        if ((rc = file_device(f, (char *)nd.p.x, (size_t)h.N * h.N * 4, false, c->stream)) != RLT2_OK) break;
        if ((rc = file_device(f, (char *)nd.p.yC, (size_t)h.tiles * 4, false, c->stream)) != RLT2_OK) break;
        if (h.with_d && !hsym &&
            (rc = file_device(f, (char *)nd.p.z, (size_t)h.z_ints * 4, false, c->stream)) != RLT2_OK)
            break;
        if (hsym && (rc = file_device(f, (char *)nd.p.T, (size_t)make_geom(h.N).classes_ints * 4, false,
                                       c->stream)) != RLT2_OK)
            break;
        if (hsym &&
            (rc = file_device(f, (char *)nd.p.du, (size_t)h.tiles * nd.DS * 4, false, c->stream)) != RLT2_OK)
            break;
        cudaError_t e = cudaMemcpyAsync(nd.p.LB, &h.LB, 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(nd.p.iter, &h.iter, 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(nd.p.stop, &h.stop, 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            rc = cuda_code(e);
            break;
        }
        c->enqueued = h.iter;
    } while (false);
    std::fclose(f);
    if (rc != RLT2_OK) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return RLT2_OK;
}

int rlt2_iterate(rlt2_ctx *c, int k)
{
    if (!c || k < 0) return RLT2_E_INVAL;
    if ((long long)c->enqueued + k > c->opts.max_iters) return RLT2_E_STATE;
    for (int t = 0; t < k; t++) {
        cudaEvent_t *ev = nullptr;
        if (c->opts.profile) {
            while (c->events.size() < c->ev_used + 5) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                c->events.push_back(e);
            }
            ev = &c->events[c->ev_used];
            c->ev_used += 5;
        }
        if (c->tuner.active()) {
            const int rc = tune_step(c->g, c->tuner, c->sm_count, c->stream, ev);
            if (rc != RLT2_OK) return rc;
        } else if (c->opts.use_graph && !ev) {
            if (!c->gexec) CK(capture_passes(c->g, c->sm_count, c->stream, 1, &c->graph, &c->gexec));
            CK(cudaGraphLaunch(c->gexec, c->stream));
        } else {
            CK(enqueue_pass(c->g, c->sm_count, c->stream, ev));  // profiling: stage by stage
        }
        c->enqueued++;
    }
    return RLT2_OK;
}

int rlt2_bound(rlt2_ctx *c, double *lb, int64_t *lb_exact, int *iters)
{
    if (!c) return RLT2_E_INVAL;
    long long v = 0;
    int it = 0;
    CK(cudaMemcpyAsync(&v, c->node.p.LB, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&it, c->node.p.iter, 4, cudaMemcpyDeviceToHost, c->stream));
    int rc = group_status(c->g, c->stream);
    if (lb) *lb = (double)v;
    if (lb_exact) *lb_exact = v;
    if (iters) *iters = it;
    return rc;
}

int rlt2_bound_history(rlt2_ctx *c, int64_t *out, int cap, int *count)
{
    if (!c || (!out && cap > 0) || cap < 0) return RLT2_E_INVAL;
    int it = 0;
    CK(cudaMemcpyAsync(&it, c->node.p.iter, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int n = std::min(std::min(it, cap), c->opts.max_iters);
    if (n > 0) CK(cudaMemcpy(out, c->node.p.hist, (size_t)n * 8, cudaMemcpyDeviceToHost));
    if (count) *count = n;
    return RLT2_OK;
}

int rlt2_get_state(rlt2_ctx *c, int level, int32_t *host, size_t count)
{
    if (!c || !host) return RLT2_E_INVAL;
    const NodeDesc &nd = c->node;
    const int N = nd.N, n = N - 2;
    if (level == 0) {
        if (count != (size_t)N * N) return RLT2_E_INVAL;
        CK(cudaMemcpyAsync(host, nd.p.x, count * 4, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 1) {
        if (count != (size_t)nd.tiles) return RLT2_E_INVAL;
        CK(cudaMemcpyAsync(host, nd.p.yC, count * 4, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 2) {
        if ((!nd.p.z && !nd.p.T) || count != (size_t)nd.tiles * n * n) return RLT2_E_INVAL;
        // the store's rows are indexed by location: drop the tile's own two
        // locations (and the padding) to reach the compact layout; the
        // class-sum store is first expanded to that layout on the device
        std::vector<int32_t> tmp;
        try {
            tmp.resize((size_t)nd.dtiles * nd.TS);
        } catch (...) {
            return RLT2_E_OOM;
        }
        if (nd.p.z) {
            CK(cudaMemcpyAsync(tmp.data(), nd.p.z, tmp.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        } else {
            int *dz = nullptr;
            cudaError_t e = cudaMallocAsync((void **)&dz, tmp.size() * 4, c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return cuda_code(e);
            }
            e = launch_materialize(nd, dz, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tmp.data(), dz, tmp.size() * 4, cudaMemcpyDeviceToHost, c->stream);
            cudaFreeAsync(dz, c->stream);
            if (e != cudaSuccess) return cuda_code(e);
        }
        CK(cudaStreamSynchronize(c->stream));
        const int m = N - 1, W = nd.W;
        size_t o = 0;
        for (long long t = 0; t < nd.tiles; t++) {
            const int nn = (int)(t % m), j = (int)((t / ((long long)m * m)) % N);
            const int ij = (int)(t / ((long long)m * m)), i = ij / N, kk = (int)((t / m) % m);
            const int k = kk + (kk >= i);
            const int nl = nn + (nn >= j);
            if (nd.paired && k < i) {  // pair store: the complement holds the pair, this tile is 0
                for (int e = 0; e < n * n; e++) host[o++] = 0;
                continue;
            }
            const long long ts = nd.paired ? ((long long)pair_index(i, k) * N + j) * m + nn : t;
            const int32_t *src = tmp.data() + (size_t)ts * nd.TS;
            for (int r = 0; r < n; r++)
                for (int q = 0; q < N; q++)
                    if (q != j && q != nl) host[o++] = src[r * W + q];
        }
    } else {
        return RLT2_E_INVAL;
    }
    CK(cudaStreamSynchronize(c->stream));
    return RLT2_OK;
}

int rlt2_dlap_shape(rlt2_ctx *c, int out[3])
{
    if (!c || !out) return RLT2_E_INVAL;
    const bool d = !c->g.rlt1_only;
    out[0] = d ? c->g.dshape[0].lanes : 0;
    out[1] = d ? dlap_cta_warps(c->g, 0) : 0;
    out[2] = d && c->tuner.active() ? 1 : 0;
    return RLT2_OK;
}

int rlt2_work(rlt2_ctx *c, int64_t out[6])
{
    if (!c || !out) return RLT2_E_INVAL;
    DevStatus s;
    CK(cudaMemcpyAsync(&s, c->g.status, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out[0] = (int64_t)s.laps;
    out[1] = (int64_t)s.steps;
    out[2] = (int64_t)s.relax;
    out[3] = (int64_t)s.dlaps;
    out[4] = (int64_t)s.dsteps;
    out[5] = (int64_t)s.drelax;
    return RLT2_OK;
}

int rlt2_stage_times(rlt2_ctx *c, double out[4], int *passes)
{
    if (!c || !out) return RLT2_E_INVAL;
    CK(cudaStreamSynchronize(c->stream));
    double acc[4] = {0, 0, 0, 0};
    for (size_t b = 0; b + 5 <= c->ev_used; b += 5)
        for (int s = 0; s < 4; s++) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->events[b + s], c->events[b + s + 1]));
            acc[s] += ms;
        }
    for (int s = 0; s < 4; s++) out[s] = acc[s];
    if (passes) *passes = (int)(c->ev_used / 5);
    return RLT2_OK;
}

int rlt2_reset_stage_times(rlt2_ctx *c)
{
    if (!c) return RLT2_E_INVAL;
    CK(cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    return RLT2_OK;
}

void *rlt2_device_state(rlt2_ctx *c, int which)
{
    if (!c) return nullptr;
    switch (which) {
    case 0: return c->node.p.x;
    case 1: return c->node.p.yC;
    case 2: return c->node.p.z ? (void *)c->node.p.z : (void *)c->node.p.T;
    case 3: return c->node.p.du;
    default: return nullptr;
    }
}

size_t rlt2_state_bytes(int N, int rlt1_only, int max_iters, int store)
{
    if (N < RLT2_MIN_N || N > RLT2_MAX_N) return 0;
    if (max_iters <= 0) max_iters = 65536;
    Arena a;
    plan_node(a, N, !rlt1_only, store, max_iters);
    a.take(sizeof(NodeDesc));
    a.take((size_t)n_triples(N) * sizeof(int4));
    a.take(4);
    a.take(sizeof(DevStatus));
    a.take((size_t)3 * N * N * 4);
    return a.used;
}

}  // extern "C"

// ------------------------------------------------------- groups of contexts

struct rlt2_group {
    Group g{};
    char *mem = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    std::vector<rlt2_ctx *> ctxs;
    cudaEvent_t done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SideStream side{};     // the small instances' D->C range beside the other one
};

static int make_side(SideStream &sd)
{
    if (cudaStreamCreateWithFlags(&sd.s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming) != cudaSuccess)
        return RLT2_E_CUDA;
    return RLT2_OK;
}

static void free_side(SideStream &sd)
{
    if (sd.s2) cudaStreamSynchronize(sd.s2);
    if (sd.fork) cudaEventDestroy(sd.fork);
    if (sd.join) cudaEventDestroy(sd.join);
    if (sd.s2) cudaStreamDestroy(sd.s2);
    sd = SideStream{};
}

static void free_group(rlt2_group *gr)
{
    if (!gr) return;
    if (gr->stream) cudaStreamSynchronize(gr->stream);
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    if (gr->done) cudaEventDestroy(gr->done);
    free_side(gr->side);
    cudaFree(gr->mem);
    if (gr->own_stream && gr->stream) cudaStreamDestroy(gr->stream);
    delete gr;
}

extern "C" {

int rlt2_group_create(rlt2_ctx *const *ctxs, int count, void *stream, rlt2_group **out)
{
    if (!out || !ctxs || count < 1) return RLT2_E_INVAL;
    *out = nullptr;
    for (int b = 0; b < count; b++) {
        if (!ctxs[b] || ctxs[b]->g.rlt1_only != ctxs[0]->g.rlt1_only || ctxs[b]->g.sym != ctxs[0]->g.sym ||
            ctxs[b]->g.paired != ctxs[0]->g.paired)
            return RLT2_E_INVAL;
        // a context twice would give two descriptors of one state, whose
        // passes in the same launches would race on it
        for (int b2 = 0; b2 < b; b2++)
            if (ctxs[b2] == ctxs[b]) return RLT2_E_INVAL;
    }
    rlt2_group *gr = new (std::nothrow) rlt2_group();
    if (!gr) return RLT2_E_OOM;
    auto fail = [&](int code) {
        free_group(gr);
        return code;
    };
    gr->ctxs.assign(ctxs, ctxs + count);
    gr->sm_count = ctxs[0]->sm_count;
    if (stream) {
        gr->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&gr->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(RLT2_E_CUDA);
        gr->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&gr->done, cudaEventDisableTiming) != cudaSuccess)
        return fail(RLT2_E_CUDA);
    if (make_side(gr->side) != RLT2_OK) return fail(RLT2_E_CUDA);
    int maxN = 0;
    bool pack = true;
    for (rlt2_ctx *c : gr->ctxs) {
        maxN = std::max(maxN, c->node.N);
        pack = pack && c->g.pack;
    }
    const int JC = p1_chunk(maxN, ctxs[0]->g.sym, ctxs[0]->g.paired);
    const std::vector<int4> tri = triple_table(maxN);
    Arena a;
    const size_t o_nodes = a.take((size_t)count * sizeof(NodeDesc));
    const size_t o_tri = a.take(tri.size() * sizeof(int4));
    const size_t o_cnt = a.take(8);
    const size_t o_st = a.take(sizeof(DevStatus));
    const size_t o_snap = a.take(3 * sizeof(DevStatus));
    cudaError_t e = cudaMalloc((void **)&gr->mem, a.used);
    if (e != cudaSuccess) {
        cudaGetLastError();
        gr->mem = nullptr;
        return fail(cuda_code(e));
    }
    // instances with N <= 16 first: their D->C units form a range of their own
    // when the group also has larger instances
    std::vector<int> order(count);
    for (int b = 0; b < count; b++) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (gr->ctxs[x]->node.N <= kSmallN) > (gr->ctxs[y]->node.N <= kSmallN);
    });
    std::vector<NodeDesc> hn(count);
    long long tiles = 0, small_tiles = 0, dtiles = 0;
    int ctas = 0, probs = 0, maxTS = 0, smallTS = 4, smallW = 4;
    for (int b = 0; b < count; b++) {
        NodeDesc &nd = hn[b];
        nd = gr->ctxs[order[b]]->node;     // the context's own state, shared
        fill_node(nd, nd.N, JC);           // the group's location chunk
        encode_zmap(nd, JC);
        nd.tile_base = tiles;
        nd.dtile_base = dtiles;
        dtiles += nd.dtiles;
        nd.cta_base = ctas;
        nd.prob_base = probs;
        tiles += nd.tiles;
        ctas += (int)(n_triples(nd.N) * nd.nchunks);
        probs += nd.N * nd.N;
        maxTS = std::max(maxTS, nd.TS);
        if (nd.N <= kSmallN) {
            small_tiles += nd.dtiles;
            smallTS = std::max(smallTS, nd.TS);
            smallW = std::max(smallW, nd.W);
        }
    }
    if (tiles >= (1LL << 31)) return fail(RLT2_E_INVAL);
    Group &g = gr->g;
    g.small_tiles = small_tiles < dtiles ? (int)small_tiles : 0;
    g.smallTS = smallTS;
    g.smallW = smallW;
    g.nodes = reinterpret_cast<const NodeDesc *>(gr->mem + o_nodes);
    g.B = count;
    g.tiles = tiles;
    g.ctas = ctas;
    g.probs = probs;
    g.maxN = maxN;
    g.maxTS = maxTS;
    g.JC = JC;
    g.pack = pack;
    g.rlt1_only = ctxs[0]->g.rlt1_only;
    g.sym = ctxs[0]->g.sym;
    g.paired = ctxs[0]->g.paired;
    g.dtiles = dtiles;
    g.counter = reinterpret_cast<unsigned *>(gr->mem + o_cnt);
    g.status = reinterpret_cast<DevStatus *>(gr->mem + o_st);
    g.snap = reinterpret_cast<DevStatus *>(gr->mem + o_snap);
    g.triples = reinterpret_cast<const int4 *>(gr->mem + o_tri);
    g.first = hn[0];
    // groups take the remembered shape or the default and do not tune: a
    // server rebuilds its group whenever membership changes, often sooner
    // than tuning would end
    const int rc_shape = setup_dshape(g, ctxs[0]->opts, nullptr);
    if (rc_shape != RLT2_OK) return fail(rc_shape);
    // the group's stream starts after every context's pending work
    for (rlt2_ctx *c : gr->ctxs) {
        if (cudaEventRecord(gr->done, c->stream) != cudaSuccess ||
            cudaStreamWaitEvent(gr->stream, gr->done, 0) != cudaSuccess)
            return fail(RLT2_E_CUDA);
    }
    e = cudaMemcpyAsync(gr->mem + o_nodes, hn.data(), (size_t)count * sizeof(NodeDesc),
                        cudaMemcpyHostToDevice, gr->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(gr->mem + o_tri, tri.data(), tri.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, gr->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.status, 0, sizeof(DevStatus), gr->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.counter, 0, 8, gr->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(gr->stream);  // host copies are on the stack
    if (e != cudaSuccess) return fail(cuda_code(e));
    *out = gr;
    return RLT2_OK;
}

int rlt2_group_iterate(rlt2_group *gr, int k)
{
    if (!gr || k < 0) return RLT2_E_INVAL;
    for (rlt2_ctx *c : gr->ctxs)
        if ((long long)c->enqueued + k > c->opts.max_iters) return RLT2_E_STATE;
    if (k == 0) return RLT2_OK;
    if (!gr->exec) CK(capture_passes(gr->g, gr->sm_count, gr->stream, 1, &gr->graph, &gr->exec, &gr->side));
    for (int t = 0; t < k; t++) CK(cudaGraphLaunch(gr->exec, gr->stream));
    for (rlt2_ctx *c : gr->ctxs) c->enqueued += k;
    // every context's later work starts after the group's passes
    CK(cudaEventRecord(gr->done, gr->stream));
    for (rlt2_ctx *c : gr->ctxs) CK(cudaStreamWaitEvent(c->stream, gr->done, 0));
    return RLT2_OK;
}

int rlt2_group_sync(rlt2_group *gr)
{
    if (!gr) return RLT2_E_INVAL;
    return group_status(gr->g, gr->stream);
}

void rlt2_group_destroy(rlt2_group *gr) { free_group(gr); }

// ----------------------------------------------------- branch-and-bound nodes

int rlt2_subproblem(const int32_t *F, const int32_t *D, int N, int k, const int32_t *fac,
                    const int32_t *loc, int32_t *Fp, int32_t *Dp, int32_t *Blin, int64_t *lb_const)
{
    if (!F || !D || N < 1 || N > RLT2_MAX_N || k < 0 || k > N || (k > 0 && (!fac || !loc)) ||
        !Fp || !Dp || !Blin || !lb_const)
        return RLT2_E_INVAL;
    std::vector<char> ffix(N, 0), lfix(N, 0);
    for (int t = 0; t < k; t++) {
        if (fac[t] < 0 || fac[t] >= N || loc[t] < 0 || loc[t] >= N || ffix[fac[t]] || lfix[loc[t]])
            return RLT2_E_INVAL;
        ffix[fac[t]] = lfix[loc[t]] = 1;
    }
    std::vector<int> fr, lr;  // free facilities, free locations (ascending)
    for (int a = 0; a < N; a++)
        if (!ffix[a]) fr.push_back(a);
    for (int l = 0; l < N; l++)
        if (!lfix[l]) lr.push_back(l);
    const int Np = N - k;
    long long c0 = 0;
    for (int t = 0; t < k; t++)
        for (int t2 = 0; t2 < k; t2++)
            if (t != t2) c0 += (long long)F[fac[t] * N + fac[t2]] * D[loc[t] * N + loc[t2]];
    for (int x = 0; x < Np; x++)
        for (int y = 0; y < Np; y++) {
            Fp[x * Np + y] = F[fr[x] * N + fr[y]];
            Dp[x * Np + y] = D[lr[x] * N + lr[y]];
            // facility fr[x] at location lr[y] against every fixed pair, both directions
            long long b = 0;
            for (int t = 0; t < k; t++)
                b += (long long)F[fr[x] * N + fac[t]] * D[lr[y] * N + loc[t]] +
                     (long long)F[fac[t] * N + fr[x]] * D[loc[t] * N + lr[y]];
            if (b > 0x7fffffffLL) return RLT2_E_OVERFLOW;
            Blin[x * Np + y] = (int32_t)b;
        }
    *lb_const = c0;
    return RLT2_OK;
}

int rlt2_batch_bound(const int32_t *F, const int32_t *D, int N, const rlt2_node *nodes, int B,
                     int iters, const rlt2_opts *opts, int64_t *lb_out, double *ms_out, int *shape_out)
{
    if (!F || !D || N < RLT2_MIN_N || N > RLT2_MAX_N || !nodes || B < 1 || iters < 0 || !lb_out)
        return RLT2_E_INVAL;
    rlt2_opts o;
    if (opts) o = *opts;
    else rlt2_default_opts(&o);
    if (o.rlt1_only) return RLT2_E_INVAL;  // the batch runs the full RLT2 dual ascent
    if (!lanes_opt_ok(o)) return RLT2_E_INVAL;
    int dev = 0, sm_count = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));

    // residual instance of every node (host)
    struct Inst {
        int Np;
        std::vector<int32_t> F, D, B;
        long long cst;
    };
    std::vector<Inst> in(B);
    int maxN = 0;
    bool pack = true;
    for (int b = 0; b < B; b++) {
        const int k = nodes[b].k;
        if (k < 0 || N - k < RLT2_MIN_N) return RLT2_E_INVAL;
        Inst &I = in[b];
        I.Np = N - k;
        const size_t nn = (size_t)I.Np * I.Np;
        I.F.resize(nn);
        I.D.resize(nn);
        I.B.resize(nn);
        int64_t cst = 0;
        int rc = rlt2_subproblem(F, D, N, k, nodes[b].fac, nodes[b].loc, I.F.data(), I.D.data(),
                                 I.B.data(), &cst);
        if (rc != RLT2_OK) return rc;
        I.cst = cst;
        long long U = 0;
        rc = check_instance(I.F.data(), I.D.data(), I.Np, I.B.data(), &U);
        if (rc != RLT2_OK) return rc;
        pack = pack && 3 * U < (1LL << 25);
        maxN = std::max(maxN, I.Np);
    }
    if (o.store != RLT2_STORE_TILES && o.store != RLT2_STORE_CLASSES && o.store != RLT2_STORE_PAIRS)
        return RLT2_E_INVAL;
    const int JC = p1_chunk(maxN, o.store == RLT2_STORE_CLASSES, o.store == RLT2_STORE_PAIRS);
    const int hist_cap = std::max(iters, 1);

    // one allocation for the whole group
    Arena a;
    std::vector<NodeOffsets> no(B);
    const bool sym = o.store == RLT2_STORE_CLASSES, paired = o.store == RLT2_STORE_PAIRS;
    for (int b = 0; b < B; b++) no[b] = plan_node(a, in[b].Np, true, o.store, hist_cap);
    const std::vector<int4> tri = triple_table(maxN);
    const size_t o_nodes = a.take((size_t)B * sizeof(NodeDesc));
    const size_t o_tri = a.take(tri.size() * sizeof(int4));
    const size_t o_cnt = a.take(8);
    const size_t o_st = a.take(sizeof(DevStatus));
    const size_t o_snap = a.take(3 * sizeof(DevStatus));
    const size_t o_stage = a.take((size_t)3 * maxN * maxN * 4 * B);
    // stream capture needs a stream other than the legacy default one
    cudaStream_t s = (cudaStream_t)o.stream;
    cudaStream_t own = nullptr;
    if (!s) {
        CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        s = own;
    }
    char *base = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, a.used);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (own) cudaStreamDestroy(own);
        return cuda_code(e);
    }
    std::vector<NodeDesc> hn(B);
    Group g{};
    long long tiles = 0;
    long long all_tiles = 0;
    for (int b = 0; b < B; b++) all_tiles += make_geom(in[b].Np).tiles;
    if (all_tiles >= (1LL << 31)) {  // tile indices of a group are 32-bit
        cudaFree(base);
        if (own) cudaStreamDestroy(own);
        return RLT2_E_INVAL;
    }
    // nodes with N' <= 16 first: their D->C units form a range of their own
    std::vector<int> order(B);
    for (int b = 0; b < B; b++) order[b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return (in[x].Np <= kSmallN) > (in[y].Np <= kSmallN); });
    int ctas = 0, probs = 0, maxTS = 0, smallTS = 4, smallW = 4;
    long long small_tiles = 0, dtiles = 0;
    for (int b = 0; b < B; b++) {
        NodeDesc &nd = hn[b];
        const int ob = order[b];
        nd.paired = paired;
        fill_node(nd, in[ob].Np, JC);
        nd.p = node_state(base, no[ob], hist_cap, o);
        encode_zmap(nd, JC);
        if (nd.N <= kSmallN) {
            small_tiles += nd.dtiles;
            smallTS = std::max(smallTS, nd.TS);
            smallW = std::max(smallW, nd.W);
        }
        nd.tile_base = tiles;
        nd.dtile_base = dtiles;
        dtiles += nd.dtiles;
        nd.cta_base = ctas;
        nd.prob_base = probs;
        tiles += nd.tiles;
        ctas += (int)(n_triples(nd.N) * nd.nchunks);
        probs += nd.N * nd.N;
        maxTS = std::max(maxTS, nd.TS);
    }
    g.nodes = reinterpret_cast<const NodeDesc *>(base + o_nodes);
    g.B = B;
    g.tiles = tiles;
    g.ctas = ctas;
    g.probs = probs;
    g.maxN = maxN;
    g.maxTS = maxTS;
    g.JC = JC;
    g.pack = pack;
    g.rlt1_only = false;
    g.sym = sym;
    g.paired = paired;
    g.dtiles = dtiles;
    g.small_tiles = small_tiles < dtiles ? (int)small_tiles : 0;
    g.smallTS = smallTS;
    g.smallW = smallW;
    g.counter = reinterpret_cast<unsigned *>(base + o_cnt);
    g.status = reinterpret_cast<DevStatus *>(base + o_st);
    g.snap = reinterpret_cast<DevStatus *>(base + o_snap);
    g.triples = reinterpret_cast<const int4 *>(base + o_tri);
    g.first = hn[0];
    // D->C shapes: opts.lanes / opts.cta_warps force the shape of both
    // ranges, 0 lets the first passes decide (tuning passes, below)
    DlapTuner tuner;
    const int rc_shape = setup_dshape(g, o, &tuner);
    if (rc_shape != RLT2_OK) {
        cudaFree(base);
        if (own) cudaStreamDestroy(own);
        return rc_shape;
    }

    cudaEvent_t t0 = nullptr, t1 = nullptr;
    SideStream side{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = RLT2_OK;
    do {
        if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) break;
        if (make_side(side) != RLT2_OK) {
            e = cudaErrorUnknown;
            break;
        }
        if ((e = cudaMemcpyAsync(base + o_nodes, hn.data(), (size_t)B * sizeof(NodeDesc),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(base + o_tri, tri.data(), tri.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            break;
        if ((e = cudaMemsetAsync(g.status, 0, sizeof(DevStatus), s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(g.counter, 0, 8, s)) != cudaSuccess) break;
        if ((e = cudaEventRecord(t0, s)) != cudaSuccess) break;
        int32_t *stage = reinterpret_cast<int32_t *>(base + o_stage);
        for (int b = 0; b < B && e == cudaSuccess; b++) {
            const Inst &I = in[order[b]];
            e = init_node(hn[b], I.F.data(), I.D.data(), I.B.data(), I.cst, stage + (size_t)b * 3 * maxN * maxN, s);
        }
        if (e != cudaSuccess) break;
        // tuning passes first (real passes), then every remaining pass of
        // every node: one captured graph, one launch
        int done = 0;
        for (; done < iters && tuner.active(); done++) {
            rc = tune_step(g, tuner, sm_count, s, nullptr);
            if (rc != RLT2_OK) break;
        }
        if (rc != RLT2_OK) break;
        if (iters > done) {
            if ((e = capture_passes(g, sm_count, s, iters - done, &graph, &exec, &side)) != cudaSuccess) break;
            if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) break;
        }
        if (shape_out) {
            for (int r = 0; r < 2; r++) {
                shape_out[2 * r] = range_empty(g, r) ? 0 : g.dshape[r].lanes;
                shape_out[2 * r + 1] = dlap_cta_warps(g, r);
            }
        }
        if ((e = cudaEventRecord(t1, s)) != cudaSuccess) break;
        rc = group_status(g, s);
        for (int b = 0; b < B && e == cudaSuccess; b++)
            e = cudaMemcpyAsync(&lb_out[order[b]], hn[b].p.LB, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && ms_out) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, t0, t1);
            *ms_out = ms;
        }
    } while (0);
    if (e != cudaSuccess) rc = cuda_code(e);
    cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    free_side(side);
    cudaFree(base);
    if (own) cudaStreamDestroy(own);
    return rc;
}

// ------------------------------------------------------------------ LAP batch

int rlt2_selftest_timeout(unsigned polls, void *stream)
{
    if (polls == 0) return RLT2_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus *st = nullptr;
    CK(cudaMallocAsync((void **)&st, sizeof(DevStatus), s));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = launch_wait_selftest(st, polls, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_code(e);
    return (err & kDevTimeout) ? RLT2_E_TIMEOUT : RLT2_OK;
}

int rlt2_lap_batch_auction(const int32_t *M, int n, int count, int64_t *S, int32_t *assign, int64_t *work,
                           void *stream)
{
    if (n < 1 || n > 64 || count < 0 || (count > 0 && (!M || !S))) return RLT2_E_INVAL;
    if (count == 0) return RLT2_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus *st = nullptr;
    CK(cudaMallocAsync((void **)&st, sizeof(DevStatus), s));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = launch_auction_batch(M, n, count, S, assign, work, st, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_code(e);
    if (err & kDevInternal) return RLT2_E_INTERNAL;
    return (err & kDevRange) ? RLT2_E_INVAL : RLT2_OK;
}

int rlt2_lap_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign, int32_t *u,
                   int32_t *v, int64_t *work, void *stream)
{
    if (n < 1 || n > 64 || count < 0 || (count > 0 && (!M || !S))) return RLT2_E_INVAL;
    if (count == 0) return RLT2_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus *st = nullptr;
    CK(cudaMallocAsync((void **)&st, sizeof(DevStatus), s));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = launch_lap_batch(M, n, count, S, assign, u, v, work, st, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_code(e);
    if (err & kDevInternal) return RLT2_E_INTERNAL;
    return (err & kDevRange) ? RLT2_E_INVAL : RLT2_OK;
}

}  // extern "C"
