// api.cu -- the C ABI declared in include/rlt2.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rlt2.h"
#include "device.cuh"
#include "kernels.h"

using namespace rlt2;

struct rlt2_ctx {
    Geom g;
    rlt2_opts opts;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int *z = nullptr, *yS = nullptr, *yC = nullptr, *x = nullptr;
    long long *LB = nullptr, *hist = nullptr;
    int *iter = nullptr, *stop = nullptr;
    unsigned *counter = nullptr;
    DevStatus *status = nullptr;
    int4 *triples = nullptr;
    int ntriples = 0;
    PassState ps{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int enqueued = 0;
    // profiling: 5 events per pass, recorded on the stream between the stages
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
};

static int cuda_code(cudaError_t e)
{
    if (e == cudaSuccess) return RLT2_OK;
    if (e == cudaErrorMemoryAllocation) return RLT2_E_OOM;
    return RLT2_E_CUDA;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_code(e_); \
    } while (0)

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
    default: return "unknown error";
    }
}

int rlt2_row_stride(int N) { return (N + 3) & ~3; }

static void free_ctx(rlt2_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    cudaFree(c->z);
    cudaFree(c->yS);
    cudaFree(c->yC);
    cudaFree(c->x);
    cudaFree(c->LB);
    cudaFree(c->hist);
    cudaFree(c->iter);
    cudaFree(c->stop);
    cudaFree(c->counter);
    cudaFree(c->status);
    cudaFree(c->triples);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

void rlt2_destroy(rlt2_ctx *c) { free_ctx(c); }

// U bounds Q(pi) - LB for every permutation pi; every reduced cost lies on some
// pi and all are >= 0, so every cost and every class sum is <= U.
static long long guard_U(const int32_t *F, const int32_t *D, int N, const int32_t *B)
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

int rlt2_create(const int32_t *F, const int32_t *D, int N, const int32_t *B_lin, int64_t lb_const,
                const rlt2_opts *opts, rlt2_ctx **out)
{
    if (!out) return RLT2_E_INVAL;
    *out = nullptr;
    if (!F || !D || N < RLT2_MIN_N || N > RLT2_MAX_N) return RLT2_E_INVAL;
    for (int e = 0; e < N * N; e++)
        if (F[e] < 0 || D[e] < 0 || (B_lin && B_lin[e] < 0)) return RLT2_E_INVAL;
    const long long U = guard_U(F, D, N, B_lin);
    if (U > RLT2_LAP_MAX_ENTRY) return RLT2_E_OVERFLOW;

    rlt2_ctx *c = new (std::nothrow) rlt2_ctx();
    if (!c) return RLT2_E_OOM;
    if (opts) c->opts = *opts;
    else rlt2_default_opts(&c->opts);
    if (c->opts.max_iters <= 0) c->opts.max_iters = 65536;
    c->g = make_geom(N);
    const Geom &g = c->g;

    int rc = RLT2_OK;
    auto fail = [&](int code) {
        free_ctx(c);
        return code;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(RLT2_E_CUDA);
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(RLT2_E_CUDA);
    if (c->opts.stream) {
        c->stream = (cudaStream_t)c->opts.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(RLT2_E_CUDA);
        c->own_stream = true;
    }
    auto A = [&](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = cuda_code(e);
            return false;
        }
        return true;
    };
    const size_t nt = (size_t)g.tiles;
    if (!c->opts.rlt1_only && !A((void **)&c->z, nt * g.TS * 4)) return fail(rc);
    if (!A((void **)&c->yS, nt * 4) || !A((void **)&c->yC, nt * 4) ||
        !A((void **)&c->x, (size_t)N * N * 4) || !A((void **)&c->LB, 8) ||
        !A((void **)&c->hist, (size_t)c->opts.max_iters * 8) || !A((void **)&c->iter, 4) ||
        !A((void **)&c->stop, 4) || !A((void **)&c->counter, 4) ||
        !A((void **)&c->status, sizeof(DevStatus)))
        return fail(rc);

    std::vector<int4> tri;
    for (int i = 0; i < N; i++)
        for (int k = i + 1; k < N; k++)
            for (int p = k + 1; p < N; p++) tri.push_back(make_int4(i, k, p, 0));
    c->ntriples = (int)tri.size();
    if (!A((void **)&c->triples, tri.size() * sizeof(int4))) return fail(rc);
    if (cudaMemcpy(c->triples, tri.data(), tri.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return fail(RLT2_E_CUDA);

    PassState &p = c->ps;
    p.z = c->z;
    p.yS = c->yS;
    p.yC = c->yC;
    p.x = c->x;
    p.LB = c->LB;
    p.hist = c->hist;
    p.iter = c->iter;
    p.stop = c->stop;
    p.counter = c->counter;
    p.status = c->status;
    p.hist_cap = c->opts.max_iters;
    p.ub = c->opts.ub;
    p.min_progress = c->opts.min_progress;
    p.pack = 3 * U < (1LL << 25);
    p.rlt1_only = c->opts.rlt1_only != 0;

    // inputs to the device, then the initialisation of Algorithm 1
    int32_t *dF = nullptr, *dD = nullptr, *dB = nullptr;
    if (!A((void **)&dF, (size_t)N * N * 4) || !A((void **)&dD, (size_t)N * N * 4) ||
        (B_lin && !A((void **)&dB, (size_t)N * N * 4))) {
        cudaFree(dF);
        cudaFree(dD);
        return fail(rc);
    }
    cudaError_t e = cudaMemcpyAsync(dF, F, (size_t)N * N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dD, D, (size_t)N * N * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && B_lin)
        e = cudaMemcpyAsync(dB, B_lin, (size_t)N * N * 4, cudaMemcpyHostToDevice, c->stream);
    long long lb0 = lb_const;
    if (e == cudaSuccess) e = launch_init(g, p, dF, dD, dB, lb0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dF);
    cudaFree(dD);
    cudaFree(dB);
    if (e != cudaSuccess) return fail(cuda_code(e));
    *out = c;
    return RLT2_OK;
}

// One pass of Algorithm 1: fused spread/complementary pass over D, D -> C,
// complementary C + C -> B, B -> LB.  ev: 5 events to record around the stages.
static cudaError_t enqueue_pass(rlt2_ctx *c, cudaEvent_t *ev)
{
    const Geom &g = c->g;
    const PassState &p = c->ps;
    cudaError_t e;
    auto mark = [&](int s) { return ev ? cudaEventRecord(ev[s], c->stream) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    if (!c->opts.rlt1_only) {
        if ((e = launch_p1(g, p, c->triples, c->ntriples, c->stream)) != cudaSuccess) return e;
        if ((e = mark(1)) != cudaSuccess) return e;
        if ((e = launch_dlap(g, p, c->sm_count, c->stream)) != cudaSuccess) return e;
    } else if ((e = mark(1)) != cudaSuccess) {
        return e;
    }
    if ((e = mark(2)) != cudaSuccess) return e;
    if ((e = launch_clap(g, p, c->stream)) != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    if ((e = launch_xlap(g, p, c->stream)) != cudaSuccess) return e;
    return mark(4);
}

static cudaError_t build_graph(rlt2_ctx *c)
{
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue_pass(c, nullptr);
    e = cudaStreamEndCapture(c->stream, &c->graph);
    if (e2 != cudaSuccess) return e2;
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&c->gexec, c->graph, 0);
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
        if (c->opts.use_graph && !ev) {
            if (!c->gexec) CK(build_graph(c));
            CK(cudaGraphLaunch(c->gexec, c->stream));
        } else {
            CK(enqueue_pass(c, ev));   // profiling launches stage by stage
        }
        c->enqueued++;
    }
    return RLT2_OK;
}

static int check_status(rlt2_ctx *c)
{
    int err = 0;
    CK(cudaMemcpyAsync(&err, &c->status->err, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (err & kDevTimeout) return RLT2_E_TIMEOUT;
    if (err & kDevInternal) return RLT2_E_INTERNAL;
    return RLT2_OK;
}

int rlt2_bound(rlt2_ctx *c, double *lb, int64_t *lb_exact, int *iters)
{
    if (!c) return RLT2_E_INVAL;
    long long v = 0;
    int it = 0;
    CK(cudaMemcpyAsync(&v, c->LB, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&it, c->iter, 4, cudaMemcpyDeviceToHost, c->stream));
    int rc = check_status(c);
    if (lb) *lb = (double)v;
    if (lb_exact) *lb_exact = v;
    if (iters) *iters = it;
    return rc;
}

int rlt2_bound_history(rlt2_ctx *c, int64_t *out, int cap, int *count)
{
    if (!c || (!out && cap > 0) || cap < 0) return RLT2_E_INVAL;
    int it = 0;
    CK(cudaMemcpyAsync(&it, c->iter, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int n = std::min(std::min(it, cap), c->opts.max_iters);
    if (n > 0) CK(cudaMemcpy(out, c->hist, (size_t)n * 8, cudaMemcpyDeviceToHost));
    if (count) *count = n;
    return RLT2_OK;
}

int rlt2_get_state(rlt2_ctx *c, int level, int32_t *host, size_t count)
{
    if (!c || !host) return RLT2_E_INVAL;
    const Geom &g = c->g;
    const int N = g.N;
    if (level == 0) {
        if (count != (size_t)N * N) return RLT2_E_INVAL;
        CK(cudaMemcpyAsync(host, c->x, count * 4, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 1) {
        if (count != (size_t)g.tiles) return RLT2_E_INVAL;
        CK(cudaMemcpyAsync(host, c->yC, count * 4, cudaMemcpyDeviceToHost, c->stream));
    } else if (level == 2) {
        if (!c->z || count != (size_t)g.tiles * g.n * g.n) return RLT2_E_INVAL;
        // the store's rows are indexed by location: drop the tile's own two
        // locations (and the padding) to reach the compact layout
        std::vector<int32_t> tmp;
        try {
            tmp.resize((size_t)g.tiles * g.TS);
        } catch (...) {
            return RLT2_E_OOM;
        }
        CK(cudaMemcpyAsync(tmp.data(), c->z, tmp.size() * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const int m = N - 1, n = g.n, W = g.W;
        size_t o = 0;
        for (long long t = 0; t < g.tiles; t++) {
            const int nn = (int)(t % m), j = (int)((t / ((long long)m * m)) % N);
            const int nl = nn + (nn >= j);
            const int32_t *src = tmp.data() + (size_t)t * g.TS;
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

int rlt2_work(rlt2_ctx *c, int64_t out[6])
{
    if (!c || !out) return RLT2_E_INVAL;
    DevStatus s;
    CK(cudaMemcpyAsync(&s, c->status, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
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
    for (size_t b = 0; b + 5 <= c->ev_used; b += 5) {
        const int map[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}};
        for (int s = 0; s < 4; s++) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->events[b + map[s][0]], c->events[b + map[s][1]]));
            acc[s] += ms;
        }
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
    case 0: return c->x;
    case 1: return c->yC;
    case 2: return c->z;
    default: return nullptr;
    }
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
