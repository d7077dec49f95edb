// lap_static.cu -- rlt2_lap_batch_static: the batched Hungarian LAP without any
// device allocation.
//
// rlt2_lap_batch needs a small block of device scratch for each call (the
// status word the kernel raises on bad input, and its work counters) and gets
// it with cudaMallocAsync.  Some callers must not let a library allocate: code
// that hands all device memory to one owning allocator (a framework's caching
// allocator, a memory budget enforced per process), real-time code that cannot
// afford an allocation's latency or failure, or callers that want the call to
// touch nothing but the buffers they pass.  This entry point serves them: its
// scratch is a fixed array in the library's own device memory.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rlt2.h"
#include "device.cuh"
#include "kernels.h"

namespace {

// The whole scratch of a call: one status block (48 bytes).  Each GPU that
// loads the library holds its own copy until the process exits.  Every call on
// that GPU reuses it and it keeps the last call's contents, so each call clears
// it first; two calls whose work overlaps on the GPU share it and race.
static __device__ __align__(256) rlt2::DevStatus g_lap_scratch[1];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
rlt2::DevStatus *g_scratch_addr[kMaxDevices] = {};

// Device address of g_lap_scratch on the current device.  In host code the
// symbol's name is only a host-side handle, so it is resolved once per device
// (with that device current) by cudaGetSymbolAddress and kept for the life of
// the process.  cudaDeviceReset unloads the module and the array may come back
// elsewhere, so a process that resets a device must not call this entry point
// on that device afterwards.
int scratch_on_current_device(rlt2::DevStatus **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RLT2_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return RLT2_E_INVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lap_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RLT2_E_CUDA;
        }
        g_scratch_addr[dev] = static_cast<rlt2::DevStatus *>(p);
    }
    *out = g_scratch_addr[dev];
    return RLT2_OK;
}

}  // namespace

extern "C" int rlt2_lap_batch_static(const int32_t *M, int n, int count, int64_t *S,
                                     int32_t *assign, int32_t *u, int32_t *v, int64_t *work,
                                     void *stream)
{
    if (n < 1 || n > RLT2_LAP_STATIC_MAX_N || count < 0 || (count > 0 && (!M || !S)))
        return RLT2_E_INVAL;
    if (count == 0) return RLT2_OK;
    rlt2::DevStatus *st = nullptr;
    const int rc = scratch_on_current_device(&st);
    if (rc != RLT2_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(rlt2::DevStatus), s);
    if (e == cudaSuccess) e = rlt2::launch_lap_batch(M, n, count, S, assign, u, v, work, st, s);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RLT2_E_OOM : RLT2_E_CUDA;
    if (err & rlt2::kDevInternal) return RLT2_E_INTERNAL;
    return (err & rlt2::kDevRange) ? RLT2_E_INVAL : RLT2_OK;
}
