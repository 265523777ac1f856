// fdas_convolve_batch_noalloc: the batched form for callers that cannot allocate GPU
// memory at call time (see include/fdas.h).  Its only scratch, the persistent kernel's
// work counters, lives in a file-scope __device__ array instead of plan memory.
#include <cuda_runtime.h>

#include <mutex>

#include "fdas_internal.cuh"

namespace {

// One work counter per kernel launch (one launch per table of kBatchMax arrays):
// at most kNoAllocLaunches * kBatchMax = 7680 arrays per call.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int kNoAllocLaunches = 64;
static __device__ __align__(256) int g_noalloc_counters[kNoAllocLaunches];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_counters_dev[kMaxDevices] = {};   // device address of the array, per device

// Set-up, once per device, with that device current: host code only sees a host-side
// stand-in under the array's name, so the kernel is given the address the runtime reports.
int counters_address(int dev, int **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fdas::set_error(FDAS_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_counters_dev[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_counters);
        if (e != cudaSuccess || !ptr)
            return fdas::set_error(FDAS_ERR_CUDA, "cudaGetSymbolAddress of the work-counter array failed");
        g_counters_dev[dev] = static_cast<int *>(ptr);
    }
    *out = g_counters_dev[dev];
    return FDAS_OK;
}

}  // namespace

extern "C" int fdas_convolve_batch_noalloc(fdas_plan p, int count, const void *const *ins, const int64_t *ns,
                                           float *const *outs, void *stream)
{
    if (!p) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null plan");
    const int dev = fdas::plan_device(p);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fdas::set_error(FDAS_ERR_CUDA, "no current CUDA device");
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
        return fdas::set_error(FDAS_ERR_CUDA, "cannot select the plan's device");
    int *counters = nullptr;
    int rc = counters_address(dev, &counters);
    if (rc == FDAS_OK)
        rc = fdas::batch_direct(p, count, ins, ns, outs, counters, kNoAllocLaunches, (cudaStream_t)stream);
    if (prev != dev) cudaSetDevice(prev);
    return rc;
}
