// Failure-detection self-test: a bounded mbarrier wait that runs out on purpose, reported
// through the plan's status word exactly as a segment kernel reports a lost copy.
//
// The probe block arms an mbarrier for 16 bytes of transaction that no copy will ever
// deliver (no copy is issued at all, so nothing is in flight when the block leaves), waits
// with the kernels' own bounded wait, and on expiry sets STATUS_WAIT_TIMEOUT; the context
// stays usable and fdas_plan_status returns FDAS_ERR_TIMEOUT once.
#include <cuda_runtime.h>

#include "fdas_internal.cuh"
#include "ptx.cuh"

namespace fdas {

__global__ void wait_timeout_probe(int *status, uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);   // a phase that cannot complete
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, STATUS_WAIT_TIMEOUT);
}

}  // namespace fdas

extern "C" int fdas_selftest_wait_timeout(fdas_plan p, double limit_ms, void *stream)
{
    if (!p) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null plan");
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) return fdas::set_error(FDAS_ERR_INVALID_ARG, "limit_ms outside (0, 1000]");
    int prev = -1;
    cudaGetDevice(&prev);
    const int dev = fdas::plan_device(p);
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return fdas::set_error(FDAS_ERR_CUDA, "cannot select plan device");
    fdas::wait_timeout_probe<<<1, 32, 0, (cudaStream_t)stream>>>(fdas::plan_status_word(p),
                                                                (uint64_t)(limit_ms * 1e6));
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return fdas::set_error(FDAS_ERR_CUDA, cudaGetErrorString(e));
    return FDAS_OK;
}
