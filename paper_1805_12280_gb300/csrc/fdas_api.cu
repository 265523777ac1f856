// Host plan layer and C ABI (see include/fdas.h for the contract of each entry point).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "fdas_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? FDAS_ERR_OOM : FDAS_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define FDAS_CUDA_TRY(call, what)                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (g_encode_err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

// 1-D tiled tensor map over n complex64 values (8-byte elements), 256-element boxes.
int encode_input_map(CUtensorMap *map, const void *in, int64_t n)
{
    auto enc = tensor_map_encoder();
    if (!enc) return fail(FDAS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(g_encode_err));
    cuuint64_t dims[1] = {(cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)n * 8};   // unused for rank 1
    cuuint32_t box[1] = {256};
    cuuint32_t estr[1] = {1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 1, const_cast<void *>(in), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FDAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return FDAS_OK;
}

constexpr int kMaxChunks = 8;

}  // namespace

struct fdas_plan_s {
    int device = -1;
    int64_t n_max = 0;
    int M = 0, K_user = 0, K = 0, L = 0, S = 0, G = 0, precision = 0;
    float2 *d_tw = nullptr;     // [L] FP32 twiddles
    double2 *d_tw64 = nullptr;  // [L] FP64 twiddles
    float4 *d_H = nullptr;      // [M][8][L/16] pre-transformed templates
    int *d_status = nullptr;
    int64_t device_bytes = 0;
    // host-buffer entry point
    std::mutex host_mu;
    void *d_in_stage = nullptr;
    float *d_out_stage = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_ev[kMaxChunks] = {};
};

namespace {

void plan_free(fdas_plan p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    cudaFree(p->d_tw);
    cudaFree(p->d_tw64);
    cudaFree(p->d_H);
    cudaFree(p->d_status);
    cudaFree(p->d_in_stage);
    cudaFree(p->d_out_stage);
    for (auto &e : p->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    delete p;
}

int validate_convolve(fdas_plan p, const void *in, int64_t n, const float *out)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in || !out) return fail(FDAS_ERR_INVALID_ARG, "null input or output pointer");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(FDAS_ERR_INVALID_ARG, "input pointer must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out) % 4) return fail(FDAS_ERR_INVALID_ARG, "output pointer must be 4-byte aligned");
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), i1 = i0 + (uintptr_t)n * 8;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(out), o1 = o0 + (uintptr_t)n * 4 * (uintptr_t)p->M;
    if (i0 < o1 && o0 < i1) return fail(FDAS_ERR_INVALID_ARG, "input and output overlap");
    return FDAS_OK;
}

int64_t n_segments(const fdas_plan p, int64_t n) { return (n + p->S - 1) / p->S; }

int enqueue_segments(fdas_plan p, const CUtensorMap *map, int64_t n, float *out, int64_t s0, int64_t s1,
                     cudaStream_t stream)
{
    fdas::OlsArgs a;
    a.H = p->d_H;
    a.tw = p->d_tw;
    a.out = out;
    a.n = n;
    a.M = p->M;
    a.G = p->G;
    a.S = p->S;
    a.K = p->K;
    a.seg_begin = (int)s0;
    a.status = p->d_status;
    cudaError_t e = fdas::launch_ols_fp32(p->L, map, a, (int)(s1 - s0), stream);
    if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch");
    return FDAS_OK;
}

}  // namespace

extern "C" {

const char *fdas_version(void) { return "fdas-gb300 0.1 (sm_103a)"; }

const char *fdas_strerror(int code)
{
    switch (code) {
    case FDAS_OK: return "ok";
    case FDAS_ERR_INVALID_ARG: return "invalid argument";
    case FDAS_ERR_OOM: return "out of memory";
    case FDAS_ERR_CUDA: return "CUDA error";
    case FDAS_ERR_TIMEOUT: return "timed out";
    case FDAS_ERR_BUSY: return "busy";
    case FDAS_ERR_REJECTED: return "rejected";
    case FDAS_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown error";
    }
}

const char *fdas_last_error(void) { return g_last_error.c_str(); }

int fdas_plan_create(fdas_plan *out, int64_t n_max, const void *templates, int M, int K, const fdas_opts *opts)
{
    if (!out) return fail(FDAS_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    fdas_opts o = {};
    if (opts) o = *opts;
    const int L = o.seg_len ? o.seg_len : 2048;
    if (L != 1024 && L != 2048 && L != 4096) return fail(FDAS_ERR_INVALID_ARG, "seg_len %d not in {1024, 2048, 4096}", L);
    if (o.precision != FDAS_PREC_FP32) return fail(FDAS_ERR_UNSUPPORTED, "precision %d not built", o.precision);
    if (!templates) return fail(FDAS_ERR_INVALID_ARG, "null templates");
    if (M < 1) return fail(FDAS_ERR_INVALID_ARG, "n_templates=%d < 1", M);
    if (K < 1 || K > L - 4) return fail(FDAS_ERR_INVALID_ARG, "tpl_len=%d outside [1, %d]", K, L - 4);
    if (n_max < 1 || n_max > (int64_t(1) << 30)) return fail(FDAS_ERR_INVALID_ARG, "n_max=%lld outside [1, 2^30]", (long long)n_max);
    if (o.tpl_per_cta < 0 || o.tpl_per_cta > M) return fail(FDAS_ERR_INVALID_ARG, "tpl_per_cta=%d outside [0, %d]", o.tpl_per_cta, M);

    fdas_plan p = new (std::nothrow) fdas_plan_s;
    if (!p) return fail(FDAS_ERR_OOM, "host allocation");
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FDAS_ERR_CUDA, "no current CUDA device");
    }
    p->n_max = n_max;
    p->M = M;
    p->K_user = K;
    p->K = (K % 2 == 0) ? K + 1 : K;           // odd frame: segment starts stay 16-byte aligned
    p->L = L;
    p->S = (L - p->K + 1) & ~3;                 // multiple of 4, <= L - K + 1
    p->G = o.tpl_per_cta ? o.tpl_per_cta : M;
    p->precision = o.precision;

    auto cleanup_fail = [&](int code) {
        plan_free(p);
        return code;
    };
    float2 *d_h32 = nullptr;
    const size_t h_bytes = sizeof(float2) * (size_t)M * K;
    const size_t H_bytes = sizeof(float4) * (size_t)M * 8 * (L / 16);
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_tw, sizeof(float2) * L)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc twiddles"));
    if ((e = cudaMalloc(&p->d_tw64, sizeof(double2) * L)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc twiddles64"));
    if ((e = cudaMalloc(&p->d_H, H_bytes)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc templates"));
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc status"));
    if ((e = cudaMalloc(&d_h32, h_bytes)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc template staging"));
    p->device_bytes = (int64_t)(sizeof(float2) * L + sizeof(double2) * L + H_bytes + sizeof(int));

    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_h32, templates, h_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = fdas::launch_twiddles(L, p->d_tw64, p->d_tw, s);
    if (e == cudaSuccess) e = fdas::launch_pretransform(L, d_h32, M, K, p->d_tw64, p->d_H, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (s) cudaStreamDestroy(s);
    cudaFree(d_h32);
    if (e != cudaSuccess) return cleanup_fail(cuda_fail(e, "plan-time kernels"));
    *out = p;
    return FDAS_OK;
}

int fdas_plan_describe(fdas_plan p, fdas_plan_desc *d)
{
    if (!p || !d) return fail(FDAS_ERR_INVALID_ARG, "null argument");
    d->n_max = p->n_max;
    d->n_templates = p->M;
    d->tpl_len = p->K_user;
    d->frame_len = p->K;
    d->seg_len = p->L;
    d->seg_step = p->S;
    d->tpl_per_cta = p->G;
    d->precision = p->precision;
    d->device = p->device;
    d->device_bytes = p->device_bytes;
    return FDAS_OK;
}

int fdas_convolve(fdas_plan p, const void *in, int64_t n, float *out, void *stream)
{
    int rc = validate_convolve(p, in, n, out);
    if (rc) return rc;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    CUtensorMap map;
    if ((rc = encode_input_map(&map, in, n))) return rc;
    return enqueue_segments(p, &map, n, out, 0, n_segments(p, n), (cudaStream_t)stream);
}

int fdas_convolve_host(fdas_plan p, const void *in_host, int64_t n, float *out_host, void *stream)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in_host || !out_host) return fail(FDAS_ERR_INVALID_ARG, "null host pointer");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    std::lock_guard<std::mutex> lk(p->host_mu);
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->d_in_stage) {
        FDAS_CUDA_TRY(cudaMalloc(&p->d_in_stage, sizeof(float2) * (size_t)p->n_max), "cudaMalloc input staging");
        FDAS_CUDA_TRY(cudaMalloc(&p->d_out_stage, sizeof(float) * (size_t)p->n_max * p->M), "cudaMalloc output staging");
        FDAS_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (auto &ev : p->chunk_ev) FDAS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        p->device_bytes += (int64_t)(sizeof(float2) * (size_t)p->n_max + sizeof(float) * (size_t)p->n_max * p->M);
    }
    FDAS_CUDA_TRY(cudaMemcpyAsync(p->d_in_stage, in_host, sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice, s), "H2D input");
    CUtensorMap map;
    int rc = encode_input_map(&map, p->d_in_stage, n);
    if (rc) return rc;
    const int64_t nseg = n_segments(p, n);
    const int chunks = (int)std::min<int64_t>(kMaxChunks, nseg);
    for (int c = 0; c < chunks; ++c) {
        const int64_t s0 = nseg * c / chunks, s1 = nseg * (c + 1) / chunks;
        if ((rc = enqueue_segments(p, &map, n, p->d_out_stage, s0, s1, s))) return rc;
        FDAS_CUDA_TRY(cudaEventRecord(p->chunk_ev[c], s), "event record");
        FDAS_CUDA_TRY(cudaStreamWaitEvent(p->copy_stream, p->chunk_ev[c], 0), "stream wait");
        const int64_t i0 = s0 * p->S, i1 = std::min<int64_t>(s1 * p->S, n);
        FDAS_CUDA_TRY(cudaMemcpy2DAsync(out_host + i0, sizeof(float) * n, p->d_out_stage + i0, sizeof(float) * n,
                                        sizeof(float) * (i1 - i0), p->M, cudaMemcpyDeviceToHost, p->copy_stream),
                      "D2H plane chunk");
    }
    FDAS_CUDA_TRY(cudaStreamSynchronize(p->copy_stream), "copy stream sync");
    FDAS_CUDA_TRY(cudaStreamSynchronize(s), "stream sync");
    return FDAS_OK;
}

int fdas_plan_status(fdas_plan p, void *stream)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    DeviceGuard g(p->device);
    FDAS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    int st = 0;
    FDAS_CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (st) {
        FDAS_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)), "status clear");
        return fail(FDAS_ERR_TIMEOUT, "an in-kernel bounded wait ran out (status 0x%x)", st);
    }
    return FDAS_OK;
}

int fdas_destroy(fdas_plan p)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    plan_free(p);
    return FDAS_OK;
}

}  // extern "C"
