// Full-length frequency-domain FIR (Eq. 2): y_z = IFFT_P(FFT_P(x) . FFT_P(h_z)) with P >= n + K - 1
// a power of two, then |y_z|^2 for i < n -- the "naive" FD-FIR that the paper weighs against
// overlap-save (Sec. 3.2.1, Table 1), kept to measure that choice on this GPU.
//
// P-point transforms in four steps, P = P1 * P2 with P1 = 2048 and P2 in {1024, 2048, 4096}:
//   n = P2 n1 + n2,  k = k1 + P1 k2,
//   X[k1 + P1 k2] = sum_n2 W_P2^{n2 k2} W_P^{n2 k1} sum_n1 x[P2 n1 + n2] W_P1^{n1 k1}.
// Column pass: the P1-point FFTs over n1 (stride P2), four columns per block staged in shared
// memory, then the twiddle W_P^{n2 k1}; row pass: the P2-point FFTs over n2 (contiguous).
// Spectra stay in the register-slot orders of the two in-block FFTs (row r = j*NT1 + t holds
// k1 of slot j of thread t; likewise the columns): the product needs only the same order for x
// and h, and the inverse runs the passes backwards to natural order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <new>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"
#include "ols_common.cuh"

namespace fdas {

namespace fd {
constexpr int P1 = 2048, NT1 = P1 / 16, TB = 4, TBP = TB + 1;   // tile rows padded to 5 values
constexpr size_t col_smem_bytes()
{
    return sizeof(float2) * ((size_t)P1 * TBP + P1 + 16 * (NT1 + 1));
}
template <int P2>
constexpr size_t row_smem_bytes()
{
    return sizeof(float2) * ((size_t)P2 + 16 * (P2 / 16 + 1));
}

// exp(dir * 2 pi i e / P), e < P <= 2^23 (the argument 2e/P is exact in FP32)
__device__ __forceinline__ float2 twiddle_p(int e, float two_over_p, float dir)
{
    float s, c;
    sincospif(dir * (float)e * two_over_p, &s, &c);
    return make_float2(c, s);
}
}  // namespace fd

// Column pass, forward: columns n2 = blockIdx.x * TB + t of in[P2 n1 + n2] (zero at and beyond
// len) -> A[r][n2] = scale * W_P^{n2 k1} * FFT_P1 over n1, row r = j*NT1 + t for slot j of t.
template <int P2>
__global__ void __launch_bounds__(fd::NT1) fdfir_col_fwd(const float2 *__restrict__ in, int64_t len,
                                                        const float2 *__restrict__ tw1, float2 *__restrict__ A,
                                                        float scale)
{
    using namespace fd;
    extern __shared__ float2 fd_smem[];
    float2 *tile = fd_smem, *e1 = tile + (size_t)P1 * TBP, *e2 = e1 + P1;
    const int tid = threadIdx.x, n2_0 = blockIdx.x * TB;
    constexpr float two_over_p = 2.0f / ((float)P1 * (float)P2);
    for (int idx = tid; idx < P1 * TB; idx += NT1) {
        const int n1 = idx / TB, t = idx % TB;
        const int64_t e = (int64_t)P2 * n1 + n2_0 + t;
        tile[n1 * TBP + t] = e < len ? in[e] : make_float2(0.f, 0.f);
    }
    for (int t = 0; t < TB; ++t) {
        __syncthreads();   // tile loaded; the previous column's exchanges are read
#pragma unroll
        for (int m = 0; m < 16; ++m) e1[m * NT1 + tid] = tile[(m * NT1 + tid) * TBP + t];
        __syncthreads();
        float2 v[16], X[16];
        forward_fft<P1>(e1, e2, tw1, v, X);
        const int n2 = n2_0 + t;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k1 = freq_of_slot(P1, tid, j);
            const float2 w = twiddle_p(n2 * k1, two_over_p, -1.f);   // n2 k1 < 2^23
            const float2 y = cmul(X[j], w);
            tile[(j * NT1 + tid) * TBP + t] = make_float2(scale * y.x, scale * y.y);
        }
    }
    __syncthreads();
    for (int idx = tid; idx < P1 * TB; idx += NT1) {
        const int r = idx / TB, t = idx % TB;
        A[(size_t)r * P2 + n2_0 + t] = tile[r * TBP + t];
    }
}

// Row pass, forward, in place: row blockIdx.x of A (natural order over n2) -> its P2-point
// spectrum, column c = j*NT2 + t for slot j of thread t.
template <int P2>
__global__ void __launch_bounds__(P2 / 16) fdfir_row_fwd(float2 *__restrict__ A, const float2 *__restrict__ tw2)
{
    constexpr int NT2 = P2 / 16;
    extern __shared__ float2 fd_smem[];
    float2 *e1 = fd_smem, *e2 = e1 + P2;
    const int tid = threadIdx.x;
    float2 *row = A + (size_t)blockIdx.x * P2;
#pragma unroll
    for (int m = 0; m < 16; ++m) e1[m * NT2 + tid] = row[m * NT2 + tid];
    __syncthreads();
    float2 v[16], X[16];
    forward_fft<P2>(e1, e2, tw2, v, X);   // every read of the row precedes its barriers
#pragma unroll
    for (int j = 0; j < 16; ++j) row[j * NT2 + tid] = X[j];
}

// Row pass, inverse, with the product: B[r][n2] = IFFT_P2 over k2 of X[r][.] * H[r][.].
template <int P2>
__global__ void __launch_bounds__(P2 / 16) fdfir_row_inv(const float2 *__restrict__ X, const float2 *__restrict__ H,
                                                         float2 *__restrict__ B, const float2 *__restrict__ tw2)
{
    constexpr int NT2 = P2 / 16;
    extern __shared__ float2 fd_smem[];
    float2 *e1 = fd_smem, *e2 = e1 + P2;
    const int tid = threadIdx.x;
    const size_t off = (size_t)blockIdx.x * P2;
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = cmul(__ldg(&X[off + j * NT2 + tid]), __ldg(&H[off + j * NT2 + tid]));
    inverse_fft<P2>(v, e1, e2, tw2);
#pragma unroll
    for (int a = 0; a < 16; ++a) B[off + a * NT2 + tid] = v[a];
}

// Column pass, inverse, with the power: out[P2 n1 + n2] = |IFFT_P1 over k1 of
// W_P^{-n2 k1} B[r(k1)][n2]|^2 for P2 n1 + n2 < n.
template <int P2>
__global__ void __launch_bounds__(fd::NT1) fdfir_col_inv(const float2 *__restrict__ B, const float2 *__restrict__ tw1,
                                                        float *__restrict__ out, int64_t n)
{
    using namespace fd;
    extern __shared__ float2 fd_smem[];
    float2 *tile = fd_smem, *e1 = tile + (size_t)P1 * TBP, *e2 = e1 + P1;
    const int tid = threadIdx.x, n2_0 = blockIdx.x * TB;
    constexpr float two_over_p = 2.0f / ((float)P1 * (float)P2);
    for (int idx = tid; idx < P1 * TB; idx += NT1) {
        const int r = idx / TB, t = idx % TB;
        tile[r * TBP + t] = B[(size_t)r * P2 + n2_0 + t];
    }
    for (int t = 0; t < TB; ++t) {
        __syncthreads();   // tile loaded; the previous column's exchanges are read
        const int n2 = n2_0 + t;
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k1 = freq_of_slot(P1, tid, j);
            v[j] = cmul(tile[(j * NT1 + tid) * TBP + t], twiddle_p(n2 * k1, two_over_p, 1.f));
        }
        inverse_fft<P1>(v, e1, e2, tw1);
#pragma unroll
        for (int a = 0; a < 16; ++a) {
            const int64_t i = (int64_t)P2 * (a * NT1 + tid) + n2;
            if (i < n) out[i] = cabs2(v[a]);
        }
    }
}

template <int P2>
static cudaError_t fdfir_attrs()
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fdfir_col_fwd<P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fd::col_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fdfir_col_inv<P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fd::col_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fdfir_row_fwd<P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fd::row_smem_bytes<P2>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fdfir_row_inv<P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fd::row_smem_bytes<P2>());
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// Forward P-point transform of in[0, len) (zero-padded) into A, times scale.
template <int P2>
static cudaError_t fdfir_forward_l(const float2 *in, int64_t len, const float2 *tw1, const float2 *tw2, float2 *A,
                                   float scale, cudaStream_t s)
{
    cudaError_t e = fdfir_attrs<P2>();
    if (e != cudaSuccess) return e;
    fdfir_col_fwd<P2><<<P2 / fd::TB, fd::NT1, fd::col_smem_bytes(), s>>>(in, len, tw1, A, scale);
    fdfir_row_fwd<P2><<<fd::P1, P2 / 16, fd::row_smem_bytes<P2>(), s>>>(A, tw2);
    return cudaGetLastError();
}

// Inverse transform of X . H into the power row out[0, n).
template <int P2>
static cudaError_t fdfir_inverse_l(const float2 *X, const float2 *H, float2 *B, const float2 *tw1, const float2 *tw2,
                                   float *out, int64_t n, cudaStream_t s)
{
    cudaError_t e = fdfir_attrs<P2>();
    if (e != cudaSuccess) return e;
    fdfir_row_inv<P2><<<fd::P1, P2 / 16, fd::row_smem_bytes<P2>(), s>>>(X, H, B, tw2);
    fdfir_col_inv<P2><<<P2 / fd::TB, fd::NT1, fd::col_smem_bytes(), s>>>(B, tw1, out, n);
    return cudaGetLastError();
}

cudaError_t fdfir_forward(int P2, const float2 *in, int64_t len, const float2 *tw1, const float2 *tw2, float2 *A,
                          float scale, cudaStream_t s)
{
    switch (P2) {
    case 1024: return fdfir_forward_l<1024>(in, len, tw1, tw2, A, scale, s);
    case 2048: return fdfir_forward_l<2048>(in, len, tw1, tw2, A, scale, s);
    case 4096: return fdfir_forward_l<4096>(in, len, tw1, tw2, A, scale, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fdfir_inverse(int P2, const float2 *X, const float2 *H, float2 *B, const float2 *tw1, const float2 *tw2,
                          float *out, int64_t n, cudaStream_t s)
{
    switch (P2) {
    case 1024: return fdfir_inverse_l<1024>(X, H, B, tw1, tw2, out, n, s);
    case 2048: return fdfir_inverse_l<2048>(X, H, B, tw1, tw2, out, n, s);
    case 4096: return fdfir_inverse_l<4096>(X, H, B, tw1, tw2, out, n, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fdas

// ---- C ABI -------------------------------------------------------------------------------

struct fdas_fdfir_s {
    int device = -1;
    int64_t n_max = 0, P = 0;
    int M = 0, K = 0, P2 = 0;
    float2 *d_H = nullptr;      // [M][P] template spectra / P (slot orders of the two passes)
    float2 *d_X = nullptr;      // [P] input spectrum
    float2 *d_B = nullptr;      // [P] row-pass output of the inverse
    float2 *d_tw1 = nullptr;    // [P1] W_P1, FP32 from FP64
    float2 *d_tw2 = nullptr;    // [P2] W_P2
    double2 *d_tw64 = nullptr;  // FP64 twiddle scratch
};

namespace {

void fdfir_free(fdas_fdfir f)
{
    if (!f) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(f->device);
    cudaFree(f->d_H);
    cudaFree(f->d_X);
    cudaFree(f->d_B);
    cudaFree(f->d_tw1);
    cudaFree(f->d_tw2);
    cudaFree(f->d_tw64);
    if (prev >= 0) cudaSetDevice(prev);
    delete f;
}

int fdfir_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return fdas::set_error(e == cudaErrorMemoryAllocation ? FDAS_ERR_OOM : FDAS_ERR_CUDA, buf);
}

}  // namespace

extern "C" {

int fdas_fdfir_create(fdas_fdfir *out, int64_t n_max, const void *templates, int M, int K)
{
    if (!out) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (!templates) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null templates");
    if (M < 1 || K < 1) return fdas::set_error(FDAS_ERR_INVALID_ARG, "n_templates and tpl_len must be >= 1");
    if (n_max < 1) return fdas::set_error(FDAS_ERR_INVALID_ARG, "n_max must be >= 1");
    int64_t P = int64_t(1) << 21;
    while (P < n_max + K - 1) P <<= 1;
    if (P > (int64_t(1) << 23)) return fdas::set_error(FDAS_ERR_INVALID_ARG, "n_max + tpl_len - 1 exceeds 2^23");
    fdas_fdfir f = new (std::nothrow) fdas_fdfir_s;
    if (!f) return fdas::set_error(FDAS_ERR_OOM, "host allocation");
    if (cudaGetDevice(&f->device) != cudaSuccess) {
        delete f;
        return fdas::set_error(FDAS_ERR_CUDA, "no current CUDA device");
    }
    f->n_max = n_max;
    f->P = P;
    f->M = M;
    f->K = K;
    f->P2 = (int)(P / fdas::fd::P1);
    cudaError_t e;
    float2 *d_h = nullptr;
    const size_t h_bytes = sizeof(float2) * (size_t)M * K;
    int rc = FDAS_OK;
    if ((e = cudaMalloc(&f->d_H, sizeof(float2) * (size_t)M * P)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc spectra");
    else if ((e = cudaMalloc(&f->d_X, sizeof(float2) * P)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc input spectrum");
    else if ((e = cudaMalloc(&f->d_B, sizeof(float2) * P)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc scratch");
    else if ((e = cudaMalloc(&f->d_tw1, sizeof(float2) * fdas::fd::P1)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc twiddles");
    else if ((e = cudaMalloc(&f->d_tw2, sizeof(float2) * f->P2)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc twiddles");
    else if ((e = cudaMalloc(&f->d_tw64, sizeof(double2) * std::max(fdas::fd::P1, f->P2))) != cudaSuccess)
        rc = fdfir_cuda(e, "cudaMalloc twiddles");
    else if ((e = cudaMalloc(&d_h, h_bytes)) != cudaSuccess) rc = fdfir_cuda(e, "cudaMalloc template staging");
    else if ((e = cudaMemcpy(d_h, templates, h_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) rc = fdfir_cuda(e, "copy templates");
    else if ((e = fdas::launch_twiddles(fdas::fd::P1, f->d_tw64, f->d_tw1, nullptr)) != cudaSuccess) rc = fdfir_cuda(e, "twiddles");
    else if ((e = fdas::launch_twiddles(f->P2, f->d_tw64, f->d_tw2, nullptr)) != cudaSuccess) rc = fdfir_cuda(e, "twiddles");
    for (int z = 0; rc == FDAS_OK && z < M; ++z) {
        e = fdas::fdfir_forward(f->P2, d_h + (size_t)z * K, K, f->d_tw1, f->d_tw2, f->d_H + (size_t)z * P,
                                1.0f / (float)P, nullptr);
        if (e != cudaSuccess) rc = fdfir_cuda(e, "template transforms");
    }
    if (rc == FDAS_OK && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = fdfir_cuda(e, "plan-time kernels");
    cudaFree(d_h);
    if (rc != FDAS_OK) {
        fdfir_free(f);
        return rc;
    }
    *out = f;
    return FDAS_OK;
}

int fdas_fdfir_length(fdas_fdfir f, int64_t *P)
{
    if (!f || !P) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null argument");
    *P = f->P;
    return FDAS_OK;
}

int fdas_fdfir_convolve(fdas_fdfir f, const void *in, int64_t n, float *out, void *stream)
{
    if (!f) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in || !out) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null input or output pointer");
    if (n < 1 || n > f->n_max) return fdas::set_error(FDAS_ERR_INVALID_ARG, "n outside [1, n_max]");
    if (reinterpret_cast<uintptr_t>(in) % 8 || reinterpret_cast<uintptr_t>(out) % 4)
        return fdas::set_error(FDAS_ERR_INVALID_ARG, "misaligned input or output pointer");
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), i1 = i0 + (uintptr_t)n * 8;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(out), o1 = o0 + (uintptr_t)n * 4 * (uintptr_t)f->M;
    if (i0 < o1 && o0 < i1) return fdas::set_error(FDAS_ERR_INVALID_ARG, "input and output overlap");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != f->device && cudaSetDevice(f->device) != cudaSuccess)
        return fdas::set_error(FDAS_ERR_CUDA, "cannot select plan device");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = fdas::fdfir_forward(f->P2, static_cast<const float2 *>(in), n, f->d_tw1, f->d_tw2, f->d_X, 1.0f, s);
    for (int z = 0; e == cudaSuccess && z < f->M; ++z)
        e = fdas::fdfir_inverse(f->P2, f->d_X, f->d_H + (size_t)z * f->P, f->d_B, f->d_tw1, f->d_tw2,
                                out + (size_t)z * n, n, s);
    if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fdfir_cuda(e, "full-length FD-FIR launch");
    return FDAS_OK;
}

int fdas_fdfir_destroy(fdas_fdfir f)
{
    if (!f) return fdas::set_error(FDAS_ERR_INVALID_ARG, "null plan");
    fdfir_free(f);
    return FDAS_OK;
}

}  // extern "C"
