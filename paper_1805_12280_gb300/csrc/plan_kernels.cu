// Plan-time kernels, FP64: twiddle tables and the template pre-transform.
//
// Algorithm 2 transforms the coefficient array once ("Fourier transform of
// coefficient array") and reuses it for every input sub-array; Table 1 leaves this
// one-off cost out because N >> K.  Here each zero-padded template is transformed
// by a direct FP64 DFT (exact integer argument reduction of k*f mod L), scaled by
// 1/L so that the segment kernel's inverse FFT needs no scaling, rounded to FP32 and
// stored in the order the segment kernel holds the forward spectrum in registers.
#include <cuda_runtime.h>

#include "fdas_internal.cuh"

namespace fdas {

// w64[e] = exp(-2 pi i e / L) in FP64; w32 = the same rounded to FP32.
__global__ void twiddle_kernel(int L, double2 *w64, float2 *w32)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L) return;
    double s, c;
    sincospi(-2.0 * (double)e / (double)L, &s, &c);   // argument exact: L is a power of two
    w64[e] = make_double2(c, s);
    w32[e] = make_float2((float)c, (float)s);
}

// One thread per (template z, thread slot tau, register slot j).
__global__ void pretransform_kernel(int L, const float2 *__restrict__ h32, int M, int K,
                                    const double2 *__restrict__ w64, float4 *__restrict__ Hperm, bool split)
{
    const int NT = L / 16;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)M * NT * 16;
    if (id >= total) return;
    const int tau = (int)(id % NT);
    const int j = (int)((id / NT) % 16);
    const int z = (int)(id / ((int64_t)NT * 16));
    const int f = freq_of_slot(L, tau, j);
    const float2 *h = h32 + (size_t)z * K;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < K; ++k) {
        const double2 w = w64[((int64_t)k * f) & (L - 1)];
        const double hr = (double)h[k].x, hi = (double)h[k].y;
        re += hr * w.x - hi * w.y;
        im += hr * w.y + hi * w.x;
    }
    re /= (double)L;
    im /= (double)L;
    if (!split) {   // slots (2p, 2p+1) as two complex values
        float *dst = reinterpret_cast<float *>(Hperm + ((size_t)z * 8 + j / 2) * NT + tau) + 2 * (j & 1);
        dst[0] = (float)re;
        dst[1] = (float)im;
    } else {        // slots (c, 8 + c) as split pairs (re_c, re_{8+c}, im_c, im_{8+c})
        float *dst = reinterpret_cast<float *>(Hperm + ((size_t)z * 8 + (j & 7)) * NT + tau);
        dst[j >> 3] = (float)re;
        dst[2 + (j >> 3)] = (float)im;
    }
}

cudaError_t launch_twiddles(int L, double2 *w64, float2 *w32, cudaStream_t s)
{
    twiddle_kernel<<<(L + 255) / 256, 256, 0, s>>>(L, w64, w32);
    return cudaGetLastError();
}

cudaError_t launch_pretransform(int L, const float2 *h32, int M, int K, const double2 *w64, float4 *Hperm,
                                bool split, cudaStream_t s)
{
    const int64_t total = (int64_t)M * (L / 16) * 16;
    pretransform_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(L, h32, M, K, w64, Hperm, split);
    return cudaGetLastError();
}

}  // namespace fdas
