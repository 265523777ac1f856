// Time-domain form: Eq. (1) evaluated term by term on the CUDA cores, followed by |y|^2.
//
// This is the paper's naive TDFIR (Sec. 3.1.1, 8NK operations per filter, Table 1), kept
// for the filter-length comparison against overlap-save.  One block of 256 threads owns a
// tile of 2048 consecutive outputs of one template; thread t owns outputs b0 + 8t + r
// (r = 0..7) and slides an 8-value window of the input through registers, so each tap
// costs one shared-memory load of the input, one broadcast load of the tap and 8 complex
// multiply-adds.  The input tile is stored with one pad slot per 8 values so that the
// 8-value stride between threads does not hit the same banks.
#include <cuda_runtime.h>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"

namespace fdas {

namespace td {
constexpr int THREADS = 256, R = 8, TILE = THREADS * R;   // 2048 outputs per block
constexpr int KCHUNK = 8;                                   // taps per unrolled step
__host__ __device__ inline int skew(int j) { return j + (j >> 3); }
}  // namespace td

// xs holds x[b0 - (KP - 1) - 8 .. b0 + TILE), KP = K rounded up to a multiple of 8 (zero taps).
__global__ void __launch_bounds__(td::THREADS)
    td_direct_kernel(const float2 *__restrict__ x, int64_t n, const float2 *__restrict__ h, int K, int KP,
                     float *__restrict__ out)
{
    using namespace td;
    extern __shared__ float2 td_smem[];
    const int z = blockIdx.y;
    const int64_t b0 = (int64_t)blockIdx.x * TILE;
    const int span = TILE + KP - 1 + 8;           // input values of this tile (+8 leading zeros)
    float2 *xs = td_smem;                         // skew(span) entries
    float2 *hs = td_smem + skew(span) + 1;        // KP taps
    const int64_t first = b0 - (KP - 1) - 8;      // global index of xs[0]
    for (int j = threadIdx.x; j < span; j += THREADS) {
        const int64_t g = first + j;
        xs[skew(j)] = (g >= 0 && g < n) ? x[g] : make_float2(0.f, 0.f);
    }
    for (int k = threadIdx.x; k < KP; k += THREADS) hs[k] = k < K ? h[(size_t)z * K + k] : make_float2(0.f, 0.f);
    __syncthreads();

    // output i = b0 + 8t + r needs x[i - k] = xs[8t + r - k + KP - 1 + 8]
    const int base = R * threadIdx.x + KP - 1 + 8;
    float2 w[R], acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        w[r] = xs[skew(base + r)];                // window for k = 0
        acc[r] = make_float2(0.f, 0.f);
    }
    for (int k0 = 0; k0 < KP; k0 += KCHUNK) {
#pragma unroll
        for (int kk = 0; kk < KCHUNK; ++kk) {
            const int k = k0 + kk;
            const float2 hk = hs[k];
            // the window holds x[i_r - k] in w[(r - kk) mod 8] after kk shifts of this chunk
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 xv = w[(r - kk + R) % R];
                acc[r].x = fmaf(xv.x, hk.x, fmaf(-xv.y, hk.y, acc[r].x));
                acc[r].y = fmaf(xv.x, hk.y, fmaf(xv.y, hk.x, acc[r].y));
            }
            // shift: the slot of w that held x[i_7 - k] now takes x[i_0 - k - 1]
            w[(R - 1 - kk + R) % R] = xs[skew(base - k - 1)];
        }
    }
    float *orow = out + (size_t)z * (size_t)n;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = b0 + R * threadIdx.x + r;
        if (i < n) orow[i] = cabs2(acc[r]);
    }
}

size_t td_smem_bytes(int KP)
{
    const int span = td::TILE + KP - 1 + 8;
    return sizeof(float2) * (td::skew(span) + 1 + KP);
}

cudaError_t launch_td_direct(const float2 *x, int64_t n, const float2 *h, int M, int K, float *out, cudaStream_t s)
{
    const int KP = (K + td::KCHUNK - 1) / td::KCHUNK * td::KCHUNK;
    const size_t smem = td_smem_bytes(KP);
    cudaError_t e = cudaFuncSetAttribute(td_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((n + td::TILE - 1) / td::TILE), M);
    td_direct_kernel<<<grid, td::THREADS, smem, s>>>(x, n, h, K, KP, out);
    return cudaGetLastError();
}

}  // namespace fdas
