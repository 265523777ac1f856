// Time-domain form: Eq. (1) evaluated term by term on the CUDA cores, followed by |y|^2.
//
// This is the paper's naive TDFIR (Sec. 3.1.1, 8NK operations per filter, Table 1), kept
// for the filter-length comparison against overlap-save.  One block of 256 threads owns a
// tile of 2048 consecutive outputs of one template; thread t owns outputs b0 + 8t + r
// (r = 0..7) and slides an 8-value window of the input through registers, so each tap
// costs one shared-memory load of the input, one broadcast load of the tap and 8 complex
// multiply-adds (two packed FP32x2 FMAs each).  The input tile is stored with one pad slot
// per 8 values so that the 8-value stride between threads does not hit the same banks.
#include <cuda_runtime.h>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"

namespace fdas {

namespace td {
constexpr int THREADS = 256, R = 8, TILE = THREADS * R;   // 2048 outputs per block
constexpr int KCHUNK = 8;                                   // taps per unrolled step
__host__ __device__ inline int skew(int j) { return j + (j >> 3); }
}  // namespace td

// Packed complex multiply-add: acc += x h as two FP32x2 FMAs,
// acc += (x.x, x.y) * (h.x, h.x) and acc += (x.y, x.x) * (-h.y, h.y), so both operands
// arrive as ready-made pairs: the input tile holds (x.x, x.y, x.y, x.x) per value and the
// taps (h.x, h.x, -h.y, h.y).
__device__ __forceinline__ void cmac2(float2 &acc, float4 x, float4 h)
{
    asm("{\n\t.reg .b64 pa, px, ps, ph, pg;\n\t"
        "mov.b64 pa, {%0, %1};\n\tmov.b64 px, {%2, %3};\n\tmov.b64 ps, {%4, %5};\n\t"
        "mov.b64 ph, {%6, %7};\n\tmov.b64 pg, {%8, %9};\n\t"
        "fma.rn.f32x2 pa, px, ph, pa;\n\tfma.rn.f32x2 pa, ps, pg, pa;\n\t"
        "mov.b64 {%0, %1}, pa;\n\t}"
        : "+f"(acc.x), "+f"(acc.y)
        : "f"(x.x), "f"(x.y), "f"(x.z), "f"(x.w), "f"(h.x), "f"(h.y), "f"(h.z), "f"(h.w));
}

// xs holds x[b0 - (KP - 1) - 8 .. b0 + TILE) as (x.x, x.y, x.y, x.x), KP = K rounded up to
// a multiple of 8 (zero taps); hs the taps as (h.x, h.x, -h.y, h.y).
__global__ void __launch_bounds__(td::THREADS)
    td_direct_kernel(const float2 *__restrict__ x, int64_t n, const float2 *__restrict__ h, int K, int KP,
                     float *__restrict__ out)
{
    using namespace td;
    extern __shared__ float4 td_smem[];
    const int z = blockIdx.y;
    const int64_t b0 = (int64_t)blockIdx.x * TILE;
    const int span = TILE + KP - 1 + 8;           // input values of this tile (+8 leading zeros)
    float4 *xs = td_smem;                         // skew(span) entries
    float4 *hs = td_smem + skew(span) + 1;        // KP taps
    const int64_t first = b0 - (KP - 1) - 8;      // global index of xs[0]
    for (int j = threadIdx.x; j < span; j += THREADS) {
        const int64_t g = first + j;
        const float2 v = (g >= 0 && g < n) ? x[g] : make_float2(0.f, 0.f);
        xs[skew(j)] = make_float4(v.x, v.y, v.y, v.x);
    }
    for (int k = threadIdx.x; k < KP; k += THREADS) {
        const float2 v = k < K ? h[(size_t)z * K + k] : make_float2(0.f, 0.f);
        hs[k] = make_float4(v.x, v.x, -v.y, v.y);
    }
    __syncthreads();

    // output i = b0 + 8t + r needs x[i - k] = xs[8t + r - k + KP - 1 + 8]
    const int base = R * threadIdx.x + KP - 1 + 8;
    float4 w[R];
    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        w[r] = xs[skew(base + r)];                // window for k = 0
        acc[r] = make_float2(0.f, 0.f);
    }
    for (int k0 = 0; k0 < KP; k0 += KCHUNK) {
#pragma unroll
        for (int kk = 0; kk < KCHUNK; ++kk) {
            const int k = k0 + kk;
            const float4 hk = hs[k];
            // the window holds x[i_r - k] in w[(r - kk) mod 8] after kk shifts of this chunk
#pragma unroll
            for (int r = 0; r < R; ++r) cmac2(acc[r], w[(r - kk + R) % R], hk);
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
    return sizeof(float4) * (td::skew(span) + 1 + KP);
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
