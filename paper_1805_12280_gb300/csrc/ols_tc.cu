// Tensor-core form of the overlap-save segment kernel (L = 2048).
//
// Same work item, TMA segment load, template prefetch and forward FFT as the FP32 kernel.
// Per template, the inverse FFT's radix-16 pass B' (over k2) is a dense DFT-matrix GEMM on the
// 5th-generation tensor cores: D[128 x 32] = A[128 x 32] . W[32 x 32], the complex 16-point
// inverse DFT written as a real 32 x 32 matrix, A = the 128 sub-transform rows of one
// template's data in fp16 (written by the threads into shared memory), W split into fp16 hi +
// lo parts (two MMAs per K-step recover the DFT matrix to ~2^-22), FP32 accumulation in tensor
// memory.  The product with H_z, the radix-8 pass C', the twiddles, the last radix-16 pass A'
// (packed FP32x2 butterflies), the discard and |y|^2 stay on the CUDA cores in FP32, so each
// template's data is rounded to fp16 once.  B' uses W/16 (an exact power of 2 that keeps the
// MMA operands' products far from the fp16 range limit); the B' twiddles carry the factor 16.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"
#include "fft_split.cuh"
#include "ols_common.cuh"
#include "ptx.cuh"
#include "tmem.cuh"

namespace fdas {

namespace tc {

constexpr int L = 2048, NT = 128, Q = 16, R = 8, LD2 = NT + 1;
// A operand [128 rows x 32 fp16], K-major, no swizzle: core matrices of 8 rows x 16 bytes;
// LBO = stride between core matrices along K, SBO = stride between 8-row groups.
constexpr uint32_t A_LBO = 160, A_SBO = 640;            // padded: conflict-free A' writes
constexpr uint32_t A_BYTES = 16 * A_SBO;                // 10240
// B operand (the DFT matrix) [32 rows (n) x 32 fp16 (k)], K-major, no swizzle.
constexpr uint32_t B_LBO = 128, B_SBO = 512, B_BYTES = 4 * B_SBO;   // 2048 per matrix
constexpr uint32_t W_BYTES = 2 * B_BYTES;               // B' hi, B' lo
constexpr uint32_t H_BYTES = sizeof(float2) * L;
// TMEM columns: D of B' [0, 32), this thread's segment spectrum [32, 64), C' twiddles
// [64, 96) and B' twiddles (times 16) [96, 128), kept there instead of registers.
constexpr uint32_t TMEM_COLS = 128, COL_DB = 0, COL_X = 32, COL_TW1 = 64, COL_TW2 = 96;
// kind::f16, D = F32, A = B = F16, both K-major, N = 32, M = 128
constexpr uint32_t IDESC = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// 53.5 KB per block, so that four blocks share an SM: the segment buffer is the forward FFT's
// first exchange and then the A operand of B'; one template buffer, refilled one ahead.
struct Smem {
    static constexpr size_t e1 = 0;                                  // segment / exchange 1 / A of B'
    static constexpr size_t e2 = e1 + sizeof(float2) * L;            // exchange 2 (forward, A')
    static constexpr size_t hb = e2 + sizeof(float2) * 16 * LD2;     // template buffer
    static constexpr size_t wm = hb + H_BYTES;                       // B' hi, B' lo
    static constexpr size_t bar = wm + W_BYTES;                     // [0] segment+W, [1] template, [2] B' MMA
    static constexpr size_t slot = bar + 3 * 8;                      // TMEM address
    static constexpr size_t total = 128 + slot + 16;
    static_assert(sizeof(float2) * L >= A_BYTES, "A operand fits the segment buffer");
    static_assert(hb % 128 == 0 && wm % 16 == 0, "bulk copy alignment");
};

__host__ __device__ inline uint32_t a_off(int r, int k)
{
    return (uint32_t)((r >> 3) * A_SBO + (k >> 3) * A_LBO + (r & 7) * 16 + (k & 7) * 2);
}
__host__ __device__ inline uint32_t b_off(int n, int k)
{
    return (uint32_t)((n >> 3) * B_SBO + (k >> 3) * B_LBO + (n & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld_f32(uint32_t taddr, float (&f)[32])
{
    uint32_t r[32];
    tmem_ld32(taddr, r);
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void st_h2(unsigned char *base, uint32_t off, float re, float im)
{
    const __half2 h = __floats2half2_rn(re, im);
    *reinterpret_cast<__half2 *>(base + off) = h;
}

// The real 32 x 32 inverse-DFT matrix of pass B' (times 1/16) as fp16 hi and lo parts,
// written once per plan in the B-operand layout.
__global__ void tc_matrix_kernel(unsigned char *out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (n, k)
    if (idx >= 32 * 32) return;
    const int n = idx / 32, k = idx % 32;
    const int b = n >> 1, ro = n & 1, kk = k >> 1, ri = k & 1;
    double s, c;
    sincospi(2.0 * (double)((kk * b) & 15) / 16.0, &s, &c);   // inverse 16-point DFT, exp(+2 pi i kk b / 16)
    const double scale = 1.0 / 16.0;
    // real form of (re_in + i im_in) * (c + i s): out_re = re c - im s, out_im = re s + im c
    double w;
    if (ro == 0) w = ri == 0 ? c : -s;
    else w = ri == 0 ? s : c;
    w *= scale;
    const __half hi = __double2half(w);
    const __half lo = __double2half(w - (double)__half2float(hi));
    __half *base = reinterpret_cast<__half *>(out);
    base[b_off(n, k) / 2] = hi;
    base[(B_BYTES + b_off(n, k)) / 2] = lo;
}

}  // namespace tc

#ifndef FDAS_TC_MINB
#define FDAS_TC_MINB 4
#endif
__global__ void __launch_bounds__(128, FDAS_TC_MINB)
    ols_tc_kernel(const __grid_constant__ CUtensorMap tmap, const OlsArgs a, const unsigned char *__restrict__ wmat)
{
    using namespace tc;
    constexpr int MASK = L - 1;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float2 *e1 = reinterpret_cast<float2 *>(sm + Smem::e1);
    float2 *e2 = reinterpret_cast<float2 *>(sm + Smem::e2);
    float4 *hb = reinterpret_cast<float4 *>(sm + Smem::hb);
    unsigned char *wm = sm + Smem::wm;
    unsigned char *aB = sm + Smem::e1;   // A operand of B' (the segment buffer, free after the forward FFT)
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Smem::bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + Smem::slot);

    const int tid = threadIdx.x, warp = tid >> 5, k1 = tid & 15, hi = tid >> 4;
    const int seg = a.seg_begin + blockIdx.x;
    const int z0 = blockIdx.y * a.G, z1 = min(z0 + a.G, a.M);

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(L * sizeof(float2)) + W_BYTES);
        const int c0 = seg * a.S - (a.K - 1);
#pragma unroll
        for (int j = 0; j < L / 256; ++j) tma_load_1d(e1 + 256 * j, &tmap, c0 + 256 * j, &bar[0]);
        bulk_load(wm, wmat, W_BYTES, &bar[0]);
        if (z0 < z1) {
            mbar_arrive_expect_tx(&bar[1], H_BYTES);
            bulk_load(hb, a.H + (size_t)z0 * 8 * NT, H_BYTES, &bar[1]);
        }
    }
    // Inverse twiddles, fixed for this thread: C' output conj W_{QR}^{c k2} and B' output
    // 16 conj W_L^{(bR + c) k1} (the 16 undoes the W/16 of the B' matrices), parked in TMEM.
    const uint32_t my = tmem + ((uint32_t)(warp * 32) << 16);
    {
        float2 tw[16];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int k2 = hi + 8 * g;
#pragma unroll
            for (int c = 0; c < R; ++c) tw[g * R + c] = cconj(__ldg(&a.tw[(16 * c * k2) & MASK]));
        }
        tmem_st_split16(my + COL_TW1, tw);   // split pairs (c, R + c)
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            const float2 w = __ldg(&a.tw[((b * R + hi) * k1) & MASK]);
            tw[b] = make_float2(16.f * w.x, -16.f * w.y);
        }
        tmem_st_c16(my + COL_TW2, tw);
    }

    const bool seg_ok = __syncthreads_and(mbar_wait_bounded(&bar[0], 0, kWaitLimitNs));
    bool ok = seg_ok;
    uint32_t h_uses = 0, h_iss = z0 < z1, b_uses = 0, b_done = 0;
    float2 v[16];
    if (ok) {
        float2 X[16];
        forward_fft<L>(e1, e2, a.tw, v, X);
        tmem_st_split16(my + COL_X, X);   // the spectrum waits in TMEM (split pairs) for the template loop
        __syncthreads();              // e1 is read: it becomes the A operand of B'
    }
    const int64_t seg_out = (int64_t)seg * a.S;
    const int64_t nvalid64 = a.n - seg_out;
    const unsigned nvalid = (unsigned)(nvalid64 < a.S ? nvalid64 : a.S);
    const int obase = tid - (a.K - 1);
    unsigned vmask = 0;   // bit j: register slot j of this thread holds a kept output
#pragma unroll
    for (int j = 0; j < 16; ++j) vmask |= ((unsigned)(j * NT + obase) < nvalid ? 1u : 0u) << j;
    const uint32_t aB_addr = smem_u32(aB), w_addr = smem_u32(wm);

    for (int z = z0; ok && z < z1; ++z) {
        const bool h_ok = mbar_wait_bounded(&bar[1], h_uses & 1, kWaitLimitNs);
        h_uses++;
        // ---- product with H_z, pass C' (radix 8), twiddle, fp16 rows of the B' operand
        // (both pass-C' groups as split pairs: packed FP32x2 product, DFTs and twiddles)
        {
            float2 re[8], im[8];
            {
                uint32_t xr[32];
                tmem_ld32(my + COL_X, xr);
                split_from_cols(xr, re, im);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 h = hb[c * NT + tid];
                cmul_split(re[c], im[c], make_float2(h.x, h.y), make_float2(h.z, h.w));
            }
            dft8x2_split<1>(re, im);
            {
                uint32_t t1r[32];
                tmem_ld32(my + COL_TW1, t1r);
                float2 twr[8], twi[8];
                split_from_cols(t1r, twr, twi);
#pragma unroll
                for (int c = 1; c < 8; ++c) cmul_split(re[c], im[c], twr[c], twi[c]);
            }
#pragma unroll
            for (int c = 0; c < R; ++c) {   // row (k1, c), K pairs k2 = hi and hi + 8
                st_h2(aB, a_off(k1 + 16 * c, 2 * hi), re[c].x, im[c].x);
                st_h2(aB, a_off(k1 + 16 * c, 2 * (hi + 8)), re[c].y, im[c].y);
            }
        }
        fence_proxy_async_smem();
        fence_before_sync();
        if (!__syncthreads_and(h_ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            fence_after_sync();
            // every thread has read the template buffer: refill it with the next template
            if (z + 1 < z1) {
                h_iss++;
                mbar_arrive_expect_tx(&bar[1], H_BYTES);
                bulk_load(hb, a.H + (size_t)(z + 1) * 8 * NT, H_BYTES, &bar[1]);
            }
            // ---- pass B': D_B = A_B . (W_hi + W_lo) / 16 over K = 32 (two K-steps)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = smem_desc(aB_addr + ks * 2 * A_LBO, A_LBO, A_SBO);
                mma_f16(tmem + COL_DB, ad, smem_desc(w_addr + ks * 2 * B_LBO, B_LBO, B_SBO), ks);
                mma_f16(tmem + COL_DB, ad, smem_desc(w_addr + B_BYTES + ks * 2 * B_LBO, B_LBO, B_SBO), 1);
            }
            mma_commit(&bar[2]);
        }
        const bool mb_ok = mbar_wait_bounded(&bar[2], b_uses & 1, kWaitLimitNs);
        b_uses++;
        b_done += mb_ok;
        fence_after_sync();
        // ---- B' output row tid = (k1, c = hi): b = 0..15, twiddle, exchange to A'
        {
            float f[32];
            tmem_ld_f32(my + COL_DB, f);
            float2 tw2[16];
            tmem_ld_c16(my + COL_TW2, tw2);
#pragma unroll
            for (int b = 0; b < Q; ++b) e2[(b * R + hi) + LD2 * k1] = cmul(make_float2(f[2 * b], f[2 * b + 1]), tw2[b]);
        }
        fence_before_sync();   // the TMEM reads of D_B precede the next B' MMA
        if (!__syncthreads_and(mb_ok)) {
            ok = false;
            break;
        }
        fence_after_sync();
        // ---- pass A': 16-point IDFT over k1 -> natural order y[a*NT + t], power, stores
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = e2[tid + LD2 * k];
        dft<16, 1>(v);
        float *orow = a.out + (size_t)z * (size_t)a.n + seg_out;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (vmask & (1u << j)) orow[j * NT + obase] = cabs2(v[j]);
    }
    if (!ok && tid == 0) {   // give outstanding copies and MMAs a bounded time to land
        atomicOr(a.status, STATUS_WAIT_TIMEOUT);
        if (!seg_ok) mbar_wait_bounded(&bar[0], 0, kWaitLimitNs);
        if (h_iss > h_uses) mbar_wait_bounded(&bar[1], h_uses & 1, kWaitLimitNs);
        if (b_done < b_uses) mbar_wait_bounded(&bar[2], (b_uses - 1) & 1, kWaitLimitNs);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

cudaError_t launch_tc_matrices(unsigned char *wmat, cudaStream_t s)
{
    tc::tc_matrix_kernel<<<(32 * 32 + 255) / 256, 256, 0, s>>>(wmat);
    return cudaGetLastError();
}

size_t tc_matrix_bytes() { return tc::W_BYTES; }

cudaError_t launch_ols_tc(const CUtensorMap *tmap, const OlsArgs &a, const unsigned char *wmat, int nseg,
                          cudaStream_t s)
{
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !done[dev]) {
        e = cudaFuncSetAttribute(ols_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::Smem::total);
        if (e == cudaSuccess)   // four blocks per SM need the largest shared-memory carveout
            e = cudaFuncSetAttribute(ols_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    dim3 grid(nseg, (a.M + a.G - 1) / a.G);
    ols_tc_kernel<<<grid, 128, tc::Smem::total, s>>>(*tmap, a, wmat);
    return cudaGetLastError();
}

}  // namespace fdas
