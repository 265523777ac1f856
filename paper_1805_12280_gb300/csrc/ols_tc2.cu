// Two-stage tensor-core form of the overlap-save segment kernel (L = 2048): the whole inverse
// FFT of every (segment, template) pair is two DFT-matrix GEMMs on the 5th-generation tensor
// cores (Algorithm 2's per-filter IFFT, the M L C log2 L term of Table 1).
//
// Index split (Cooley-Tukey, L = 32 x 64): frequency k = k2 + 64 k1, output n = n1 + 32 n2,
//   y[n] = sum_k2 W64^{n2 k2} [ W2048^{n1 k2} ( sum_k1 W32^{n1 k1} Y[k2 + 64 k1] ) ],
// with W_N^e = exp(+2 pi i e / N) and Y = X . H_z (Eq. 1 through the convolution theorem).
//
//   stage 1  D1[(k2, s)][(n1, re/im)] = A1 . B1: A1 = Y in fp16, one TMEM lane per (k2, segment s)
//            written by the CUDA cores right after the product; B1 = the real 64 x 64 form of
//            the 32-point inverse DFT in shared memory.  M 128, N 64, K 64.
//   twiddle  Z = D1 . W2048^{n1 k2} / 32 on the CUDA cores (packed FP32x2), rounded to fp16 and
//            written MN-major into shared memory: the stage-1 rows become stage-2 columns.
//   stage 2  D2[(n1, s, template)][(n2, re/im)] = Z . G: Z in shared memory (MN-major A operand),
//            G = the real 128 x 128 form of the 64-point inverse DFT (K-major B operand, loaded
//            once per block).  M 128, N 128, K 128: two templates of two segments per MMA.
//   power    one TMEM lane per (n1, segment, template) holds re and im of its 64 outputs
//            n1 + 32 n2: |y|^2 in packed FP32x2, the discard of the first K-1 outputs, and stores
//            in which a warp writes 32 consecutive outputs (128 contiguous bytes) -- or, in the
//            threshold instantiation, the crossings of a threshold as records, no plane.
//
// A work item is a pair of consecutive segments and a range of template pairs (each block an
// equal share of them); a tile is one template of both segments (stage 1), a pair two tiles
// (stage 2).  Roles: warps 0-3 run the forward FFTs (FP32, once per segment) and the products,
// warps 4-7 the twiddles, warps 8-11 the power epilogue, warps 12 and 14 issue the stage-1 and
// stage-2 MMAs, warp 13 the TMA loads.  mbarriers carry the MMA completions, the copies and the
// handoffs of written operands to the MMA warps; named barriers carry the handoffs of read
// accumulators back to them.
//
// Range: the forward spectrum of each segment is scaled by a power of two chosen from its
// largest component (|X| < 2^11) and the templates by one power of two per plan (|H| <= 16),
// so the fp16 operands cannot overflow for any finite input; the powers carry the inverse
// factor, an exact power of two.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"
#include "fft_split.cuh"
#include "ols_common.cuh"
#include "ptx.cuh"
#include "tmem.cuh"

namespace fdas {
namespace tc2 {

constexpr int L = 2048, NT = 128;
constexpr int kThreads = 3 * NT + 96;          // product, twiddle, power groups + 2 MMA warps + loader
constexpr int NH = 4;                          // template buffers in flight
constexpr int CAND_STAGE = 64;                 // threshold crossings staged per power warp
constexpr uint32_t H_ROW = 144;                // bytes per k2 row of a template: 32 half2 + 16 B pad
constexpr uint32_t H_BYTES = 64 * H_ROW;       // 9216 per template
// B1 [N 64 x K 64] fp16, K-major, no swizzle: core matrices 8 rows x 16 B, K step LBO, row-group step SBO.
constexpr uint32_t LBO1 = 128, SBO1 = 1024, B1_BYTES = 8 * SBO1;
// Z [M 128 x K 128] fp16, MN-major, no swizzle: core matrices 8 K-rows x 16 B of M; the
// descriptor's LBO is the step between K groups, SBO the step between M groups.
constexpr uint32_t LBO2 = 2048, SBO2 = 128, B2_BYTES = 16 * LBO2;
// G [N 128 x K 128] fp16, K-major, no swizzle.
constexpr uint32_t LBOG = 128, SBOG = 16 * LBOG, G_BYTES = 16 * SBOG;
// Plan constants: B1 image | G image | twiddles (64 k2 x 64 floats).
constexpr uint32_t CB_B1 = 0, CB_G = CB_B1 + B1_BYTES, CB_TW = CB_G + G_BYTES;
constexpr uint32_t CONST_BYTES = CB_TW + 64 * 64 * 4;
// TMEM columns: A1 x 2, D1 x 3, D2 x 2.
constexpr uint32_t COL_A1 = 0, COL_D1 = 64, COL_D2 = 256, TMEM_COLS = 512;
constexpr uint32_t ND1 = 3;                    // stage-1 accumulators in flight (A1: 2)
// kind::f16, D = F32, A = B = F16, M = 128.  Stage 1: A from TMEM, B K-major, N = 64.
// Stage 2: A MN-major (bit 15), B K-major, N = 128.
constexpr uint32_t IDESC1 = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t IDESC2 = (1u << 4) | (1u << 15) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

// mbarriers
enum : int {
    B_SEG_FULL = 0, B_SEG_FREE, B_B1_FULL,
    B_SCALE0, B_SCALE1, B_SFREE0, B_SFREE1,   // per-item power factors: written / read
    B_H_FULL, B_H_FREE = B_H_FULL + NH,
    B_MMA1 = B_H_FREE + NH, B_MMA2 = B_MMA1 + ND1,   // tcgen05.commit: stage 1 of tile t, stage 2 of pair q
    B_B2F = B_MMA2 + 2,                                  // stage-2 operand of pair q written (128 twiddle threads)
    B_A1W = B_B2F + 2,                                   // stage-1 operand of tile t written (128 product threads)
    B_COUNT = B_A1W + 2
};

struct Smem {
    static constexpr size_t seg = 0;                                  // 2 segments (TMA) / spectra
    static constexpr size_t e2 = seg + 2 * sizeof(float2) * L;         // forward-FFT exchange
    static constexpr size_t hb = e2 + sizeof(float2) * 16 * (NT + 1);  // NH template buffers
    static constexpr size_t b1 = hb + NH * H_BYTES;
    static constexpr size_t g = b1 + B1_BYTES;                        // stage-2 DFT matrix
    static constexpr size_t b2 = g + G_BYTES;                         // 2 stage-2 operand buffers
    static constexpr size_t stage = b2 + 2 * B2_BYTES;                // threshold epilogue: 64 records per power warp
    static constexpr size_t red = stage + 4 * 64 * 16;                // per-warp maxima [4][2]
    static constexpr size_t scale = red + 8 * sizeof(float);          // [2 items][2 segments]
    static constexpr size_t bar = scale + 4 * sizeof(float);
    static constexpr size_t misc = bar + B_COUNT * 8;                 // TMEM address, abort flag
    static constexpr size_t total = 1024 + misc + 16;
    static_assert(e2 % 128 == 0 && hb % 128 == 0 && b1 % 128 == 0 && b2 % 128 == 0, "alignment");
    static_assert(bar % 8 == 0, "mbarrier alignment");
};

struct Args {
    const unsigned char *H16;   // [M even][64][36] half2 per template, times 2^eH
    const unsigned char *cst;   // plan constants (CONST_BYTES)
    const float2 *tw;           // [L] W_L^e = exp(-2 pi i e / L), FP32 (forward FFT)
    int M, S, K;                // templates, segment step, frame length
    int ng, ZP;                 // template-pair groups per segment pair, template pairs
    int eH;                     // template scale exponent
    int *status;
    // threshold epilogue (fdas_convolve_candidates): crossings instead of the plane when cand != null
    fdas_candidate *cand;
    unsigned long long *cand_count;
    long long cand_max;
    float threshold;
};

// A work item: template pairs [zp0, zp1) of segment pair `sp` of one array.
struct Item {
    const CUtensorMap *map;     // the array's input tensor map
    float *out;                 // its plane [M][n]
    int64_t n;
    int seg_begin, nseg;        // the segments [seg_begin, seg_begin + nseg) this launch covers
    int sp, zp0, zp1;
};
// One array (fdas_convolve): the n_sp x ZP (segment pair, template pair) units in order, an
// equal share per block (q units, one more for the first r blocks), cut into items at
// segment-pair boundaries; a segment pair split between two blocks has its forward FFTs done
// by both (the unit count fits 32 bits: the launcher checks it).
struct SingleSrc {
    const CUtensorMap *map;
    float *out;
    int64_t n;
    int seg_begin, nseg, n_sp, ZP;
    int q, r;
    __device__ __forceinline__ unsigned u0() const
    {
        const unsigned b = blockIdx.x;
        return b * (unsigned)q + (b < (unsigned)r ? b : (unsigned)r);
    }
    __device__ __forceinline__ unsigned u1() const { return u0() + (unsigned)q + (blockIdx.x < (unsigned)r ? 1u : 0u); }
    __device__ __forceinline__ int count() const
    {
        const unsigned a0 = u0(), a1 = u1();
        return a1 > a0 ? (int)((a1 - 1) / (unsigned)ZP - a0 / (unsigned)ZP + 1) : 0;
    }
    __device__ __forceinline__ Item item(int k) const
    {
        const unsigned a0 = u0(), a1 = u1();
        const int sp = (int)(a0 / (unsigned)ZP) + k;
        const unsigned b0 = (unsigned)sp * (unsigned)ZP, e0 = b0 + (unsigned)ZP;
        const int zp0 = (int)((a0 > b0 ? a0 : b0) - b0), zp1 = (int)((a1 < e0 ? a1 : e0) - b0);
        return Item{map, out, n, seg_begin, nseg, sp, zp0, zp1};
    }
};
// A short array (a few units per block): items (segment pair, one of ng template-pair groups)
// in turn by block, so that no block's share crosses a segment pair.
struct SingleGroupSrc {
    const CUtensorMap *map;
    float *out;
    int64_t n;
    int seg_begin, nseg, n_sp, ZP, ng;
    __device__ __forceinline__ int count() const
    {
        const unsigned items = (unsigned)n_sp * (unsigned)ng, b = blockIdx.x;
        return b < items ? (int)((items - 1 - b) / gridDim.x + 1) : 0;
    }
    __device__ __forceinline__ Item item(int k) const
    {
        const int it = (int)blockIdx.x + k * (int)gridDim.x, grp = it % ng;
        return Item{map, out, n, seg_begin, nseg, it / ng, ZP * grp / ng, ZP * (grp + 1) / ng};
    }
};
// Many arrays (fdas_convolve_batch): array i owns segment pairs [item_off_i, item_off_i +
// n_sp_i) of the launch; the units (segment pair, template pair) of all arrays in order are
// shared out like those of one array, items cut at segment-pair (so also array) boundaries.
struct BatchSrc {
    const BatchTable *t;
    int ZP;
    __device__ __forceinline__ unsigned units() const { return (unsigned)t->total_items * (unsigned)ZP; }
    __device__ __forceinline__ unsigned u0() const
    {
        const unsigned U = units(), b = blockIdx.x, q = U / gridDim.x, r = U % gridDim.x;
        return b * q + (b < r ? b : r);
    }
    __device__ __forceinline__ unsigned u1() const
    {
        const unsigned U = units(), b = blockIdx.x, q = U / gridDim.x, r = U % gridDim.x;
        return b * q + (b < r ? b : r) + q + (b < r ? 1u : 0u);
    }
    __device__ __forceinline__ int count() const
    {
        const unsigned a0 = u0(), a1 = u1();
        return a1 > a0 ? (int)((a1 - 1) / (unsigned)ZP - a0 / (unsigned)ZP + 1) : 0;
    }
    __device__ __forceinline__ Item item(int k) const
    {
        const unsigned a0 = u0(), a1 = u1();
        const int gsp = (int)(a0 / (unsigned)ZP) + k;
        int lo = 0, hi = t->count - 1;   // the last array whose first segment pair is <= gsp
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t->arr[mid].item_off <= gsp) lo = mid;
            else hi = mid - 1;
        }
        const BatchArray &ba = t->arr[lo];
        const unsigned b0 = (unsigned)gsp * (unsigned)ZP, e0 = b0 + (unsigned)ZP;
        const int zp0 = (int)((a0 > b0 ? a0 : b0) - b0), zp1 = (int)((a1 < e0 ? a1 : e0) - b0);
        return Item{&ba.map, ba.out, ba.n, 0, ba.nseg, gsp - (int)ba.item_off, zp0, zp1};
    }
};

__host__ __device__ inline uint32_t b1_off(int j, int k)
{
    return (uint32_t)((j >> 3) * SBO1 + (k >> 3) * LBO1 + (j & 7) * 16 + (k & 7) * 2);
}
__host__ __device__ inline uint32_t g_off(int c, int k)
{
    return (uint32_t)((c >> 3) * SBOG + (k >> 3) * LBOG + (c & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// D (TMEM) (+)= A (shared-memory descriptor) . B (shared-memory descriptor)
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// D (TMEM) (+)= A (TMEM) . B (shared-memory descriptor)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Named barrier of the product group (warps 0-3).
struct PSync {
    static __device__ __forceinline__ void sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
};
// All 128 threads of the product group agree on `ok` (and synchronise).
__device__ __forceinline__ bool p_all(bool ok)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.and.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)ok)
                 : "memory");
    return r != 0;
}

// Named hardware barriers for the handoffs of read accumulators (D1 by the twiddle group, D2 by
// the power group) back to the MMA warp that overwrites them: a group of 128 threads arrives
// once its tcgen05.ld have completed, the MMA warp syncs.  They wake the consumer sooner than an
// mbarrier.  The handoffs of written operands (A1 in tensor memory, the stage-2 operand in
// shared memory) go through mbarriers instead: with named barriers there, about one launch in
// a hundred of the 2^22-point plane had one (segment, template) tile differ between relaunches,
// with or without a fence.acq_rel.cta before the arrive; with mbarriers none in 3000 launches.
// Every role runs its loops to the end, skipping a tile's work once one of its waits has given
// up (a warp vote on the waits' results) but still arriving, so that no consumer waits on an
// arrival that never comes.
enum : int { NB_D1 = 4, NB_D2 = 9 };   // D1 x 3, D2 x 2
constexpr int NB_COUNT = NT + 32;
__device__ __forceinline__ void nb_arrive(int id) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(NB_COUNT) : "memory"); }
__device__ __forceinline__ void nb_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(NB_COUNT) : "memory"); }

// Bounded wait that also returns early once another role has given up (abort flag set).
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// ---------------------------------------------------------------------------------------
// Plan-time kernels (FP64).
// ---------------------------------------------------------------------------------------

// exp(+2 pi i num / den) for an exact integer numerator (reduced mod den first).
__device__ inline double2 expi(int64_t num, int den)
{
    const int64_t r = ((num % den) + den) % den;
    double s, c;
    sincospi(2.0 * (double)r / (double)den, &s, &c);
    return make_double2(c, s);
}

// B1, G and the twiddle table, one thread per entry.
__global__ void tc2_constants_kernel(unsigned char *cst)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id < 64 * 64) {   // B1[j][k]: j = 4q + 2ro + e (output n1 = 2q + e, part ro), k = 2 k1 + ri
        const int j = id / 64, k = id % 64;
        const int n1 = 2 * (j / 4) + (j & 1), ro = (j / 2) & 1, k1 = k / 2, ri = k & 1;
        const double2 w = expi((int64_t)n1 * k1, 32);
        const double v = ro == 0 ? (ri == 0 ? w.x : -w.y) : (ri == 0 ? w.y : w.x);
        reinterpret_cast<__half *>(cst + CB_B1)[b1_off(j, k) / 2] = __double2half(v);
    } else if (id < 64 * 64 + 128 * 128) {   // G[c][kappa]: c = 4 (n2/2) + 2 ro + n2 % 2, kappa = 64 ri + k2
        const int e = id - 64 * 64, c = e / 128, kap = e % 128;
        const int n2 = 2 * (c / 4) + (c & 1), ro = (c / 2) & 1, ri = kap / 64, k2 = kap % 64;
        const double2 w = expi((int64_t)n2 * k2, 64);
        const double v = ro == 0 ? (ri == 0 ? w.x : -w.y) : (ri == 0 ? w.y : w.x);
        reinterpret_cast<__half *>(cst + CB_G)[g_off(c, kap) / 2] = __double2half(v);
    } else if (id < 64 * 64 + 128 * 128 + 64 * 32) {   // T[k2][n1] = exp(+2 pi i n1 k2 / 2048) / 32
        const int e = id - 64 * 64 - 128 * 128, k2 = e / 32, n1 = e % 32;
        const double2 w = expi((int64_t)n1 * k2, L);
        float *t = reinterpret_cast<float *>(cst + CB_TW) + k2 * 64 + 4 * (n1 / 2) + (n1 & 1);
        t[0] = (float)(w.x / 32.0);
        t[2] = (float)(w.y / 32.0);
    }
}

// H16[z][k2][k1] = FFT_L(h_z)[k2 + 64 k1] * 2^eH in fp16 (direct FP64 DFT of the zero-padded
// template, exact argument reduction), k1 = 32..35 zero padding; templates z >= M are zero.
__global__ void tc2_pretransform_kernel(const float2 *__restrict__ h32, int M, int K, const double2 *__restrict__ w64,
                                        int eH, int M_even, unsigned char *__restrict__ H16)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)M_even * 64 * 36) return;
    const int k1 = (int)(id % 36), k2 = (int)((id / 36) % 64), z = (int)(id / (36 * 64));
    double re = 0.0, im = 0.0;
    if (z < M && k1 < 32) {
        const int f = k2 + 64 * k1;
        const float2 *h = h32 + (size_t)z * K;
        for (int k = 0; k < K; ++k) {
            const double2 w = w64[((int64_t)k * f) & (L - 1)];
            const double hr = (double)h[k].x, hi = (double)h[k].y;
            re += hr * w.x - hi * w.y;
            im += hr * w.y + hi * w.x;
        }
        re = ldexp(re, eH);
        im = ldexp(im, eH);
    }
    __half2 *dst = reinterpret_cast<__half2 *>(H16 + (size_t)z * H_BYTES + (size_t)k2 * H_ROW) + k1;
    *dst = __halves2half2(__double2half(re), __double2half(im));
}

}  // namespace tc2

// ---------------------------------------------------------------------------------------
// The segment kernel: one block per SM, each with its share of the work items (segment pair,
// template-pair range) from the item source Src.
// ---------------------------------------------------------------------------------------
template <bool CAND, class Src>
__device__ __forceinline__ void tc2_body(const Src &src, const tc2::Args &a)
{
    using namespace tc2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *segb = reinterpret_cast<float2 *>(sm + Smem::seg);
    float2 *e2 = reinterpret_cast<float2 *>(sm + Smem::e2);
    unsigned char *hb = sm + Smem::hb;
    unsigned char *b2 = sm + Smem::b2;
    float *red = reinterpret_cast<float *>(sm + Smem::red);
    float *scl = reinterpret_cast<float *>(sm + Smem::scale);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + Smem::bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Smem::misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + Smem::misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = src.count();   // this block's items
    constexpr int CTRL = 3 * NT;   // the MMA thread initialises the barriers

    if (tid == CTRL) {
        mbar_init(&bar[B_SEG_FULL], 1);
        mbar_init(&bar[B_SEG_FREE], NT);
        mbar_init(&bar[B_B1_FULL], 1);
        mbar_init(&bar[B_SCALE0], 1);
        mbar_init(&bar[B_SCALE1], 1);
        mbar_init(&bar[B_SFREE0], 4);   // lane 0 of each power warp
        mbar_init(&bar[B_SFREE1], 4);
        for (int i = 0; i < NH; ++i) {
            mbar_init(&bar[B_H_FULL + i], 1);
            mbar_init(&bar[B_H_FREE + i], 4);   // one lane per product warp
        }
        for (int i = 0; i < (int)ND1; ++i)
            mbar_init(&bar[B_MMA1 + i], 1);        // stage 1 of tile t done: D1[t % 3] full, A1[t % 2] free
        for (int i = 0; i < 2; ++i) mbar_init(&bar[B_MMA2 + i], 1);   // stage 2 of pair q: D2 full, B2 free
        // the written-operand and template-free handoffs: one elected lane per producer warp
        // arrives after a __syncwarp, so 4 arrivals instead of 128 shared atomics per handoff
        for (int i = 0; i < 2; ++i) mbar_init(&bar[B_B2F + i], 4);
        for (int i = 0; i < 2; ++i) mbar_init(&bar[B_A1W + i], 4);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 12) tmem_alloc(tslot, TMEM_COLS);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp < 4) {
        // ---------------- product group: forward FFTs, X . H_z into the stage-1 operand ----------------
        const int k2 = tid & 63, sg = tid >> 6;
        uint32_t t = 0;
        int il = 0;
        for (int k = 0; k < nk; ++k, ++il) {
            const Item ii = src.item(k);
            const int zp0 = ii.zp0, zp1 = ii.zp1;
            if (!p_all(!*abort_flag && wait_bar(&bar[B_SEG_FULL], il & 1, abort_flag))) {
                for (int j = 0; j < 2 * (zp1 - zp0); ++j, ++t)   // keep the handoffs
                    if (lane == 0) mbar_arrive(&bar[B_A1W + (t & 1)]);
                continue;
            }
            float2 v[16], Xa[16], Xb[16];
            forward_fft<L, NoHook, PSync>(segb, segb, e2, a.tw, v, Xa);
            forward_fft<L, NoHook, PSync>(segb + L, segb + L, e2, a.tw, v, Xb);
            float ma = 0.f, mb = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                ma = fmaxf(ma, fmaxf(fabsf(Xa[j].x), fabsf(Xa[j].y)));
                mb = fmaxf(mb, fmaxf(fabsf(Xb[j].x), fabsf(Xb[j].y)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
                mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
            }
            if (lane == 0) {
                red[2 * warp] = ma;
                red[2 * warp + 1] = mb;
            }
            PSync::sync();   // every read of the segment buffers is done; maxima visible
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int f = freq_of_slot(L, tid, j);
                segb[f] = Xa[j];
                segb[L + f] = Xb[j];
            }
            int ex[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float m = fmaxf(fmaxf(red[s], red[2 + s]), fmaxf(red[4 + s], red[6 + s]));
                int E = 0;
                frexpf(m, &E);
                ex[s] = min(100, max(-60, 11 - E));   // |X| 2^e < 2^11 (|X| < 2^71)
            }
            if (tid == 0) {   // power factor 2^(2 (-6 - e - eH)) of each segment for the epilogue
                if (il >= 2) wait_bar(&bar[B_SFREE0 + (il & 1)], ((il >> 1) - 1) & 1, abort_flag);
                scl[2 * (il & 1)] = ldexpf(1.f, 2 * (-6 - ex[0] - a.eH));
                scl[2 * (il & 1) + 1] = ldexpf(1.f, 2 * (-6 - ex[1] - a.eH));
                mbar_arrive(&bar[B_SCALE0 + (il & 1)]);
            }
            PSync::sync();   // spectra in natural order visible
            __half2 x[32], xs[32];
            {
                const float f = ldexpf(1.f, sg ? ex[1] : ex[0]);
                const float2 *Xs = segb + sg * L + k2;
#pragma unroll
                for (int k1 = 0; k1 < 32; ++k1) {
                    const float2 c = Xs[64 * k1];
                    x[k1] = __floats2half2_rn(c.x * f, c.y * f);
                    xs[k1] = __floats2half2_rn(-c.y * f, c.x * f);
                }
            }
            mbar_arrive(&bar[B_SEG_FREE]);
            for (int zp = zp0; zp < zp1; ++zp) {
#pragma unroll
                for (int zz = 0; zz < 2; ++zz, ++t) {
                    const int slot = (int)(t % NH);
                    bool okw = wait_bar(&bar[B_H_FULL + slot], (t / NH) & 1, abort_flag);
                    if (t >= 2) okw = wait_bar(&bar[B_MMA1 + (t - 2) % ND1], ((t - 2) / ND1) & 1, abort_flag) && okw;
                    if (!__all_sync(0xffffffffu, okw)) {
                        if (lane == 0) mbar_arrive(&bar[B_A1W + (t & 1)]);
                        continue;
                    }
                    tmem_fence_after_sync();
                    const uint4 *hrow = reinterpret_cast<const uint4 *>(hb + slot * H_BYTES + k2 * H_ROW);
                    uint32_t y[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint4 hv = hrow[c];
                        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const __half2 h = *reinterpret_cast<const __half2 *>(&hw[i]);
                            const __half2 r = __hfma2(__low2half2(h), x[4 * c + i], __hmul2(__high2half2(h), xs[4 * c + i]));
                            y[4 * c + i] = *reinterpret_cast<const uint32_t *>(&r);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[B_H_FREE + slot]);
                    tmem_st32(tmem_lane_addr(tmem, COL_A1 + 32 * (t & 1)), y);
                    tmem_fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bar[B_A1W + (t & 1)]);
                }
            }
        }
    } else if (warp < 8) {
        // ---------------- twiddle group: D1 . W2048^{n1 k2} / 32 -> fp16 stage-2 operand ----------------
        const int ht = tid - NT, k2 = ht & 63, sg = ht >> 6;
        float tw[64];
        {
            const float4 *src = reinterpret_cast<const float4 *>(a.cst + CB_TW) + k2 * 16;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float4 q = __ldg(src + i);
                tw[4 * i] = q.x;
                tw[4 * i + 1] = q.y;
                tw[4 * i + 2] = q.z;
                tw[4 * i + 3] = q.w;
            }
        }
        uint32_t t = 0;
        for (int k = 0; k < nk; ++k) {
            const Item ii = src.item(k);
            const int zp0 = ii.zp0, zp1 = ii.zp1;
            for (int zp = zp0; zp < zp1; ++zp) {
#pragma unroll 1
                for (int zz = 0; zz < 2; ++zz, ++t) {
                    const uint32_t p = t >> 1;
                    bool okw = wait_bar(&bar[B_MMA1 + t % ND1], (t / ND1) & 1, abort_flag);
                    if (zz == 0 && p >= 2) okw = wait_bar(&bar[B_MMA2 + (p & 1)], ((p - 2) >> 1) & 1, abort_flag) && okw;
                    if (!__all_sync(0xffffffffu, okw)) {
                        nb_arrive(NB_D1 + t % ND1);
                        if (zz == 1 && lane == 0) mbar_arrive(&bar[B_B2F + (p & 1)]);
                        continue;
                    }
                    tmem_fence_after_sync();
                    unsigned char *base = b2 + (p & 1) * B2_BYTES + (size_t)(4 * sg + 8 * zz) * SBO2;
                    const uint32_t dcol = tmem_lane_addr(tmem, COL_D1 + 64 * (t % ND1));
                    auto chunk = [&](int j, const uint32_t (&d)[16]) {   // n1 = 8 j .. 8 j + 7
                        uint32_t hr[4], hi[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {   // outputs n1 = 8 j + 2 q, +1
                            const float2 re = make_float2(__uint_as_float(d[4 * q]), __uint_as_float(d[4 * q + 1]));
                            const float2 im = make_float2(__uint_as_float(d[4 * q + 2]), __uint_as_float(d[4 * q + 3]));
                            const int w = 4 * (4 * j + q);
                            const float2 tr = make_float2(tw[w], tw[w + 1]), ti = make_float2(tw[w + 2], tw[w + 3]);
                            const float2 zr = csub(pmul(re, tr), pmul(im, ti));
                            const float2 zi = pfma(re, ti, pmul(im, tr));
                            hr[q] = pack_h2(zr.x, zr.y);
                            hi[q] = pack_h2(zi.x, zi.y);
                        }
#pragma unroll
                        for (int ri = 0; ri < 2; ++ri) {
                            const int kap = 64 * ri + k2;
                            unsigned char *row = base + (kap >> 3) * LBO2 + (kap & 7) * 16;
                            const uint32_t *hv = ri ? hi : hr;
                            *reinterpret_cast<uint4 *>(row + j * SBO2) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        }
                    };
                    // each chunk's arithmetic overlaps the next chunk's load; D1 is free once the last has landed
                    uint32_t da[16], db[16];
                    tmem_ld16_issue(dcol, da);
                    tmem_ld16_wait(da);
                    tmem_ld16_issue(dcol + 16, db);
                    chunk(0, da);
                    tmem_ld16_wait(db);
                    tmem_ld16_issue(dcol + 32, da);
                    chunk(1, db);
                    tmem_ld16_wait(da);
                    tmem_ld16_issue(dcol + 48, db);
                    chunk(2, da);
                    tmem_ld16_wait(db);
                    tmem_fence_before_sync();
                    nb_arrive(NB_D1 + t % ND1);
                    chunk(3, db);
                    if (zz == 1) {
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&bar[B_B2F + (p & 1)]);
                    }
                }
            }
        }
    } else if (warp < 12) {
        // ---------------- power group: |D2|^2 x 2^(2f), discard, stores ----------------
        // Warp q reads TMEM lanes 32 q .. 32 q + 31 = (n1 = lane, segment q % 2, template q / 2 of
        // the pair); columns 4 g + (0, 1, 2, 3) = re(2g), re(2g + 1), im(2g), im(2g + 1) of n2.
        const int q = warp & 3, sq = q & 1, zq = q >> 1;
        const uint32_t my = tmem_lane_addr(tmem, COL_D2);
        // threshold epilogue: crossings staged per warp in shared memory at slots given by warp
        // ballots (no atomics), one global reservation per flush of the staging
        fdas_candidate *stg = reinterpret_cast<fdas_candidate *>(sm + Smem::stage) + CAND_STAGE * q;
        unsigned nst = 0;   // staged records (warp-uniform)
        const unsigned lt = (1u << lane) - 1u;
        auto flush_stage = [&]() {   // whole warp
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0 && nst > 0) base = atomicAdd(a.cand_count, (unsigned long long)nst);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (unsigned i = lane; i < nst; i += 32)
                if (base + i < (unsigned long long)a.cand_max) a.cand[base + i] = stg[i];
            __syncwarp();
            nst = 0;
        };
        uint32_t p = 0;
        int il = 0;
        for (int k = 0; k < nk; ++k, ++il) {
            const Item ii = src.item(k);
            const int sp = ii.sp;
            const int zp0 = ii.zp0, zp1 = ii.zp1;
            wait_bar(&bar[B_SCALE0 + (il & 1)], (il >> 1) & 1, abort_flag);
            const float fs = scl[2 * (il & 1) + sq];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[B_SFREE0 + (il & 1)]);
            // outputs kept in this segment: t in [0, lim) (the step S, cut at n; none past the launch)
            const int64_t segrow = (int64_t)(ii.seg_begin + 2 * sp + sq) * a.S;
            const int64_t left = ii.n - segrow;
            const int lim = (2 * sp + sq < ii.nseg && left > 0) ? (int)(left < a.S ? left : a.S) : 0;
            const int tbase = lane - (a.K - 1);   // output index of n2 = 0
            for (int zp = zp0; zp < zp1; ++zp, ++p) {
                const bool okw = wait_bar(&bar[B_MMA2 + (p & 1)], (p >> 1) & 1, abort_flag);
                if (!__all_sync(0xffffffffu, okw)) {
                    nb_arrive(NB_D2 + (p & 1));
                    continue;
                }
                tmem_fence_after_sync();
                const int z = 2 * zp + zq;
                float *o = ii.out + (size_t)z * (size_t)ii.n + segrow;
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {   // n2 = 16 cc .. 16 cc + 15
                    uint32_t r[32];
                    tmem_ld32(my + 128 * (p & 1) + 32 * cc, r);
                    if (cc == 3) {
                        tmem_fence_before_sync();
                        nb_arrive(NB_D2 + (p & 1));
                    }
                    if (z >= a.M) continue;
                    float2 pw[8];
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const float2 re = make_float2(__uint_as_float(r[4 * g]), __uint_as_float(r[4 * g + 1]));
                        const float2 im = make_float2(__uint_as_float(r[4 * g + 2]), __uint_as_float(r[4 * g + 3]));
                        pw[g] = pmul(pfma(re, re, pmul(im, im)), make_float2(fs, fs));
                    }
                    if constexpr (CAND) {   // threshold epilogue: the kept outputs above the threshold, no plane
                        float mx = fmaxf(pw[0].x, pw[0].y);
#pragma unroll
                        for (int g = 1; g < 8; ++g) mx = fmaxf(mx, fmaxf(pw[g].x, pw[g].y));
                        if (!__any_sync(0xffffffffu, mx > a.threshold)) continue;   // most chunks: no crossing
                        const int c0 = 512 * cc - (a.K - 1);
                        const bool whole = c0 >= 0 && c0 + 511 < lim;   // every output of the chunk is kept
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            const int t0 = tbase + 32 * (16 * cc + 2 * g);
                            const bool cx = pw[g].x > a.threshold && (whole || (unsigned)t0 < (unsigned)lim);
                            const bool cy = pw[g].y > a.threshold && (whole || (unsigned)(t0 + 32) < (unsigned)lim);
                            const unsigned bx = __ballot_sync(0xffffffffu, cx), by = __ballot_sync(0xffffffffu, cy);
                            if ((bx | by) == 0) continue;
                            const unsigned nx = __popc(bx), nxy = nx + __popc(by);
                            if (nst + nxy > (unsigned)CAND_STAGE) flush_stage();
                            if (cx) {
                                fdas_candidate c;
                                c.tpl = z;
                                c.power = pw[g].x;
                                c.bin = segrow + t0;
                                stg[nst + __popc(bx & lt)] = c;
                            }
                            if (cy) {
                                fdas_candidate c;
                                c.tpl = z;
                                c.power = pw[g].y;
                                c.bin = segrow + t0 + 32;
                                stg[nst + nx + __popc(by & lt)] = c;
                            }
                            nst += nxy;
                        }
                        continue;
                    }
                    const int c0 = 512 * cc - (a.K - 1);   // output of lane 0 at n2 = 16 cc (warp-uniform)
                    if (c0 >= 0 && c0 + 511 < lim) {       // the whole chunk is kept: no per-store checks
                        float *oc = o + (c0 + lane);
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            oc[64 * g] = pw[g].x;
                            oc[64 * g + 32] = pw[g].y;
                        }
                    } else {
#pragma unroll
                        for (int g = 0; g < 8; ++g) {
                            const int t0 = tbase + 32 * (16 * cc + 2 * g);
                            if ((unsigned)t0 < (unsigned)lim) o[t0] = pw[g].x;
                            if ((unsigned)(t0 + 32) < (unsigned)lim) o[t0 + 32] = pw[g].y;
                        }
                    }
                }

            }
        }
        if constexpr (CAND) flush_stage();
    } else if (warp == 12) {
        // ---------------- stage-1 MMA warp (lane 0 issues) ----------------
        const uint32_t b1a = smem_u32(sm + Smem::b1);
        bool ok = wait_bar(&bar[B_B1_FULL], 0, abort_flag);
        __syncwarp();
        uint32_t t = 0;
        for (int k = 0; k < nk; ++k) {
            const Item ii = src.item(k);
            const int ntiles = 2 * (ii.zp1 - ii.zp0);
            for (int j = 0; j < ntiles; ++j, ++t) {
                const bool oka = wait_bar(&bar[B_A1W + (t & 1)], (t >> 1) & 1, abort_flag);   // A1[t % 2] written
                if (t >= ND1) nb_sync(NB_D1 + t % ND1);    // D1[t % 3] read by the twiddle group
                if (lane == 0 && ok && oka && !*abort_flag) {
                    tmem_fence_after_sync();
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_ts(tmem + COL_D1 + 64 * (t % ND1), tmem + COL_A1 + 32 * (t & 1) + 8 * ks,
                               smem_desc(b1a + ks * 2 * LBO1, LBO1, SBO1), IDESC1, ks > 0);
                    mma_commit(&bar[B_MMA1 + t % ND1]);
                }
                __syncwarp();
            }
        }
        if (lane == 0) {   // no MMA may be in flight when the tensor memory is released
            for (uint32_t i = (t > ND1 ? t - ND1 : 0); i < t; ++i)
                mbar_wait_bounded(&bar[B_MMA1 + i % ND1], (i / ND1) & 1, kWaitLimitNs);
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicOr(a.status, STATUS_WAIT_TIMEOUT);
            }
        }
    } else if (warp == 14) {
        // ---------------- stage-2 MMA warp (lane 0 issues) ----------------
        const uint32_t b2a = smem_u32(b2), ga = smem_u32(sm + Smem::g);
        bool ok = wait_bar(&bar[B_B1_FULL], 0, abort_flag);
        __syncwarp();
        uint32_t q = 0;
        for (int k = 0; k < nk; ++k) {
            const Item ii = src.item(k);
            const int npairs = ii.zp1 - ii.zp0;
            for (int j = 0; j < npairs; ++j, ++q) {
                const bool okb = wait_bar(&bar[B_B2F + (q & 1)], (q >> 1) & 1, abort_flag);   // both tiles of pair q transposed
                if (q >= 2) nb_sync(NB_D2 + (q & 1));      // D2[q % 2] read by the power group
                if (lane == 0 && ok && okb && !*abort_flag) {
                    tmem_fence_after_sync();
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)
                        mma_ss(tmem + COL_D2 + 128 * (q & 1), smem_desc(b2a + (q & 1) * B2_BYTES + ks * 2 * LBO2, LBO2, SBO2),
                               smem_desc(ga + ks * 2 * LBOG, LBOG, SBOG), IDESC2, ks > 0);
                    mma_commit(&bar[B_MMA2 + (q & 1)]);
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            for (uint32_t i = (q > 2 ? q - 2 : 0); i < q; ++i)
                mbar_wait_bounded(&bar[B_MMA2 + (i & 1)], (i >> 1) & 1, kWaitLimitNs);
            if (!ok || *abort_flag) {
                *abort_flag = 1;
                atomicOr(a.status, STATUS_WAIT_TIMEOUT);
            }
        }
    } else if (warp == 13 && lane == 0) {
        // ---------------- loader thread (warp 13): segments and templates by TMA ----------------
        mbar_arrive_expect_tx(&bar[B_B1_FULL], B1_BYTES + G_BYTES);   // both DFT matrices
        bulk_load(sm + Smem::b1, a.cst + CB_B1, B1_BYTES, &bar[B_B1_FULL]);
        bulk_load(sm + Smem::g, a.cst + CB_G, G_BYTES, &bar[B_B1_FULL]);
        uint32_t seg_issued = 0, tH = 0;
        bool ok = true;
        auto issue_segments = [&](int k) {
            const Item ii = src.item(k);
            mbar_arrive_expect_tx(&bar[B_SEG_FULL], 2u * L * (uint32_t)sizeof(float2));
#pragma unroll 1
            for (int s2 = 0; s2 < 2; ++s2) {
                const int c0 = (ii.seg_begin + 2 * ii.sp + s2) * a.S - (a.K - 1);
#pragma unroll
                for (int j = 0; j < L / 256; ++j) tma_load_1d(segb + s2 * L + 256 * j, ii.map, c0 + 256 * j, &bar[B_SEG_FULL]);
            }
            ++seg_issued;
        };
        if (nk > 0) issue_segments(0);
        int il = 0;
        for (int k = 0; ok && k < nk; ++k, ++il) {
            const Item ii = src.item(k);
            const int zp0 = ii.zp0, zp1 = ii.zp1;
            const int ntiles = 2 * (zp1 - zp0);
            for (int j = 0; ok && j < ntiles; ++j, ++tH) {
                const uint32_t slot = tH % NH;
                if (tH >= NH) ok = wait_bar(&bar[B_H_FREE + slot], ((tH / NH) - 1) & 1, abort_flag);
                if (!ok) break;
                mbar_arrive_expect_tx(&bar[B_H_FULL + slot], H_BYTES);
                bulk_load(hb + slot * H_BYTES, a.H16 + (size_t)(2 * zp0 + j) * H_BYTES, H_BYTES, &bar[B_H_FULL + slot]);
                // once the product group has taken this item's spectra, fetch the next item's segments
                if (j == min(NH, ntiles) - 1 && k + 1 < nk) {
                    ok = wait_bar(&bar[B_SEG_FREE], il & 1, abort_flag);
                    if (ok) issue_segments(k + 1);
                }
            }
        }
        // nothing may be in flight when the block leaves: the copies issued land first
        if (seg_issued) mbar_wait_bounded(&bar[B_SEG_FULL], (seg_issued - 1) & 1, kWaitLimitNs);
        for (uint32_t i = (tH > NH ? tH - NH : 0); i < tH; ++i)
            mbar_wait_bounded(&bar[B_H_FULL + i % NH], (i / NH) & 1, kWaitLimitNs);
        if (!ok || *abort_flag) {
            *abort_flag = 1;
            atomicOr(a.status, STATUS_WAIT_TIMEOUT);
        }
    }
    __syncwarp();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 12) tmem_dealloc(tmem, TMEM_COLS);
}

// One array: segments [s.seg_begin, s.seg_begin + s.nseg); CAND: the threshold crossings
// instead of the plane (a separate instantiation, so the plane kernel carries none of it).
template <bool CAND, class Src>
__global__ void __launch_bounds__(tc2::kThreads, 1)
    ols_tc2_kernel(const __grid_constant__ CUtensorMap tmap, const tc2::Args a, const Src s0)
{
    Src src = s0;
    src.map = &tmap;
    tc2_body<CAND>(src, a);
}

// Many arrays, one persistent launch: the same items and arithmetic per array as the
// single-array kernel, so every plane is bit-identical to that array's fdas_convolve.
// (Same parameter list as the FP32 batch kernel; the work counter is not used: each block takes
// an equal share of the launch's (segment pair, template pair) units.)
__global__ void __launch_bounds__(tc2::kThreads, 1)
    ols_tc2_batch(const __grid_constant__ BatchTable t, const OlsArgs o, int *counter)
{
    (void)counter;
    tc2::Args a;
    a.H16 = o.H16;
    a.cst = o.cst;
    a.tw = o.tw;
    a.M = o.M;
    a.S = o.S;
    a.K = o.K;
    a.ng = o.ng;
    a.ZP = (o.M + 1) / 2;
    a.eH = o.eH;
    a.status = o.status;
    a.cand = nullptr;
    a.cand_count = nullptr;
    a.cand_max = 0;
    a.threshold = 0.f;
    tc2::BatchSrc src;
    src.t = &t;
    src.ZP = a.ZP;
    tc2_body<false>(src, a);
}

// ---------------------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------------------
size_t tc2_const_bytes() { return tc2::CONST_BYTES; }
size_t tc2_template_bytes(int M) { return (size_t)(2 * ((M + 1) / 2)) * tc2::H_BYTES; }

cudaError_t launch_tc2_constants(unsigned char *cst, cudaStream_t s)
{
    const int total = 64 * 64 + 128 * 128 + 64 * 32;
    tc2::tc2_constants_kernel<<<(total + 255) / 256, 256, 0, s>>>(cst);
    return cudaGetLastError();
}

cudaError_t launch_tc2_pretransform(const float2 *h32, int M, int K, const double2 *w64, int eH, unsigned char *H16,
                                    cudaStream_t s)
{
    const int M_even = 2 * ((M + 1) / 2);
    const int64_t total = (int64_t)M_even * 64 * 36;
    tc2::tc2_pretransform_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(h32, M, K, w64, eH, M_even, H16);
    return cudaGetLastError();
}

// Template-pair groups per segment pair: the fewest waves of (one block per SM) x the items'
// length in template pairs plus about two pairs of fixed cost (the two forward FFTs and the
// pipeline fill and drain).
// Fewer units than this per block (a few template pairs) and a block's share would cross a
// segment pair for a handful of units, doubling its forward FFTs: short arrays take groups.
constexpr int kMinUnitsPerBlock = 12;

static int tc2_groups(int64_t n_sp, int ZP, int sms)
{
    int best_ng = 1;
    double best = 1e300;
    for (int ng = 1; ng <= ZP && ng <= 64; ++ng) {
        const int64_t items = n_sp * ng;
        const int64_t waves = (items + sms - 1) / sms;
        const double cost = (double)waves * ((double)((ZP + ng - 1) / ng) + 2.0);
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            best_ng = ng;
        }
    }
    return best_ng;
}

static cudaError_t tc2_setup(int *sms_out)
{
    static bool done[64] = {};
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
        const void *fns[4] = {(const void *)ols_tc2_kernel<false, tc2::SingleSrc>, (const void *)ols_tc2_kernel<true, tc2::SingleSrc>,
                              (const void *)ols_tc2_kernel<false, tc2::SingleGroupSrc>,
                              (const void *)ols_tc2_kernel<true, tc2::SingleGroupSrc>};
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc2::Smem::total);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ols_tc2_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc2::Smem::total);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    *sms_out = sms[dev];
    return cudaSuccess;
}

int tc2_groups_for(int64_t n_sp, int M)
{
    int sms = 0;
    if (tc2_setup(&sms) != cudaSuccess || sms <= 0) sms = 1;
    return tc2_groups(n_sp, (M + 1) / 2, sms);
}

cudaError_t tc2_batch_kernel(BatchKernel *k)
{
    int sms = 0;
    cudaError_t e = tc2_setup(&sms);
    if (e != cudaSuccess) return e;
    k->fn = reinterpret_cast<const void *>(ols_tc2_batch);
    k->block = tc2::kThreads;
    k->smem = tc2::Smem::total;
    k->resident = sms;   // one block per SM (tensor memory and shared memory)
    return cudaSuccess;
}

cudaError_t launch_ols_tc2(const CUtensorMap *tmap, const OlsArgs &o, const unsigned char *H16,
                           const unsigned char *cst, int eH, int nseg, cudaStream_t s)
{
    int sms = 0;
    cudaError_t e = tc2_setup(&sms);
    if (e != cudaSuccess) return e;
    if (nseg <= 0) return cudaSuccess;
    tc2::Args a;
    a.H16 = H16;
    a.cst = cst;
    a.tw = o.tw;
    a.M = o.M;
    a.S = o.S;
    a.K = o.K;
    a.ZP = (o.M + 1) / 2;
    a.eH = eH;
    a.status = o.status;
    a.cand = o.cand;
    a.cand_count = o.cand_count;
    a.cand_max = o.cand_max;
    a.threshold = o.threshold;
    const int n_sp = (nseg + 1) / 2;
    const int64_t units = (int64_t)n_sp * a.ZP;
    if (units >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    if (units >= (int64_t)kMinUnitsPerBlock * sms) {   // equal unit shares
        tc2::SingleSrc src;
        src.map = nullptr;   // the kernel points it at its own parameter copy of the map
        src.out = o.out;
        src.n = o.n;
        src.seg_begin = o.seg_begin;
        src.nseg = nseg;
        src.n_sp = n_sp;
        src.ZP = a.ZP;
        src.q = (int)(units / sms);
        src.r = (int)(units % sms);
        a.ng = 0;
        if (a.cand) ols_tc2_kernel<true><<<sms, tc2::kThreads, tc2::Smem::total, s>>>(*tmap, a, src);
        else ols_tc2_kernel<false><<<sms, tc2::kThreads, tc2::Smem::total, s>>>(*tmap, a, src);
    } else {   // short array: whole template-pair groups of one segment pair per item
        tc2::SingleGroupSrc src;
        src.map = nullptr;
        src.out = o.out;
        src.n = o.n;
        src.seg_begin = o.seg_begin;
        src.nseg = nseg;
        src.n_sp = n_sp;
        src.ZP = a.ZP;
        a.ng = src.ng = tc2_groups(n_sp, a.ZP, sms);
        const int64_t items = (int64_t)n_sp * src.ng;
        const int grid = (int)(items < sms ? items : sms);
        if (a.cand) ols_tc2_kernel<true><<<grid, tc2::kThreads, tc2::Smem::total, s>>>(*tmap, a, src);
        else ols_tc2_kernel<false><<<grid, tc2::kThreads, tc2::Smem::total, s>>>(*tmap, a, src);
    }
    return cudaGetLastError();
}

}  // namespace fdas
