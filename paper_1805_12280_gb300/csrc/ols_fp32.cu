// Fused FP32 overlap-save segment kernels (Algorithm 2 with the forward FFT shared by
// all templates, Table 1 text; power output, Sec. 4.3).
//
// One work item = (array, segment, template group).  A block of NT = L/16 threads:
//   1. TMA loads the L-point segment x[s*S - (K-1) .. s*S - (K-1) + L) into shared
//      memory; the tensor map zero-fills before 0 (the K-1 leading zeros of the first
//      segment) and past n;
//   2. forward FFT (passes A, B, C; two shared-memory exchanges); the spectrum waits in
//      the thread's TMEM lane for the whole template loop;
//   3. per template: element-wise product with the pre-transformed template (prefetched
//      by cp.async.bulk into shared memory, one template ahead in a single buffer at
//      L = 2048 and 4096, two ahead in a double buffer at L = 1024), inverse FFT (passes
//      C', B', A'; two exchanges; 1/L is folded into the template), discard of the first
//      K-1 points, |y|^2, coalesced stores of the valid S points.
// ols_fp32_kernel runs one item per block (grid = segments x groups of one array);
// ols_fp32_batch is persistent: resident blocks pull items of many arrays from a
// device work counter.
#include <cuda.h>
#include <cuda_runtime.h>

#include "fdas_internal.cuh"
#include "fft_regs.cuh"
#include "ols_common.cuh"
#include "ptx.cuh"
#include "tmem.cuh"

// Minimum resident blocks per SM requested from the compiler (caps registers per thread).
#ifndef FDAS_MINB_1024
#define FDAS_MINB_1024 4
#endif
#ifndef FDAS_MINB_2048
#define FDAS_MINB_2048 4
#endif
#ifndef FDAS_MINB_4096
#define FDAS_MINB_4096 2
#endif

// Template buffers per block: 2 prefetches two templates ahead; 1 prefetches one ahead and
// frees L*8 bytes of shared memory (one more resident block per SM at L = 2048 and 4096).
#ifndef FDAS_HBUF_2048
#define FDAS_HBUF_2048 1
#endif
#ifndef FDAS_HBUF_4096
#define FDAS_HBUF_4096 1
#endif

namespace fdas {

template <int L>
__host__ __device__ constexpr int hbuf() { return L == 2048 ? FDAS_HBUF_2048 : (L == 4096 ? FDAS_HBUF_4096 : 2); }

template <int L>
struct Smem {
    static constexpr size_t seg_bytes = sizeof(float2) * L;                   // segment / exchange 1
    static constexpr size_t e2_bytes = sizeof(float2) * 16 * Geo<L>::LD2;    // exchange 2
    static constexpr size_t h_bytes = sizeof(float2) * L;                     // one pre-transformed template
    static constexpr size_t total = 128 + seg_bytes + e2_bytes + hbuf<L>() * h_bytes + 3 * 8 + 8;   // + TMEM slot
};

// Tensor memory per block: each thread keeps its inverse twiddles (2 x 32 columns) and the
// segment spectrum (32 columns) in its own TMEM lane instead of registers; threads of the
// second warpgroup (L = 4096) use columns 96.. of the same lanes.
template <int L>
constexpr uint32_t kTmemCols = (L / 16 > 128) ? 256u : 128u;
constexpr uint32_t kColTw1 = 0, kColTw2 = 32, kColX = 64, kColGroup = 96;

constexpr int kCandCap = 256;    // candidates staged per block before one global reservation (4 KB: four blocks per SM still fit)
constexpr size_t kCandSmem = sizeof(fdas_candidate) * kCandCap + 16;

template <int L>
constexpr int minb()
{
    return L == 4096 ? FDAS_MINB_4096 : (L == 2048 ? FDAS_MINB_2048 : FDAS_MINB_1024);
}

// The persistent batch kernel carries its item loop in registers too: its own bound.
#ifndef FDAS_BATCH_MINB_2048
#define FDAS_BATCH_MINB_2048 4
#endif
template <int L>
constexpr int batch_minb()
{
    return L == 2048 ? FDAS_BATCH_MINB_2048 : minb<L>();
}

// Shared-memory carve-up and mbarrier phase bookkeeping of one block.
template <int L>
struct Block {
    float2 *e1;      // segment, then exchange buffer 1 [L]
    float2 *e2;      // exchange buffer 2 [16][NT + 1]
    float4 *hb;      // template buffer(s) [hbuf<L>()][8][NT]
    uint64_t *bar;   // [0] segment, [1], [2] template buffers
    uint32_t *tslot; // TMEM base address written by the allocating warp
    uint32_t tmem = 0;
    fdas_candidate *sb = nullptr;   // candidate staging [kCandCap] (candidate kernel only)
    unsigned *sc = nullptr;         // staging reservation counter
    uint32_t seg_uses = 0, h_uses0 = 0, h_uses1 = 0;   // completed phases per barrier (scalars:
                                                       // a runtime-indexed array would spill to local memory)

    __device__ explicit Block(unsigned char *raw)
    {
        e1 = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
        e2 = e1 + L;
        hb = reinterpret_cast<float4 *>(e2 + 16 * Geo<L>::LD2);
        bar = reinterpret_cast<uint64_t *>(hb + hbuf<L>() * 8 * Geo<L>::NT);
        tslot = reinterpret_cast<uint32_t *>(bar + 3);
    }
};

template <int L>
__device__ __forceinline__ void init_block(Block<L> &B, const OlsArgs &a)
{
    using Gm = Geo<L>;
    constexpr int NT = Gm::NT, Q = Gm::Q, R = Gm::R, GB = Gm::GB, GC = Gm::GC, MASK = L - 1;
    const int tid = threadIdx.x, k1 = tid & 15, hi = tid >> 4;
    if (tid == 0) {
        mbar_init(&B.bar[0], 1);
        mbar_init(&B.bar[1], 1);
        mbar_init(&B.bar[2], 1);
        fence_mbar_init();
    }
    if ((tid >> 5) == 0) tmem_alloc(B.tslot, kTmemCols<L>);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    B.tmem = *B.tslot;
    // Inverse-transform twiddles, fixed for this thread across all items and templates.
    float2 tw1[16], tw2[16];
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const int k2 = hi + (NT / 16) * g;
#pragma unroll
        for (int c = 0; c < R; ++c) tw1[g * R + c] = cconj(__ldg(&a.tw[(16 * c * k2) & MASK]));
    }
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int cg = hi + (NT / 16) * g;
#pragma unroll
        for (int b = 0; b < Q; ++b) tw2[g * Q + b] = cconj(__ldg(&a.tw[((b * R + cg) * k1) & MASK]));
    }
    const uint32_t my = tmem_lane_addr(B.tmem, (uint32_t)(tid >> 7) * kColGroup);
    tmem_st_c16(my + kColTw1, tw1);
    tmem_st_c16(my + kColTw2, tw2);
    __syncthreads();
}

// Every thread of the block, after its last TMEM access: the allocating warp frees it.
template <int L>
__device__ __forceinline__ void release_block(Block<L> &B)
{
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(B.tmem, kTmemCols<L>);
}

// After a timed-out wait: give each copy that may still be in flight a bounded time to
// land before the block exits.  `pending` bit i: barrier i has an issued, un-awaited phase
// whose parity is `parity` bit i.
__device__ __noinline__ void drain(uint64_t *bar, unsigned pending, unsigned parity)
{
    for (int i = 0; i < 3; ++i)
        if (pending & (1u << i)) mbar_wait_bounded(&bar[i], (parity >> i) & 1u, kWaitLimitNs);
}

// No item follows (one item per block).
struct NoNext {
    __device__ __forceinline__ bool operator()(const CUtensorMap **, int *) const { return false; }
};

// One work item.  Every thread of the block calls it with the same arguments after a
// block-wide barrier that follows the previous item.  Returns false (block-uniformly)
// if a bounded wait ran out; the status bit is then set.
//
// Cross-item prefetch (single template buffer only): when thread 0's `next` names the
// following item's input (tensor map and first coordinate), its segment is loaded into the
// template buffer as soon as the last template of this item has been read; the following
// item is then called with `prefetched` set, transforms the segment from there and loads
// its first template only after the forward pass A.
//
// VMASK: the plane stores test a bit mask of the thread's kept slots (per item; per template
// near the array end for grouped plans) instead of comparing each output index: fewer instructions per
// template in the one-item kernel; the persistent kernel, at its register limit, runs faster
// without it.
template <int L, bool CAND = false, class Next = NoNext, bool VMASK = false>
__device__ __forceinline__ bool run_item(Block<L> &B, const OlsArgs &a, const CUtensorMap *map, int seg, int z0,
                                         int z1, int64_t n, float *out, bool prefetched = false, Next next = Next())
{
    using Gm = Geo<L>;
    constexpr int NT = Gm::NT, Q = Gm::Q, R = Gm::R, GB = Gm::GB, GC = Gm::GC, LD2 = Gm::LD2;
    constexpr uint32_t HBYTES = (uint32_t)Smem<L>::h_bytes;
    constexpr int NHB = hbuf<L>();
    float2 *e1 = B.e1, *e2 = B.e2;
    float4 *hb = B.hb;
    uint64_t *bar = B.bar;
    const int tid = threadIdx.x, k1 = tid & 15, hi = tid >> 4;

    static_assert(NHB == 2 || HBYTES == L * sizeof(float2), "a prefetched segment fills the template buffer");
    static_assert(NHB == 2 || (sizeof(float2) * (L + 16 * Gm::LD2)) % 128 == 0, "TMA destination alignment");
    if (tid == 0 && !prefetched) {
        fence_proxy_async_smem();   // earlier generic writes to e1/hb are ordered before the async copies
        mbar_arrive_expect_tx(&bar[0], (uint32_t)(L * sizeof(float2)));
        const int c0 = seg * a.S - (a.K - 1);
#pragma unroll
        for (int j = 0; j < L / 256; ++j) tma_load_1d(e1 + 256 * j, map, c0 + 256 * j, &bar[0]);
        for (int i = 0; i < NHB && z0 + i < z1; ++i) {
            mbar_arrive_expect_tx(&bar[1 + i], HBYTES);
            bulk_load(hb + i * 8 * NT, a.H + (size_t)(z0 + i) * 8 * NT, HBYTES, &bar[1 + i]);
        }
    }
    // Block-uniform decision: every thread leaves together if the segment never arrived.
    const bool seg_ok = mbar_wait_bounded(&bar[0], B.seg_uses & 1, kWaitLimitNs);
    B.seg_uses++;
    if (!__syncthreads_and(seg_ok)) {
        if (tid == 0) {
            atomicOr(a.status, STATUS_WAIT_TIMEOUT);
            const unsigned pending = prefetched ? 1u : (1u | 2u | (NHB == 2 && z0 + 1 < z1 ? 4u : 0u));
            const unsigned parity = ((B.seg_uses - 1) & 1u) | ((B.h_uses0 & 1u) << 1) | ((B.h_uses1 & 1u) << 2);
            drain(bar, pending, parity);
        }
        return false;
    }

    float2 v[16];
    const uint32_t my = tmem_lane_addr(B.tmem, (uint32_t)(tid >> 7) * kColGroup);
    {
        float2 X[16];
        if (prefetched) {   // segment in the template buffer: its first template follows pass A
            forward_fft<L>(reinterpret_cast<const float2 *>(hb), e1, e2, a.tw, v, X, [&]() {
                if (tid == 0) {
                    mbar_arrive_expect_tx(&bar[1], HBYTES);
                    bulk_load(hb, a.H + (size_t)z0 * 8 * NT, HBYTES, &bar[1]);
                }
            });
        } else {
            forward_fft<L>(e1, e2, a.tw, v, X);
        }
        tmem_st_c16(my + kColX, X);   // the spectrum waits in TMEM for the template loop
    }
    __syncthreads();   // every thread has read e1 before the template loop rewrites it

    const int64_t seg_out = (int64_t)seg * a.S;                 // first output index of this segment
    const int64_t nvalid64 = n - seg_out;
    const unsigned nvalid = (unsigned)(nvalid64 < a.S ? nvalid64 : a.S);
    const int obase = tid - (a.K - 1);                          // output index of register slot 0
    unsigned vmask0 = 0;   // bit j: register slot j of this thread holds a kept output
    if constexpr (VMASK) {
#pragma unroll
        for (int j = 0; j < 16; ++j) vmask0 |= ((unsigned)(j * NT + obase) < nvalid ? 1u : 0u) << j;
    }

    for (int z = z0; z < z1; ++z) {
        // output row and shift of this template (identity unless the plan groups templates)
        int row = z;
        int64_t shift = 0;
        unsigned nv = nvalid;
        unsigned vmask = vmask0;
        if (a.rows) {
            row = __ldg(&a.rows[z]);
            shift = __ldg(&a.shifts[z]);
            const int64_t rem = n - shift - seg_out;
            nv = rem <= 0 ? 0u : (unsigned)(rem < a.S ? rem : a.S);
            if (VMASK && nv != nvalid) {   // only near the end of the array
                vmask = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) vmask |= ((unsigned)(j * NT + obase) < nv ? 1u : 0u) << j;
            }
            if (seg == 0 && shift > 0) {   // outputs before the first nonzero tap are zero
                const int64_t lim = shift < n ? shift : n;
                for (int64_t i = tid; i < lim; i += NT) {
                    if constexpr (CAND) {
                        if (0.f > a.threshold) {
                            const unsigned long long g = atomicAdd(a.cand_count, 1ull);
                            if (g < (unsigned long long)a.cand_max) {
                                fdas_candidate c;
                                c.tpl = row;
                                c.power = 0.f;
                                c.bin = i;
                                a.cand[g] = c;
                            }
                        }
                    } else {
                        out[(size_t)row * (size_t)n + i] = 0.f;
                    }
                }
            }
        }
        const int buf = NHB == 2 ? ((z - z0) & 1) : 0;
        const float4 *hz = hb + buf * 8 * NT;
        const uint32_t hu = buf ? B.h_uses1 : B.h_uses0;
        const bool h_ok = mbar_wait_bounded(&bar[1 + buf], hu & 1, kWaitLimitNs);
        if (buf) B.h_uses1++; else B.h_uses0++;
        // ---- element-wise product with H_z (1/L folded in)
        tmem_ld_c16(my + kColX, v);
#pragma unroll
        for (int jp = 0; jp < 8; ++jp) {
            const float4 h = hz[jp * NT + tid];
            v[2 * jp] = cmul(v[2 * jp], make_float2(h.x, h.y));
            v[2 * jp + 1] = cmul(v[2 * jp + 1], make_float2(h.z, h.w));
        }
        // ---- inverse pass C': R-point IDFT over k3, twiddle conj W_{QR}^{c k2}
        uint32_t t1r[32];   // the C' twiddles come back from TMEM during the radix-R DFTs
        tmem_ld32_issue(my + kColTw1, t1r);
        dft<R, 1, 1, 0>(v);
        if constexpr (GC == 2) dft<R, 1, 1, R>(v);
        tmem_ld32_wait(t1r);
        float2 tw1[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tw1[j] = make_float2(__uint_as_float(t1r[2 * j]), __uint_as_float(t1r[2 * j + 1]));
        if constexpr (GC == 2) {
            // the thread's two k2 values (hi and hi + Q/2) of each c share one 16-byte slot:
            // k1 + 16 (k2 mod Q/2) + 8 Q c; pass B' reads both halves with one load
            static_assert(NT / 16 == Q / 2, "paired exchange layout");
            float4 *e1q = reinterpret_cast<float4 *>(e1);
#pragma unroll
            for (int c = 0; c < R; ++c) {
                const float2 u0 = (c == 0) ? v[0] : cmul(v[c], tw1[c]);
                const float2 u1 = (c == 0) ? v[R] : cmul(v[R + c], tw1[R + c]);
                e1q[k1 + 16 * hi + 8 * Q * c] = make_float4(u0.x, u0.y, u1.x, u1.y);
            }
        } else {
#pragma unroll
            for (int c = 0; c < R; ++c)
                e1[k1 + 16 * hi + 16 * Q * c] = (c == 0) ? v[0] : cmul(v[c], tw1[c]);
        }
        if (!__syncthreads_and(h_ok)) {      // a template buffer never arrived: leave together
            if (tid == 0) {
                atomicOr(a.status, STATUS_WAIT_TIMEOUT);
                const int other = 1 - buf;
                const unsigned pending = (2u << buf) | (NHB == 2 && z + 1 < z1 ? (2u << other) : 0u);
                const uint32_t hb_ = buf ? B.h_uses1 : B.h_uses0, ho_ = buf ? B.h_uses0 : B.h_uses1;
                const unsigned parity = (((hb_ - 1) & 1u) << (1 + buf)) | ((ho_ & 1u) << (1 + other));
                drain(bar, pending, parity);
            }
            return false;
        }
        // every thread has read hb[buf]: refill it with the template NHB ahead, or, after the
        // last template, with the following item's segment
        if (tid == 0) {
            if (z + NHB < z1) {
                mbar_arrive_expect_tx(&bar[1 + buf], HBYTES);
                bulk_load(hb + buf * 8 * NT, a.H + (size_t)(z + NHB) * 8 * NT, HBYTES, &bar[1 + buf]);
            } else if (NHB == 1 && z + 1 == z1) {
                const CUtensorMap *nmap;
                int nc0;
                if (next(&nmap, &nc0)) {
                    mbar_arrive_expect_tx(&bar[0], (uint32_t)(L * sizeof(float2)));
                    float2 *dst = reinterpret_cast<float2 *>(hb);
#pragma unroll
                    for (int j = 0; j < L / 256; ++j) tma_load_1d(dst + 256 * j, nmap, nc0 + 256 * j, &bar[0]);
                }
            }
        }
        // ---- inverse pass B': Q-point IDFT over k2, twiddle conj W_L^{(bR + c) k1}
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int cg = hi + (NT / 16) * g;
            if constexpr (GC == 2) {
                const float4 *e1q = reinterpret_cast<const float4 *>(e1);
#pragma unroll
                for (int k2 = 0; k2 < Q / 2; ++k2) {
                    const float4 w = e1q[k1 + 16 * k2 + 8 * Q * cg];
                    v[g * Q + k2] = make_float2(w.x, w.y);
                    v[g * Q + k2 + Q / 2] = make_float2(w.z, w.w);
                }
            } else {
#pragma unroll
                for (int k2 = 0; k2 < Q; ++k2) v[g * Q + k2] = e1[k1 + 16 * k2 + 16 * Q * cg];
            }
        }
        dft<Q, 1, 1, 0>(v);
        if constexpr (GB == 2) dft<Q, 1, 1, Q>(v);
        float2 tw2[16];
        tmem_ld_c16(my + kColTw2, tw2);
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int cg = hi + (NT / 16) * g;
#pragma unroll
            for (int b = 0; b < Q; ++b) e2[(b * R + cg) + LD2 * k1] = cmul(v[g * Q + b], tw2[g * Q + b]);
        }
        __syncthreads();
        // ---- inverse pass A': 16-point IDFT over k1 -> natural order y[a*NT + t]
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = e2[tid + LD2 * k];
        dft<16, 1>(v);
        // ---- discard the first K-1 points, power, store the valid ones
        if constexpr (CAND) {
            // threshold crossings instead of the plane, staged per block in shared memory
            float pw[16], pmax = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                pw[j] = cabs2(v[j]);
                pmax = fmaxf(pmax, pw[j]);
            }
            // only lanes holding a crossing take the append path (one shared-memory atomic per
            // crossing); the short path keeps the warps of a block in step between barriers
            if (pmax > a.threshold) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {     // static slots: pw stays in registers
                    const int o = j * NT + obase;
                    if ((unsigned)o < nv && pw[j] > a.threshold) {
                        fdas_candidate c;
                        c.tpl = row;
                        c.power = pw[j];
                        c.bin = shift + seg_out + o;
                        const unsigned idx = atomicAdd(B.sc, 1u);
                        if (idx < (unsigned)kCandCap) {
                            B.sb[idx] = c;
                        } else {   // the block's staging is full: straight to global memory
                            const unsigned long long g = atomicAdd(a.cand_count, 1ull);
                            if (g < (unsigned long long)a.cand_max) a.cand[g] = c;
                        }
                    }
                }
            }
        } else {
            float *orow = out + (size_t)row * (size_t)n + shift + seg_out;
            if constexpr (VMASK) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (vmask & (1u << j)) orow[j * NT + obase] = cabs2(v[j]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int o = j * NT + obase;
                    if ((unsigned)o < nv) orow[o] = cabs2(v[j]);
                }
            }
        }
    }
    if constexpr (CAND) {   // one global reservation for the block's staged candidates
        __shared__ unsigned long long flush_base;
        __syncthreads();
        const unsigned staged = min(*B.sc, (unsigned)kCandCap);
        if (tid == 0) flush_base = staged ? atomicAdd(a.cand_count, (unsigned long long)staged) : 0ull;
        __syncthreads();
        for (unsigned i = tid; i < staged; i += NT)
            if (flush_base + i < (unsigned long long)a.cand_max) a.cand[flush_base + i] = B.sb[i];
        __syncthreads();
        if (tid == 0) *B.sc = 0;
    }
    return true;
}

// One item per block: blockIdx.x = segment (from a.seg_begin), blockIdx.y = template group.
// CAND: candidate epilogue instead of the plane stores.
template <int L, int MINB, bool CAND>
__global__ void __launch_bounds__(L / 16, MINB)
    ols_fp32_kernel(const __grid_constant__ CUtensorMap tmap, const OlsArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    Block<L> B(smem_raw);
    if constexpr (CAND) {
        B.sb = reinterpret_cast<fdas_candidate *>(smem_raw + Smem<L>::total);
        B.sc = reinterpret_cast<unsigned *>(B.sb + kCandCap);
        if (threadIdx.x == 0) *B.sc = 0;
    }
    init_block<L>(B, a);   // its barriers also publish *B.sc = 0
    const int z0 = blockIdx.y * a.G;
    run_item<L, CAND, NoNext, !CAND>(B, a, &tmap, a.seg_begin + blockIdx.x, z0, min(z0 + a.G, a.M), a.n, a.out);
    release_block<L>(B);
}

// Array of a batch item: the last array whose first item is <= item.
__device__ __forceinline__ int batch_array_of(const BatchTable &tab, int64_t item)
{
    int lo = 0, hi = tab.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab.arr[mid].item_off <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent: resident blocks take items (array, group, segment) from *counter until the
// table is exhausted.  Items are numbered array by array, group-major inside an array, so
// concurrently running blocks share templates and neighbouring segments in L2.  Thread 0
// takes the following item's number while the current one runs and, with a single template
// buffer, prefetches that item's segment behind the current item's last template.
template <int L, int MINB>
__global__ void __launch_bounds__(L / 16, MINB)
    ols_fp32_batch(const __grid_constant__ BatchTable tab, const OlsArgs a, int *counter)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int item_sh;
    Block<L> B(smem_raw);
    init_block<L>(B, a);
    if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1);
    __syncthreads();
    int64_t item = item_sh;
    bool prefetched = false;
    while (item < tab.total_items) {
        const BatchArray &ar = tab.arr[batch_array_of(tab, item)];
        const int64_t local = item - ar.item_off;
        const int g = (int)(local / ar.nseg), seg = (int)(local % ar.nseg);
        const int z0 = g * a.G;
        int64_t nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(counter, 1);   // consumed at the last template
        auto next = [&](const CUtensorMap **m, int *c0) -> bool {
            if (nxt >= tab.total_items) return false;
            const BatchArray &na = tab.arr[batch_array_of(tab, nxt)];
            *m = &na.map;
            *c0 = (int)((nxt - na.item_off) % na.nseg) * a.S - (a.K - 1);
            return true;
        };
        if (!run_item<L>(B, a, &ar.map, seg, z0, min(z0 + a.G, a.M), ar.n, ar.out, prefetched, next)) break;
        __syncthreads();                       // every thread has read item_sh
        if (threadIdx.x == 0) item_sh = (int)nxt;
        __syncthreads();
        item = item_sh;
        prefetched = hbuf<L>() == 1 && item < tab.total_items;
    }
    release_block<L>(B);
}

template <int L>
static cudaError_t set_smem_attr(const void *fn, bool *done, size_t bytes = Smem<L>::total)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    // prefer the largest shared-memory carveout: the occupancy query (and the persistent
    // grid sized from it) otherwise assumes a smaller one
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <int L, bool CAND>
static cudaError_t launch_lc(const CUtensorMap *tmap, const OlsArgs &a, int nseg, cudaStream_t s)
{
    auto kern = ols_fp32_kernel<L, minb<L>(), CAND>;
    constexpr size_t smem = Smem<L>::total + (CAND ? kCandSmem : 0);
    static bool done[64] = {};
    cudaError_t e = set_smem_attr<L>((const void *)kern, done, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nseg, (a.M + a.G - 1) / a.G);
    kern<<<grid, L / 16, smem, s>>>(*tmap, a);
    return cudaGetLastError();
}

template <int L>
static cudaError_t launch_l(const CUtensorMap *tmap, const OlsArgs &a, int nseg, cudaStream_t s)
{
    return a.cand ? launch_lc<L, true>(tmap, a, nseg, s) : launch_lc<L, false>(tmap, a, nseg, s);
}

cudaError_t launch_ols_fp32(int L, const CUtensorMap *tmap, const OlsArgs &a, int nseg, cudaStream_t s)
{
    switch (L) {
    case 1024: return launch_l<1024>(tmap, a, nseg, s);
    case 2048: return launch_l<2048>(tmap, a, nseg, s);
    case 4096: return launch_l<4096>(tmap, a, nseg, s);
    default: return cudaErrorInvalidValue;
    }
}

// Blocks per SM from the kernel's own resource use (registers, shared memory, threads and
// TMEM columns).  The persistent kernel's blocks never wait for one another, so a grid larger
// than what fits at once is still correct; the count only has to fill the GPU.
template <int L>
static cudaError_t batch_kernel_l(BatchKernel *k)
{
    auto kern = ols_fp32_batch<L, batch_minb<L>()>;
    static bool done[64] = {};
    cudaError_t e = set_smem_attr<L>((const void *)kern, done);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    int dev = 0;
    if ((e = cudaFuncGetAttributes(&fa, (const void *)kern)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    cudaDeviceProp pr;
    if ((e = cudaGetDeviceProperties(&pr, dev)) != cudaSuccess) return e;
    const int threads = L / 16, warps = threads / 32;
    const int regs_per_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = pr.regsPerMultiprocessor / (warps * regs_per_warp);
    const size_t smem_block = Smem<L>::total + fa.sharedSizeBytes + pr.reservedSharedMemPerBlock;
    const int by_smem = (int)(pr.sharedMemPerMultiprocessor / smem_block);
    const int by_threads = pr.maxThreadsPerMultiProcessor / threads;
    const int by_tmem = 512 / (int)kTmemCols<L>;
    int per_sm = by_regs;
    per_sm = per_sm < by_smem ? per_sm : by_smem;
    per_sm = per_sm < by_threads ? per_sm : by_threads;
    per_sm = per_sm < by_tmem ? per_sm : by_tmem;
    per_sm = per_sm < pr.maxBlocksPerMultiProcessor ? per_sm : pr.maxBlocksPerMultiProcessor;
    if (per_sm < 1) per_sm = 1;
    k->fn = (const void *)kern;
    k->block = threads;
    k->smem = Smem<L>::total;
    k->resident = per_sm * pr.multiProcessorCount;
    return cudaSuccess;
}

cudaError_t batch_kernel(int L, BatchKernel *k)
{
    switch (L) {
    case 1024: return batch_kernel_l<1024>(k);
    case 2048: return batch_kernel_l<2048>(k);
    case 4096: return batch_kernel_l<4096>(k);
    default: return cudaErrorInvalidValue;
    }
}

size_t ols_fp32_smem_bytes(int L)
{
    switch (L) {
    case 1024: return Smem<1024>::total;
    case 2048: return Smem<2048>::total;
    case 4096: return Smem<4096>::total;
    default: return 0;
    }
}

}  // namespace fdas
