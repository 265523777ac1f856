// Harmonic summing of a power plane: the stage that receives the plane from the
// FT-convolution module (Sec. 3 names it; read here as the incoherent harmonic sum).
//
// Rows of the plane are ordered by drift, z = y - c with c = (m-1)/2, and column bin0
// holds frequency bin 0 (for templates centred in a frame of F taps, bin0 = (F-1)/2).
// The k-th harmonic of a signal at bin r with drift z lies at bin k r with drift k z, so for
// the fundamental (r, z), r >= 1,
//     S_h(r, z) = sum_{k=1..h} P[c + k z][bin0 + k r],      h = 1, 2, 4, .., H,
// is defined where |h z| <= c and bin0 + h r <= n - 1, and every S_h above its level's
// threshold becomes a candidate.
//
// A thread takes Q fundamentals of one row, 256 apart (Q H = 64 for H >= 8, Q = 8 below):
// all Q H loads of their harmonics are issued before the first is used (predicated on the
// harmonic lying inside the plane), then each sum is formed in the order k = 1, 2, .., the
// running sum compared with the threshold at every power of two.  A block takes tiles of
// 256 Q consecutive fundamentals of one row (the k = 1 loads of a warp are one 128-byte
// line; the k-th are a k-strided gather over k lines); in the 64-bit kernel its crossings
// are staged per block and reserved in the output with one atomic per tile.  The kernel is bound by
// instruction issue, so for planes narrower than 2^31 columns: rows are launched in runs of
// equal kz = min(H, c / |z|) (the harmonics whose drift lies in the plane), each run by a
// kernel compiled for exactly kz harmonics; each harmonic k has one base address per tile,
// the thread's Q loads sit at fixed offsets 256 k q from it, and the test "bin0 + k r inside
// the plane" is one 32-bit compare against r_lim[k] = (n-1-bin0)/k; crossings are staged per
// warp, with no block barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <utility>

#include "fdas_internal.cuh"

namespace fdas {
namespace {

constexpr int kHsThreads = 256;
constexpr int kHsStage = 256;                        // records staged per block and tile
constexpr int kHsMaxLevels = 6;                      // h = 1 .. 32

struct HsThresholds {
    float t[kHsMaxLevels];
};

struct HsLimits {   // r_lim[k] = (n - 1 - bin0) / k: harmonic k of r lies in the plane iff r <= r_lim[k]
    int r_lim[33];
};

// fundamentals per thread and tile: loads in flight per thread Q H = 64 (8 for H = 1)
template <int H>
__host__ __device__ constexpr int hs_per_thread()
{
    return H <= 8 ? 8 : 64 / H;
}

template <int H>
__global__ void __launch_bounds__(kHsThreads) harmonic_kernel(const float *__restrict__ P, int m, int64_t n,
                                                              int64_t bin0, int64_t tiles_per_row, HsThresholds thr,
                                                              fdas_harmonic_candidate *__restrict__ out,
                                                              int64_t max_cand, unsigned long long *__restrict__ count)
{
    constexpr int Q = hs_per_thread<H>();
    constexpr int64_t TILE = (int64_t)kHsThreads * Q;
    __shared__ fdas_harmonic_candidate stage[kHsStage];
    __shared__ unsigned n_staged, n_flush;
    __shared__ unsigned long long flush_base;
    const int c = (m - 1) / 2;
    const int64_t rmax = n - 1 - bin0;   // fundamentals r = 1 .. rmax
    const int64_t tiles = (int64_t)m * tiles_per_row;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int y = (int)(tile / tiles_per_row);
        const int z = y - c;
        const int az = z < 0 ? -z : z;
        const int kz = az == 0 ? H : min(H, c / az);   // harmonics whose drift k z lies in the plane
        const int64_t r0 = 1 + (tile - (int64_t)y * tiles_per_row) * TILE + threadIdx.x;
        const int64_t origin = (int64_t)c * n + bin0;   // cell of k = 0
        const int64_t step_z = (int64_t)z * n;
        if (threadIdx.x == 0) n_staged = 0;
        __syncthreads();
        float v[Q][H];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t r = r0 + q * kHsThreads;
            const int64_t step = step_z + r;   // from harmonic k to k + 1
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const bool in = k <= kz && (int64_t)k * r <= rmax;   // r <= rmax is the case k = 1
                v[q][k - 1] = in ? __ldg(P + origin + (int64_t)k * step) : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t r = r0 + q * kHsThreads;
            float acc = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                acc += v[q][k - 1];
                if ((k & (k - 1)) == 0) {   // level h = k
                    const int j = 31 - __clz(k);
                    if (k <= kz && (int64_t)k * r <= rmax && acc > thr.t[j]) {
                        fdas_harmonic_candidate rec;
                        rec.tpl = y;
                        rec.power = acc;
                        rec.bin = bin0 + r;
                        rec.nharm = k;
                        rec.reserved = 0;
                        const unsigned slot = atomicAdd(&n_staged, 1u);
                        if (slot < (unsigned)kHsStage) {
                            stage[slot] = rec;
                        } else {   // staging full: reserve this record on its own
                            const unsigned long long at = atomicAdd(count, 1ull);
                            if ((long long)at < max_cand) out[at] = rec;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned ns = min(n_staged, (unsigned)kHsStage);
            n_flush = ns;
            flush_base = ns ? atomicAdd(count, (unsigned long long)ns) : 0ull;
        }
        __syncthreads();
        for (unsigned i = threadIdx.x; i < n_flush; i += kHsThreads)
            if ((long long)(flush_base + i) < max_cand) out[flush_base + i] = stage[i];
        __syncthreads();   // the stage is read before the next tile refills it
    }
}

// Planes of fewer than 2^31 columns: fundamentals, bins and the in-row offsets are 32-bit.
// Crossings are staged per warp (no block barrier: each warp runs its tiles at its own pace)
// and a warp reserves its staged records with one atomic once 32 or more are waiting.
constexpr int kWarpStage = 64, kWarpFlush = 32;

__device__ __forceinline__ void warp_flush(fdas_harmonic_candidate *stage, unsigned *n_staged, int lane,
                                           fdas_harmonic_candidate *__restrict__ out, int64_t max_cand,
                                           unsigned long long *__restrict__ count)
{
    const unsigned ns = min(*n_staged, (unsigned)kWarpStage);
    unsigned long long base = 0;
    if (lane == 0 && ns) base = atomicAdd(count, (unsigned long long)ns);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (unsigned i = lane; i < ns; i += 32)
        if ((long long)(base + i) < max_cand) out[base + i] = stage[i];
    __syncwarp();
    if (lane == 0) *n_staged = 0;
    __syncwarp();
}

// One launch per run of rows with the same number KZ = min(H, c / |z|) of harmonics inside
// the plane's drift range, compiled for exactly that many: no work on harmonics a row lacks.
template <int KZ>
__global__ void __launch_bounds__(kHsThreads, 2) harmonic_kernel_narrow(const float *__restrict__ P, int m, int n,
                                                                        int bin0, int y0, int nrows, int tiles_per_row,
                                                                        HsThresholds thr, HsLimits lim,
                                                                        fdas_harmonic_candidate *__restrict__ out,
                                                                        int64_t max_cand,
                                                                        unsigned long long *__restrict__ count)
{
    constexpr int H = KZ;
    constexpr int Q = hs_per_thread<H>();
    constexpr int TILE = kHsThreads * Q;
    __shared__ fdas_harmonic_candidate stage[kHsThreads / 32][kWarpStage];
    __shared__ unsigned n_staged[kHsThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the next run of rows reads the same plane and appends to the same list: nothing here
    // feeds it, so it may start as soon as this launch's blocks leave room
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (lane == 0) n_staged[warp] = 0;
    __syncwarp();
    const int c = (m - 1) / 2;
    const int64_t tiles = (int64_t)nrows * tiles_per_row;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int yr = (int)(tile / tiles_per_row);
        const int y = y0 + yr;
        const int z = y - c;
        const int r0 = 1 + (int)(tile - (int64_t)yr * tiles_per_row) * TILE + (int)threadIdx.x;
        float v[Q][H];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            // cell (c + k z, bin0 + k r0); read only where the harmonic lies in the plane
            const float *base = P + ((int64_t)(c + k * z) * n + bin0 + (int64_t)k * r0);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const bool in = r0 + q * kHsThreads <= lim.r_lim[k];
                v[q][k - 1] = in ? __ldg(base + k * kHsThreads * q) : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = r0 + q * kHsThreads;
            float acc = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                acc += v[q][k - 1];
                if ((k & (k - 1)) == 0) {   // level h = k
                    const int j = 31 - __clz(k);
                    if (r <= lim.r_lim[k] && acc > thr.t[j]) {
                        fdas_harmonic_candidate rec;
                        rec.tpl = y;
                        rec.power = acc;
                        rec.bin = bin0 + r;
                        rec.nharm = k;
                        rec.reserved = 0;
                        const unsigned slot = atomicAdd(&n_staged[warp], 1u);
                        if (slot < (unsigned)kWarpStage) {
                            stage[warp][slot] = rec;
                        } else {   // staging full: reserve this record on its own
                            const unsigned long long at = atomicAdd(count, 1ull);
                            if ((long long)at < max_cand) out[at] = rec;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (n_staged[warp] >= (unsigned)kWarpFlush) warp_flush(stage[warp], &n_staged[warp], lane, out, max_cand, count);
    }
    __syncwarp();
    if (n_staged[warp]) warp_flush(stage[warp], &n_staged[warp], lane, out, max_cand, count);
}

using NarrowKernel = void (*)(const float *, int, int, int, int, int, int, HsThresholds, HsLimits,
                              fdas_harmonic_candidate *, int64_t, unsigned long long *);

template <int... K>
constexpr std::array<NarrowKernel, sizeof...(K)> narrow_table(std::integer_sequence<int, K...>)
{
    return {&harmonic_kernel_narrow<K + 1>...};
}

// harmonic_kernel_narrow<KZ> for KZ = 1 .. 32
constexpr std::array<NarrowKernel, 32> kNarrow = narrow_table(std::make_integer_sequence<int, 32>{});

cudaError_t resident_grid(const void *fn, int64_t tiles, unsigned *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kHsThreads, 0)) != cudaSuccess) return e;
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (unsigned)(tiles < resident ? tiles : resident);
    return cudaSuccess;
}

cudaError_t launch_hs(int H, const float *P, int m, int64_t n, int64_t bin0, const HsThresholds &thr,
                      fdas_harmonic_candidate *out, int64_t max_cand, unsigned long long *count, cudaStream_t s)
{
    const int64_t rmax = n - 1 - bin0;
    const int c = (m - 1) / 2;
    cudaError_t e;
    unsigned grid = 0;
    // 32-bit fundamentals and bins, with room for the last tile's overhang past rmax
    if (n <= (((int64_t)1 << 31) - ((int64_t)1 << 16))) {
        HsLimits lim{};
        for (int k = 1; k <= 32; ++k) lim.r_lim[k] = (int)(rmax / k);
        auto kz_of = [&](int y) { const int az = std::abs(y - c); return az == 0 ? H : std::min(H, c / az); };
        for (int y0 = 0; y0 < m;) {   // runs of rows with the same kz
            const int kz = kz_of(y0);
            int y1 = y0 + 1;
            while (y1 < m && kz_of(y1) == kz) ++y1;
            const NarrowKernel fn = kNarrow[kz - 1];
            const int64_t tile = (int64_t)kHsThreads * (kz <= 8 ? 8 : 64 / kz);   // hs_per_thread<kz>()
            const int64_t tiles_per_row = (rmax + tile - 1) / tile;
            if ((e = resident_grid((const void *)fn, (int64_t)(y1 - y0) * tiles_per_row, &grid)) != cudaSuccess)
                return e;
            // launches after the first may overlap the one before (programmatic dependent launch):
            // the runs are independent, and the tail of one run fills with the next
            cudaLaunchAttribute attr{};
            attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr.val.programmaticStreamSerializationAllowed = 1;
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(kHsThreads);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = s;
            cfg.attrs = &attr;
            cfg.numAttrs = y0 > 0 ? 1 : 0;
            if ((e = cudaLaunchKernelEx(&cfg, fn, P, m, (int)n, (int)bin0, y0, y1 - y0, (int)tiles_per_row, thr, lim, out,
                                        max_cand, count)) != cudaSuccess)
                return e;
            y0 = y1;
        }
        return cudaSuccess;
    }
    const void *fn = nullptr;
    int64_t tile = 0;
    switch (H) {
    case 1: fn = (const void *)harmonic_kernel<1>; tile = kHsThreads * hs_per_thread<1>(); break;
    case 2: fn = (const void *)harmonic_kernel<2>; tile = kHsThreads * hs_per_thread<2>(); break;
    case 4: fn = (const void *)harmonic_kernel<4>; tile = kHsThreads * hs_per_thread<4>(); break;
    case 8: fn = (const void *)harmonic_kernel<8>; tile = kHsThreads * hs_per_thread<8>(); break;
    case 16: fn = (const void *)harmonic_kernel<16>; tile = kHsThreads * hs_per_thread<16>(); break;
    default: fn = (const void *)harmonic_kernel<32>; tile = kHsThreads * hs_per_thread<32>(); break;
    }
    const int64_t tiles_per_row = (rmax + tile - 1) / tile;
    if ((e = resident_grid(fn, (int64_t)m * tiles_per_row, &grid)) != cudaSuccess) return e;
    switch (H) {
    case 1: harmonic_kernel<1><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    case 2: harmonic_kernel<2><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    case 4: harmonic_kernel<4><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    case 8: harmonic_kernel<8><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    case 16: harmonic_kernel<16><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    default: harmonic_kernel<32><<<grid, kHsThreads, 0, s>>>(P, m, n, bin0, tiles_per_row, thr, out, max_cand, count); break;
    }
    return cudaGetLastError();
}

int hs_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return set_error(FDAS_ERR_CUDA, buf);
}

}  // namespace
}  // namespace fdas

extern "C" int fdas_harmonic_sum(const float *plane_dev, int n_templates, int64_t n, int64_t bin0, int max_harm,
                                 const float *thresholds, fdas_harmonic_candidate *cand_dev, int64_t max_cand,
                                 unsigned long long *count_dev, void *stream)
{
    using namespace fdas;
    if (!plane_dev || !count_dev || !thresholds || (max_cand > 0 && !cand_dev))
        return set_error(FDAS_ERR_INVALID_ARG, "null pointer");
    if (max_cand < 0) return set_error(FDAS_ERR_INVALID_ARG, "max_cand must be >= 0");
    if (n_templates < 1 || (n_templates & 1) == 0)
        return set_error(FDAS_ERR_INVALID_ARG, "n_templates must be odd (rows z = -c .. c)");
    if (n < 1 || bin0 < 0 || bin0 >= n) return set_error(FDAS_ERR_INVALID_ARG, "need n >= 1 and 0 <= bin0 < n");
    if (max_harm < 1 || max_harm > 32 || (max_harm & (max_harm - 1)))
        return set_error(FDAS_ERR_INVALID_ARG, "max_harm must be a power of two in [1, 32]");
    if (reinterpret_cast<uintptr_t>(plane_dev) % 4 || reinterpret_cast<uintptr_t>(count_dev) % 8 ||
        reinterpret_cast<uintptr_t>(cand_dev) % 8)
        return set_error(FDAS_ERR_INVALID_ARG, "misaligned plane, counter or candidate array");
    HsThresholds thr{};
    for (int j = 0; (1 << j) <= max_harm; ++j) thr.t[j] = thresholds[j];
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return hs_cuda(e, "clear candidate counter");
    if (n - 1 - bin0 < 1) return FDAS_OK;   // no fundamental r >= 1 inside the plane
    e = launch_hs(max_harm, plane_dev, n_templates, n, bin0, thr, cand_dev, max_cand, count_dev, s);
    if (e != cudaSuccess) return hs_cuda(e, "harmonic-sum launch");
    return FDAS_OK;
}
