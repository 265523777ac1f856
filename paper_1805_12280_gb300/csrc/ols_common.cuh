// Forward segment FFT shared by the FP32 and tensor-core segment kernels.
#pragma once
#include "fdas_internal.cuh"
#include "fft_regs.cuh"

namespace fdas {

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Barrier between the passes of a transform: the whole block by default; kernels whose
// transform runs in one warp group pass a named-barrier policy.
struct BlockSync {
    static __device__ __forceinline__ void sync() { __syncthreads(); }
};

// Forward L-point FFT of the segment in `src` (natural order; e1 or another buffer) by the
// NT = L/16 threads of a block: passes A and B exchange through e2 and e1, pass C leaves the
// spectrum in X ("C distribution": slot g*R + k3 of thread t holds X[k1 + 16 k2 + 16 Q k3]
// with k1 = t % 16, k2 = t / 16 + (NT/16) g).  `after_a` runs in every thread after the
// barrier that follows pass A, when no thread reads `src` any more.  Ends before the barrier
// that must follow it.
template <int L, class Hook = NoHook, class Sync = BlockSync>
__device__ __forceinline__ void forward_fft(const float2 *src, float2 *e1, float2 *e2, const float2 *__restrict__ tw,
                                            float2 (&v)[16], float2 (&X)[16], Hook after_a = Hook())
{
    using Gm = Geo<L>;
    constexpr int NT = Gm::NT, Q = Gm::Q, R = Gm::R, GB = Gm::GB, GC = Gm::GC, LD2 = Gm::LD2;
    constexpr int MASK = L - 1;
    const int tid = threadIdx.x, k1 = tid & 15, hi = tid >> 4;
    // ---- forward pass A: 16-point DFT over the top digit, twiddle W_L^{t k1}
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = src[j * NT + tid];
    dft<16, -1>(v);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], __ldg(&tw[(tid * k) & MASK]));
#pragma unroll
    for (int k = 0; k < 16; ++k) e2[tid + LD2 * k] = v[k];
    Sync::sync();
    after_a();
    // ---- forward pass B: Q-point DFT over b, twiddle W_{QR}^{c k2}
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int cg = hi + (NT / 16) * g;
#pragma unroll
        for (int b = 0; b < Q; ++b) v[g * Q + b] = e2[(b * R + cg) + LD2 * k1];
    }
    dft<Q, -1, 1, 0>(v);
    if constexpr (GB == 2) dft<Q, -1, 1, Q>(v);
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int cg = hi + (NT / 16) * g;
        if constexpr (GC == 2) {
            // k2 and k2 + Q/2 share one 16-byte slot, k1 + 16 (k2 mod Q/2) + 8 Q c: pass C
            // holds both and reads them with one load
            static_assert(NT / 16 == Q / 2, "paired exchange layout");
            float4 *e1q = reinterpret_cast<float4 *>(e1);
#pragma unroll
            for (int k2 = 0; k2 < Q / 2; ++k2) {
                const float2 w0 = (k2 == 0) ? make_float2(1.f, 0.f) : __ldg(&tw[(16 * cg * k2) & MASK]);
                const float2 w1 = __ldg(&tw[(16 * cg * (k2 + Q / 2)) & MASK]);
                const float2 u0 = (k2 == 0) ? v[g * Q] : cmul(v[g * Q + k2], w0);
                const float2 u1 = cmul(v[g * Q + k2 + Q / 2], w1);
                e1q[k1 + 16 * k2 + 8 * Q * cg] = make_float4(u0.x, u0.y, u1.x, u1.y);
            }
        } else {
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) {
                const float2 w = (k2 == 0) ? make_float2(1.f, 0.f) : __ldg(&tw[(16 * cg * k2) & MASK]);
                e1[k1 + 16 * k2 + 16 * Q * cg] = cmul(v[g * Q + k2], w);
            }
        }
    }
    Sync::sync();
    // ---- forward pass C: R-point DFT over c; spectrum stays in registers
    if constexpr (GC == 2) {
        const float4 *e1q = reinterpret_cast<const float4 *>(e1);
#pragma unroll
        for (int c = 0; c < R; ++c) {
            const float4 w = e1q[k1 + 16 * hi + 8 * Q * c];
            X[c] = make_float2(w.x, w.y);
            X[R + c] = make_float2(w.z, w.w);
        }
    } else {
#pragma unroll
        for (int c = 0; c < R; ++c) X[c] = e1[k1 + 16 * hi + 16 * Q * c];
    }
    dft<R, -1, 1, 0>(X);
    if constexpr (GC == 2) dft<R, -1, 1, R>(X);
}

// Inverse L-point FFT (unnormalised, exp(+2 pi i nk / L)) by the NT = L/16 threads of a
// block, from the C distribution the forward transform leaves (slot j of thread t holds
// X[freq_of_slot(L, t, j)]) to natural order: on return v[a] = y[a*NT + t].  Passes C', B', A'
// with conjugate twiddles read from the table; e1 and e2 must be free on entry (a barrier
// after their last use) and are in use until the caller's next barrier.
template <int L>
__device__ __forceinline__ void inverse_fft(float2 (&v)[16], float2 *e1, float2 *e2, const float2 *__restrict__ tw)
{
    using Gm = Geo<L>;
    constexpr int NT = Gm::NT, Q = Gm::Q, R = Gm::R, GB = Gm::GB, GC = Gm::GC, LD2 = Gm::LD2;
    constexpr int MASK = L - 1;
    const int tid = threadIdx.x, k1 = tid & 15, hi = tid >> 4;
    // ---- pass C': R-point IDFT over k3, twiddle conj W_{QR}^{c k2}; exchange through e1
    dft<R, 1, 1, 0>(v);
    if constexpr (GC == 2) dft<R, 1, 1, R>(v);
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const int k2 = hi + (NT / 16) * g;
#pragma unroll
        for (int c = 0; c < R; ++c)
            e1[k1 + 16 * k2 + 16 * Q * c] = (c == 0) ? v[g * R] : cmul(v[g * R + c], cconj(__ldg(&tw[(16 * c * k2) & MASK])));
    }
    __syncthreads();
    // ---- pass B': Q-point IDFT over k2, twiddle conj W_L^{(bR + c) k1}; exchange through e2
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int cg = hi + (NT / 16) * g;
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[g * Q + k2] = e1[k1 + 16 * k2 + 16 * Q * cg];
    }
    dft<Q, 1, 1, 0>(v);
    if constexpr (GB == 2) dft<Q, 1, 1, Q>(v);
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int cg = hi + (NT / 16) * g;
#pragma unroll
        for (int b = 0; b < Q; ++b)
            e2[(b * R + cg) + LD2 * k1] = cmul(v[g * Q + b], cconj(__ldg(&tw[((b * R + cg) * k1) & MASK])));
    }
    __syncthreads();
    // ---- pass A': 16-point IDFT over k1 -> natural order
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = e2[tid + LD2 * k];
    dft<16, 1>(v);
}

// The segment in e1.
template <int L>
__device__ __forceinline__ void forward_fft(float2 *e1, float2 *e2, const float2 *__restrict__ tw, float2 (&v)[16],
                                            float2 (&X)[16])
{
    forward_fft<L>(e1, e1, e2, tw, v, X);
}

}  // namespace fdas
