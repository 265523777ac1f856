// Register-resident small DFTs (2, 4, 8, 16 points) for the FP32 segment kernel.
//
// DIR = -1 gives the forward transform X[k] = sum_n x[n] exp(-2 pi i nk / R),
// DIR = +1 the unnormalised inverse.  Inputs and outputs are in natural order.
// Every twiddle here is a compile-time multiple of exp(2 pi i / 16); trivial ones
// (1, -1, +-i, (+-1 +- i)/sqrt 2) are applied without general multiplies.
#pragma once
#include <cuda_runtime.h>

namespace fdas {

// Complex add and subtract as one packed FP32x2 instruction each (sm_100 family): both
// lanes round exactly as two scalar operations would.
__device__ __forceinline__ float2 cadd(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a + S i b for S = +-1, in scalar form: the lane swap of i b would cost moves in packed form.
template <int S>
__device__ __forceinline__ float2 cadd_i(float2 a, float2 b)
{
    return S > 0 ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// cos(j pi / 8), j = 0..4
constexpr float kC8[5] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f,
                          0.38268343236508977173f, 0.0f};

// a * exp(DIR * 2 pi i * E / N) for compile-time E and N with N dividing 16.
template <int E, int N, int DIR>
__device__ __forceinline__ float2 twc(float2 a)
{
    constexpr int e = ((E * (16 / N)) % 16 + 16) % 16;   // angle in units of 2 pi / 16
    if constexpr (e == 0) {
        return a;
    } else if constexpr (e == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (e == 4) {                       // exp(DIR i pi/2) = DIR i
        return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else if constexpr (e == 12) {                      // -DIR i
        return DIR < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
        // (cr + i si) with |cr| = |si| = 1/sqrt 2
        constexpr float r = kC8[2];
        constexpr float cr = (e == 2 || e == 14) ? r : -r;
        constexpr float si0 = (e == 2 || e == 6) ? r : -r;   // sin for DIR = +1
        constexpr float si = DIR < 0 ? -si0 : si0;
        // (a.x + i a.y)(cr + i si)
        if constexpr (cr == si) {
            return make_float2(cr * (a.x - a.y), cr * (a.x + a.y));
        } else {
            return make_float2(cr * (a.x + a.y), cr * (a.y - a.x));
        }
    } else {
        // general multiple of pi/8
        constexpr int q = e % 8;                           // 1, 3, 5, 7
        constexpr float c_abs = (q == 1 || q == 7) ? kC8[1] : kC8[3];
        constexpr float s_abs = (q == 1 || q == 7) ? kC8[3] : kC8[1];
        constexpr float cr = (e < 4 || e > 12) ? c_abs : -c_abs;
        constexpr float si0 = (e < 8) ? s_abs : -s_abs;
        constexpr float si = DIR < 0 ? -si0 : si0;
        return make_float2(fmaf(a.x, cr, -a.y * si), fmaf(a.x, si, a.y * cr));
    }
}

// 2-point
template <int DIR>
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1)
{
    float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

// 4-point, natural order in/out
template <int DIR>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const float2 t2 = cadd(a1, a3), d = csub(a1, a3);   // the odd part, times DIR i below
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd_i<DIR>(t1, d);
    a3 = cadd_i<-DIR>(t1, d);
}

// dft4 whose third input enters multiplied by DIR i (the exp(DIR i pi/2) twiddle of a
// radix-16 column): a2 is passed untwiddled.
template <int DIR>
__device__ __forceinline__ void dft4_i2(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = cadd_i<DIR>(a0, a2), t1 = cadd_i<-DIR>(a0, a2);
    const float2 t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd_i<DIR>(t1, d);
    a3 = cadd_i<-DIR>(t1, d);
}

namespace detail {
template <int R, int DIR, int ST, int OFF>
struct Dft;

template <int DIR, int ST, int OFF>
struct Dft<2, DIR, ST, OFF> {
    static __device__ __forceinline__ void run(float2 *v) { dft2<DIR>(v[OFF], v[OFF + ST]); }
};

template <int DIR, int ST, int OFF>
struct Dft<4, DIR, ST, OFF> {
    static __device__ __forceinline__ void run(float2 *v)
    {
        dft4<DIR>(v[OFF], v[OFF + ST], v[OFF + 2 * ST], v[OFF + 3 * ST]);
    }
};

// 8 = 4 x 2 (even/odd split)
template <int DIR, int ST, int OFF>
struct Dft<8, DIR, ST, OFF> {
    static __device__ __forceinline__ void run(float2 *v)
    {
        // n = 2 n1 + n2 (n1 < 4, n2 < 2); k = k1 + 4 k2 (k1 < 4, k2 < 2)
        float2 e0 = v[OFF + 0 * ST], e1 = v[OFF + 2 * ST], e2 = v[OFF + 4 * ST], e3 = v[OFF + 6 * ST];
        float2 o0 = v[OFF + 1 * ST], o1 = v[OFF + 3 * ST], o2 = v[OFF + 5 * ST], o3 = v[OFF + 7 * ST];
        dft4<DIR>(e0, e1, e2, e3);
        dft4<DIR>(o0, o1, o2, o3);
        o1 = twc<1, 8, DIR>(o1);
        o3 = twc<3, 8, DIR>(o3);
        v[OFF + 0 * ST] = cadd(e0, o0); v[OFF + 4 * ST] = csub(e0, o0);
        v[OFF + 1 * ST] = cadd(e1, o1); v[OFF + 5 * ST] = csub(e1, o1);
        // o2 enters times exp(DIR i pi/2) = DIR i
        v[OFF + 2 * ST] = cadd_i<DIR>(e2, o2); v[OFF + 6 * ST] = cadd_i<-DIR>(e2, o2);
        v[OFF + 3 * ST] = cadd(e3, o3); v[OFF + 7 * ST] = csub(e3, o3);
    }
};

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
template <int DIR, int ST, int OFF>
struct Dft<16, DIR, ST, OFF> {
    static __device__ __forceinline__ void run(float2 *v)
    {
        float2 a[4][4];   // a[n2][k1]
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            a[n2][0] = v[OFF + (0 + n2) * ST];
            a[n2][1] = v[OFF + (4 + n2) * ST];
            a[n2][2] = v[OFF + (8 + n2) * ST];
            a[n2][3] = v[OFF + (12 + n2) * ST];
            dft4<DIR>(a[n2][0], a[n2][1], a[n2][2], a[n2][3]);
        }
        a[1][1] = twc<1, 16, DIR>(a[1][1]);
        a[1][2] = twc<2, 16, DIR>(a[1][2]);
        a[1][3] = twc<3, 16, DIR>(a[1][3]);
        a[2][1] = twc<2, 16, DIR>(a[2][1]);
        a[2][3] = twc<6, 16, DIR>(a[2][3]);   // a[2][2] enters times DIR i inside dft4_i2
        a[3][1] = twc<3, 16, DIR>(a[3][1]);
        a[3][2] = twc<6, 16, DIR>(a[3][2]);
        a[3][3] = twc<9, 16, DIR>(a[3][3]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            if (k1 == 2) dft4_i2<DIR>(a[0][k1], a[1][k1], a[2][k1], a[3][k1]);
            else dft4<DIR>(a[0][k1], a[1][k1], a[2][k1], a[3][k1]);
            v[OFF + (k1 + 0) * ST] = a[0][k1];
            v[OFF + (k1 + 4) * ST] = a[1][k1];
            v[OFF + (k1 + 8) * ST] = a[2][k1];
            v[OFF + (k1 + 12) * ST] = a[3][k1];
        }
    }
};
}  // namespace detail

// R-point DFT in place on v[OFF + ST*j], j = 0..R-1 (R in {2, 4, 8, 16}).
template <int R, int DIR, int ST = 1, int OFF = 0>
__device__ __forceinline__ void dft(float2 *v) { detail::Dft<R, DIR, ST, OFF>::run(v); }

}  // namespace fdas
