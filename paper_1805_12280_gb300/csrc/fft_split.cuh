// Split-pair arithmetic for the pass-C' groups of the tensor-core segment kernel: two complex
// values a, b held as re = (a.x, b.x), im = (a.y, b.y), so that every lane-wise operation,
// multiplications included, is one packed FP32x2 instruction; and the TMEM column order that
// stores a thread's 16 values as such pairs.
#pragma once
#include "fft_regs.cuh"
#include "tmem.cuh"

namespace fdas {

__device__ __forceinline__ float2 pmul(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// (re, im) *= (wr, wi) for both lanes: re wr - im wi, re wi + im wr.
__device__ __forceinline__ void cmul_split(float2 &re, float2 &im, float2 wr, float2 wi)
{
    const float2 r = csub(pmul(re, wr), pmul(im, wi));
    im = pfma(re, wi, pmul(im, wr));
    re = r;
}

// 4-point DFT of both lanes (natural order in and out).
template <int DIR>
__device__ __forceinline__ void dft4_split(float2 &r0, float2 &i0, float2 &r1, float2 &i1, float2 &r2, float2 &i2,
                                           float2 &r3, float2 &i3)
{
    const float2 t0r = cadd(r0, r2), t0i = cadd(i0, i2), t1r = csub(r0, r2), t1i = csub(i0, i2);
    const float2 t2r = cadd(r1, r3), t2i = cadd(i1, i3), dr = csub(r1, r3), di = csub(i1, i3);
    r0 = cadd(t0r, t2r);
    i0 = cadd(t0i, t2i);
    r2 = csub(t0r, t2r);
    i2 = csub(t0i, t2i);
    // outputs 1 and 3: t1 +- DIR i d, i d = (-di, dr)
    if constexpr (DIR > 0) {
        r1 = csub(t1r, di); i1 = cadd(t1i, dr);
        r3 = cadd(t1r, di); i3 = csub(t1i, dr);
    } else {
        r1 = cadd(t1r, di); i1 = csub(t1i, dr);
        r3 = csub(t1r, di); i3 = cadd(t1i, dr);
    }
}

// (re, im) *= exp(DIR 2 pi i e / 16) for e in {2, 6, 10, 14}, both lanes.
template <int E, int DIR>
__device__ __forceinline__ void rot8_split(float2 &re, float2 &im)
{
    constexpr float r = kC8[2];
    constexpr float cr = (E == 2 || E == 14) ? r : -r;
    constexpr float si0 = (E == 2 || E == 6) ? r : -r;
    constexpr float si = DIR < 0 ? -si0 : si0;
    const float2 c2 = make_float2(cr, cr);
    if constexpr (cr == si) {   // cr (re - im, re + im)
        const float2 d = csub(re, im), s = cadd(re, im);
        re = pmul(d, c2);
        im = pmul(s, c2);
    } else {                    // cr (re + im, im - re)
        const float2 s = cadd(re, im), d = csub(im, re);
        re = pmul(s, c2);
        im = pmul(d, c2);
    }
}

// Two 8-point DFTs in lockstep on split pairs: lane 0 transforms (re[c].x, im[c].x),
// lane 1 (re[c].y, im[c].y), c = 0..7 (same decomposition as dft<8>).
template <int DIR>
__device__ __forceinline__ void dft8x2_split(float2 (&re)[8], float2 (&im)[8])
{
    float2 er0 = re[0], ei0 = im[0], er1 = re[2], ei1 = im[2], er2 = re[4], ei2 = im[4], er3 = re[6], ei3 = im[6];
    float2 or0 = re[1], oi0 = im[1], or1 = re[3], oi1 = im[3], or2 = re[5], oi2 = im[5], or3 = re[7], oi3 = im[7];
    dft4_split<DIR>(er0, ei0, er1, ei1, er2, ei2, er3, ei3);
    dft4_split<DIR>(or0, oi0, or1, oi1, or2, oi2, or3, oi3);
    rot8_split<2, DIR>(or1, oi1);
    rot8_split<6, DIR>(or3, oi3);
    re[0] = cadd(er0, or0); im[0] = cadd(ei0, oi0); re[4] = csub(er0, or0); im[4] = csub(ei0, oi0);
    re[1] = cadd(er1, or1); im[1] = cadd(ei1, oi1); re[5] = csub(er1, or1); im[5] = csub(ei1, oi1);
    // o2 enters times DIR i: e2 +- DIR i o2, i o2 = (-oi2, or2)
    if constexpr (DIR > 0) {
        re[2] = csub(er2, oi2); im[2] = cadd(ei2, or2); re[6] = cadd(er2, oi2); im[6] = csub(ei2, or2);
    } else {
        re[2] = cadd(er2, oi2); im[2] = csub(ei2, or2); re[6] = csub(er2, oi2); im[6] = cadd(ei2, or2);
    }
    re[3] = cadd(er3, or3); im[3] = cadd(ei3, oi3); re[7] = csub(er3, or3); im[7] = csub(ei3, oi3);
}

// 16 complex values, slots j and 8 + j as split pairs: columns 4j .. 4j+3 hold
// (v[j].x, v[8+j].x, v[j].y, v[8+j].y), so that a load returns (re, im) pairs directly.
__device__ __forceinline__ void tmem_st_split16(uint32_t taddr, const float2 (&v)[16])
{
    uint32_t r[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        r[4 * j] = __float_as_uint(v[j].x);
        r[4 * j + 1] = __float_as_uint(v[8 + j].x);
        r[4 * j + 2] = __float_as_uint(v[j].y);
        r[4 * j + 3] = __float_as_uint(v[8 + j].y);
    }
    tmem_st32(taddr, r);
}

__device__ __forceinline__ void split_from_cols(const uint32_t (&r)[32], float2 (&re)[8], float2 (&im)[8])
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        re[j] = make_float2(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]));
        im[j] = make_float2(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
    }
}

}  // namespace fdas
