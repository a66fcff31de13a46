// pw_pair.cuh -- paired-FP32 ("double-float") arithmetic on sm_103a.
//
// A value is carried as an unevaluated sum h + l of two floats (about 48
// significant bits). Sums use Knuth's TwoSum (TAOCP vol. 2, 4.2.2) on the
// high parts, products the FMA form of Dekker's exact product (Dekker 1971):
// p = a*b, e = fma(a, b, -p) gives a*b = p + e exactly. Pairs are kept
// unnormalised ("sloppy" double-float): the low-part arithmetic rounds in
// FP32, so every operation's error is at most a few units of 2^-48 of the
// magnitudes of its operands -- the scale against which the library states
// its accuracy (the sum of the absolute product terms at a point).
//
// Conversions between double and pairs use integer bit operations only:
// on sm_103a a conversion to or from FP64 issues on the FP64 pipe (about two
// per clock per SM), which would cap the kernel far below the memory bound.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pw {

struct pf {
    float h, l;
};

__device__ __forceinline__ pf two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ pf padd(pf a, pf b) {
    pf s = two_sum(a.h, b.h);
    s.l += a.l + b.l;
    return s;
}

__device__ __forceinline__ pf psub(pf a, pf b) {
    pf s = two_sum(a.h, -b.h);
    s.l += a.l - b.l;
    return s;
}

__device__ __forceinline__ pf pmul(pf a, pf b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return {p, e};
}

// Split a double into (h, l): h = d rounded to 24 significant bits (ties
// away from zero), l = float(d - h). |d - (h + l)| <= 2^-49 |d|. Valid for
// 2^-74 <= |d| < 2^128; zero and smaller magnitudes give (0, 0). The words
// are read as 32-bit integers: tests written on the 64-bit pattern can be
// turned into FP64 comparisons by the compiler.
__device__ __forceinline__ pf split_double(double d) {
    const unsigned hw = static_cast<unsigned>(__double2hiint(d));
    const unsigned lw = static_cast<unsigned>(__double2loint(d));
    // the high-word term moves the exponent bias from 1023 to 127 (896 << 20);
    // h rounds up when the 29 dropped bits are at least half its last unit
    const unsigned up = (lw >> 28) & 1u;
    const unsigned hb = (__funnelshift_l(lw, hw + 0xC8000000u, 3) + up) | (hw & 0x80000000u);
    // the dropped bits as a signed count of d's last-bit unit (minus 2^29 when h rounded up)
    const int rem = static_cast<int>(lw << 3) >> 3;
    const unsigned ex = hw & 0x7FF00000u;
    // +-2^(E - 1075) (E = d's biased exponent): the weight of d's last bit
    const unsigned sb = ((ex - (948u << 20)) << 3) | (hw & 0x80000000u);
    const float hi = __uint_as_float(hb);
    const float lo = __int2float_rn(rem) * __uint_as_float(sb);
    const bool tiny = ex < (949u << 20);
    return {tiny ? 0.0f : hi, tiny ? 0.0f : lo};
}

// Exact float -> double by bit operations (normal floats and zero).
__device__ __forceinline__ double float_bits_to_double(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned mag = b & 0x7FFFFFFFu;
    const unsigned sign = b & 0x80000000u;
    const unsigned hi = mag ? (((mag >> 3) + (896u << 20)) | sign) : sign;
    const unsigned lo = b << 29;
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// h + l rounded once to double (one FP64 add).
__device__ __forceinline__ double pair_to_double(pf a) {
    return float_bits_to_double(a.h) + float_bits_to_double(a.l);
}

}  // namespace pw

// ---------------------------------------------------------------------------
// Packed pairs: two independent paired values in the lanes of float2s
// (h = (h0, h1), l = (l0, l1)), evaluated with the sm_100+ f32x2 add, mul
// and fma. Each lane rounds exactly as the scalar operations above, so a
// packed evaluation gives the scalar results bit for bit in half the issued
// instructions.
namespace pw {

struct pf2 {
    float2 h, l;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ pf2 two_sum2(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    const float2 e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
    return {s, e};
}

__device__ __forceinline__ pf2 padd2(pf2 a, pf2 b) {
    pf2 s = two_sum2(a.h, b.h);
    s.l = __fadd2_rn(s.l, __fadd2_rn(a.l, b.l));
    return s;
}

__device__ __forceinline__ pf2 psub2(pf2 a, pf2 b) {
    pf2 s = two_sum2(a.h, neg2(b.h));
    s.l = __fadd2_rn(s.l, __fadd2_rn(a.l, neg2(b.l)));
    return s;
}

__device__ __forceinline__ pf2 pmul2(pf2 a, pf2 b) {
    const float2 p = __fmul2_rn(a.h, b.h);
    float2 e = __ffma2_rn(a.h, b.h, neg2(p));
    e = __ffma2_rn(a.h, b.l, e);
    e = __ffma2_rn(a.l, b.h, e);
    return {p, e};
}

// The same pair in both lanes.
__device__ __forceinline__ pf2 dup2(pf a) { return {make_float2(a.h, a.h), make_float2(a.l, a.l)}; }

}  // namespace pw
