// pw_dadd.cuh -- binary64 addition rounded to nearest even, done in 32-bit
// integer operations, so that a kernel bound by GB300's FP64 pipe (about two
// FP64 lane operations per clock per SM) can move part of its additions to
// the integer ALU, which it otherwise leaves mostly idle. It costs about 80
// instructions (about 60 on the ALU pipe) where the FP64 unit takes one, so
// it pays only where the FP64 pipe is the bottleneck and the issue slots are
// not: the perturbation pass of pw_split_field hands it one subtraction in
// eight.
//
// dadd_int(x, y, &r) forms r = x + y exactly as IEEE 754 binary64 addition
// with round-to-nearest-even does, for the operands it accepts: both normal
// (not zero, subnormal, infinite or NaN), the result normal and nonzero. It
// returns false for any other case and the caller then adds in FP64. The
// steps are the textbook ones for a floating-point adder: order the operands
// by magnitude, align the smaller significand to the larger exponent keeping
// the bits shifted out as a sticky bit, add or subtract, normalise, round to
// 53 bits (ties to even), and pack sign, exponent and fraction. Every step
// uses 32-bit words; no 64-bit integer type appears, since the compiler may
// lower 64-bit comparisons of a double's bit pattern to FP64 instructions.
//
// The same code compiles for the host, where tests compare it with the
// host's own binary64 addition.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PW_HD __host__ __device__ __forceinline__
#else
#define PW_HD inline
#endif

namespace pw {
namespace dadd_detail {

PW_HD uint32_t hi_word(double x) {
#if defined(__CUDA_ARCH__)
    return static_cast<uint32_t>(__double2hiint(x));
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return static_cast<uint32_t>(b >> 32);
#endif
}

PW_HD uint32_t lo_word(double x) {
#if defined(__CUDA_ARCH__)
    return static_cast<uint32_t>(__double2loint(x));
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return static_cast<uint32_t>(b);
#endif
}

PW_HD double from_words(uint32_t h, uint32_t l) {
#if defined(__CUDA_ARCH__)
    return __hiloint2double(static_cast<int>(h), static_cast<int>(l));
#else
    const uint64_t b = (static_cast<uint64_t>(h) << 32) | l;
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

// Shifts for counts 0..31 (callers keep them in range).
PW_HD uint32_t shl(uint32_t x, uint32_t n) { return n < 32u ? x << n : 0u; }
PW_HD uint32_t shr(uint32_t x, uint32_t n) { return n < 32u ? x >> n : 0u; }

// Low word of (hi:lo) >> n for n in 0..31.
PW_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t n) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, n);
#else
    return n == 0u ? lo : (lo >> n) | (hi << (32u - n));
#endif
}

// High word of (hi:lo) << n for n in 0..31.
PW_HD uint32_t funnel_l(uint32_t lo, uint32_t hi, uint32_t n) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, n);
#else
    return n == 0u ? hi : (hi << n) | (lo >> (32u - n));
#endif
}

PW_HD uint32_t clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return static_cast<uint32_t>(__clz(static_cast<int>(x)));
#else
    uint32_t n = 0;
    if (x == 0) return 32u;
    while (!(x & 0x80000000u)) {
        x <<= 1;
        ++n;
    }
    return n;
#endif
}

}  // namespace dadd_detail

PW_HD bool dadd_int(double x, double y, double* r) {
    using namespace dadd_detail;
    const uint32_t xh = hi_word(x), xl = lo_word(x), yh = hi_word(y), yl = lo_word(y);
    // A: the operand of larger magnitude (its sign is the result's)
    const uint32_t xm = xh & 0x7FFFFFFFu, ym = yh & 0x7FFFFFFFu;
    const bool swap = (ym > xm) || (ym == xm && yl > xl);
    const uint32_t ah = swap ? yh : xh, al = swap ? yl : xl;
    const uint32_t bh = swap ? xh : yh, bl = swap ? xl : yl;
    const uint32_t ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu;
    bool ok = (ea - 1u < 2046u) && (eb - 1u < 2046u);
    const bool sub = ((ah ^ bh) >> 31) != 0u;
    // significands with their leading 1, shifted up by 10: bits 62..10 of a
    // 64-bit word (hi:lo), so that alignment and normalisation keep guard bits
    const uint32_t Ah = (((ah & 0xFFFFFu) | 0x100000u) << 10) | (al >> 22), Al = al << 10;
    const uint32_t Bh = (((bh & 0xFFFFFu) | 0x100000u) << 10) | (bl >> 22), Bl = bl << 10;
    // B >> d, and whether any bit was shifted out
    const uint32_t d = ea - eb;  // >= 0
    uint32_t Sh, Sl, lost;
    if (d < 32u) {
        Sh = shr(Bh, d);
        Sl = funnel_r(Bl, Bh, d);
        lost = shl(Bl, 32u - d);
    } else if (d < 64u) {
        Sh = 0u;
        Sl = shr(Bh, d - 32u);
        lost = Bl | shl(Bh, 64u - d);
    } else {
        Sh = 0u;
        Sl = 0u;
        lost = 1u;  // B is nonzero
    }
    const uint32_t st = lost != 0u ? 1u : 0u;
    // R = A + S, or A - S - st (the bits lost below make the exact value
    // R + a fraction in (0, 1) either way; st keeps that fraction)
    uint32_t Rh, Rl;
    if (!sub) {
        Rl = Al + Sl;
        Rh = Ah + Sh + (Rl < Al ? 1u : 0u);
    } else {
        const uint32_t t = Sl + st;  // S + st < A, and S + st fits 64 bits
        const uint32_t th = Sh + (t < Sl ? 1u : 0u);
        Rl = Al - t;
        Rh = Ah - th - (Al < t ? 1u : 0u);
    }
    ok = ok && (Rh | Rl) != 0u;
    // normalise: leading 1 to bit 63 of (Rh:Rl)
    const uint32_t lz = Rh != 0u ? clz32(Rh) : 32u + clz32(Rl);
    uint32_t Nh, Nl;
    if (lz < 32u) {
        Nh = funnel_l(Rl, Rh, lz);
        Nl = shl(Rl, lz);
    } else {
        Nh = shl(Rl, lz - 32u);
        Nl = 0u;
    }
    // exponent of the leading bit: A's leading 1 sat at bit 62
    const int e = static_cast<int>(ea) + 1 - static_cast<int>(lz);
    // keep bits 63..11 (53 bits); bit 10 is the round bit
    const uint32_t guard = (Nl >> 10) & 1u, rest = (Nl & 0x3FFu) | st, lsb = (Nl >> 11) & 1u;
    const uint32_t inc = guard & ((rest != 0u ? 1u : 0u) | lsb);
    uint32_t Ml = funnel_r(Nl, Nh, 11u), Mh = Nh >> 11;  // leading 1 at bit 52 (Mh bit 20)
    Ml += inc;
    Mh += (Ml < inc) ? 1u : 0u;
    // pack: the leading 1 adds one to the exponent field, hence e - 1; a
    // carry out of rounding (M = 2^53) moves the exponent up by itself
    const uint32_t h = (ah & 0x80000000u) + (static_cast<uint32_t>(e - 1) << 20) + Mh;
    const uint32_t ef = (h >> 20) & 0x7FFu;
    ok = ok && e >= 1 && (ef - 1u < 2046u);
    *r = from_words(h, Ml);
    return ok;
}

}  // namespace pw

#undef PW_HD
