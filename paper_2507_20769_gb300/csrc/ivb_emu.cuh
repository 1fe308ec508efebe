// ivb_emu.cuh -- directed-rounding binary64 multiply and add on the integer
// pipes, bit-identical to the FP64 instructions (__dmul_rd/_ru, __dadd_rd/_ru).
//
// GB300's FP64 pipe retires about two lanes per clock per SM, while the
// integer pipes retire tens; the pipes issue independently, so a kernel
// whose endpoint arithmetic keeps the FP64 pipe busy gains throughput when
// part of that arithmetic runs here instead (measured: hardware and
// emulated multiplies side by side reach 1.8x the hardware rate alone).
//
// Both operations follow the textbook construction of IEEE 754 arithmetic
// on integer significands: 53-bit significands with the hidden bit, exact
// 106-bit products from four 32x32->64 multiplies, alignment with the bits
// shifted out OR-ed ("jammed") into the lowest bit, normalisation, and
// rounding of the magnitude away from zero exactly when the discarded bits
// are nonzero and the rounding direction points away from zero (toward +inf
// for a positive result, toward -inf for a negative one). The packed result
// is sign | (E - 1) << 52 plus the 53-bit significand, so a carry out of the
// significand increments the exponent, and a carry out of the largest
// exponent gives the infinity that directed rounding away from zero requires.
// Operands or results outside the normal range (subnormals, infinities,
// NaNs, exponent overflow or underflow) take the FP64 instruction in an
// out-of-line function, which the compiler cannot hoist onto the fast path.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ivb {

static __device__ __noinline__ double mul_rd_hw(double x, double y) { return __dmul_rd(x, y); }
static __device__ __noinline__ double mul_ru_hw(double x, double y) { return __dmul_ru(x, y); }
static __device__ __noinline__ double add_rd_hw(double x, double y) { return __dadd_rd(x, y); }
static __device__ __noinline__ double add_ru_hw(double x, double y) { return __dadd_ru(x, y); }

// x * y rounded toward +inf (up) or -inf; ok = false when an operand is not
// a normal number or the exponent of the result leaves [1, 2046]
__device__ __forceinline__ double mul_dir_emu_fast(double x, double y, bool up, bool& ok) {
    const unsigned long long bx = (unsigned long long)bits(x), by = (unsigned long long)bits(y);
    const unsigned xh = (unsigned)(bx >> 32), xl = (unsigned)bx;
    const unsigned yh = (unsigned)(by >> 32), yl = (unsigned)by;
    const unsigned ex = (xh >> 20) & 0x7FFu, ey = (yh >> 20) & 0x7FFu;
    const unsigned sign = (xh ^ yh) & 0x80000000u;
    const unsigned mxh = (xh & 0xFFFFFu) | 0x100000u, myh = (yh & 0xFFFFFu) | 0x100000u;
    // P = mx * my (< 2^106) as w0 (bits 0..31), w1 (32..63), hi (64..105)
    const unsigned long long ll = (unsigned long long)xl * yl;
    unsigned long long t = (unsigned long long)xl * myh + (ll >> 32);
    t += (unsigned long long)mxh * yl;
    const unsigned long long hi = (unsigned long long)mxh * myh + (t >> 32);
    const unsigned w0 = (unsigned)ll, w1 = (unsigned)t;
    // P >= 2^105: the significand is P >> 53, else P >> 52
    const unsigned top = (unsigned)(hi >> 41);
    const unsigned long long m = ((hi << 12) | (w1 >> 20)) >> top;
    const unsigned low_mask = (0x100000u << top) - 1u;
    const bool inexact = (w0 | (w1 & low_mask)) != 0u;
    const int e = (int)(ex + ey) - 1023 + (int)top;   // biased exponent of the result
    ok = (ex - 1u < 2046u) && (ey - 1u < 2046u) && e >= 1 && e <= 2046;
    unsigned long long r = ((unsigned long long)sign << 32) + ((unsigned long long)(unsigned)(e - 1) << 52) + m;
    const bool away = inexact && ((sign == 0u) == up);
    return from_bits((long long)(r + (away ? 1ull : 0ull)));
}

// x + y rounded toward +inf (up) or -inf; ok = false when an operand is not
// normal (a zero addend is handled), the sum cancels exactly, or the result
// is not a normal number
__device__ __forceinline__ double add_dir_emu_fast(double x, double y, bool up, bool& ok) {
    const unsigned long long bx = (unsigned long long)bits(x), by = (unsigned long long)bits(y);
    const unsigned long long ax = bx & 0x7FFFFFFFFFFFFFFFull, ay = by & 0x7FFFFFFFFFFFFFFFull;
    // a: the operand of larger magnitude
    const bool swap = ay > ax;
    const unsigned long long ba = swap ? by : bx, bb = swap ? bx : by, mag_b = swap ? ax : ay;
    const unsigned ea = (unsigned)(ba >> 52) & 0x7FFu, eb = (unsigned)(bb >> 52) & 0x7FFu;
    const bool b_zero = mag_b == 0ull;
    // significands with the hidden bit at bit 62 (10 guard bits below bit 10)
    const unsigned long long ma = ((ba & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 10;
    const unsigned long long mb = ((bb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 10;
    const unsigned d = ea - eb;
    // align b; the shifted-out bits are jammed into bit 0
    unsigned long long mbs = 1ull;
    if (d == 0u) mbs = mb;
    else if (d < 64u) mbs = (mb >> d) | ((mb << (64u - d)) != 0ull ? 1ull : 0ull);
    const bool sub = ((ba ^ bb) >> 63) != 0ull;
    unsigned long long s = sub ? ma - mbs : ma + mbs;
    int e = (int)ea;
    // normalise: leading one to bit 62
    const unsigned lz = (unsigned)__clzll((long long)s);   // 64 for s == 0
    if (lz == 0u) {                                        // carry out of an addition
        s = (s >> 1) | (s & 1ull);
        e += 1;
    } else if (lz > 1u && lz < 64u) {                      // cancellation (exact when d <= 1)
        s <<= (lz - 1u);
        e -= (int)(lz - 1u);
    }
    ok = (ea - 1u < 2046u) && ((eb - 1u < 2046u) || b_zero) && s != 0ull && e >= 1 && e <= 2046;
    const bool inexact = (s & 0x3FFull) != 0ull;
    const unsigned long long sa = ba & 0x8000000000000000ull;
    unsigned long long r = sa + ((unsigned long long)(unsigned)(e - 1) << 52) + (s >> 10);
    const bool away = inexact && ((sa == 0ull) == up);
    r += away ? 1ull : 0ull;
    // x + 0 = x exactly for normal x
    return from_bits((long long)(b_zero ? ba : r));
}

__device__ __forceinline__ double mul_rd_emu(double x, double y) {
    bool ok;
    const double r = mul_dir_emu_fast(x, y, false, ok);
    return ok ? r : mul_rd_hw(x, y);
}
__device__ __forceinline__ double mul_ru_emu(double x, double y) {
    bool ok;
    const double r = mul_dir_emu_fast(x, y, true, ok);
    return ok ? r : mul_ru_hw(x, y);
}
__device__ __forceinline__ double add_rd_emu(double x, double y) {
    bool ok;
    const double r = add_dir_emu_fast(x, y, false, ok);
    return ok ? r : add_rd_hw(x, y);
}
__device__ __forceinline__ double add_ru_emu(double x, double y) {
    bool ok;
    const double r = add_dir_emu_fast(x, y, true, ok);
    return ok ? r : add_ru_hw(x, y);
}

}  // namespace ivb
