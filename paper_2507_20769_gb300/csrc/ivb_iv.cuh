// ivb_iv.cuh -- outward-rounded binary64 interval arithmetic for sm_103a.
//
// Natural interval extensions of the intrinsics (Section 2.2) with directed
// rounding from the CUDA rounding-mode intrinsics (__dadd_rd / __dmul_ru /
// __ddiv_rd / __dsqrt_ru / __drcp_rd ...; Section 3.2 notes that basic
// operations support all rounding modes on the GPU), and two-ulp outward
// widening of exp/log, whose documented error is one ulp.
//
// GB300 has a narrow FP64 pipe (one warp instruction per 64 cycles per SM
// sub-partition) while the integer pipes are wide, so everything that is not
// a rounded endpoint operation runs on integers: sign and zero tests, min and
// max (ordered-integer compares of the bit patterns), negation, neighbour
// steps. Products pick their endpoint pair by sign case, so an interval
// product costs two directed multiplies (four only when both factors contain
// zero in their interior).
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ivb {

struct iv {
    double lo, hi;
};

// Bit-pattern views of a double. The moves are written in PTX so that the
// compiler does not recognise the integer operations on the pattern (sign
// flips, zero and sign tests, magnitude masks) and turn them back into FP64
// negations, compares or absolute values, which would each take an issue
// slot of the narrow FP64 pipe.
__device__ __forceinline__ long long bits(double x) {
    long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
}
__device__ __forceinline__ double from_bits(long long b) {
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
}

// x >= 0 (includes -0), x <= 0 (includes +0), x == 0 (either sign); no NaNs
__device__ __forceinline__ bool ge0(double x) {
    long long b = bits(x);
    return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool le0(double x) { return bits(x) <= 0; }
__device__ __forceinline__ bool is0(double x) { return (bits(x) << 1) == 0; }
__device__ __forceinline__ bool gt0(double x) { return bits(x) > 0; }              // x > 0
__device__ __forceinline__ bool lt0(double x) {                                    // x < 0
    long long b = bits(x);
    return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool isinf_(double x) { return (bits(x) << 1) == (long long)0xFFE0000000000000ULL; }
__device__ __forceinline__ bool isnan_(double x) {
    return (unsigned long long)(bits(x) << 1) > 0xFFE0000000000000ULL;
}

// monotone signed key: key(x) < key(y) <=> x < y (with -0 < +0)
__device__ __forceinline__ long long okey(double x) {
    long long b = bits(x);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double imin(double x, double y) { return okey(x) <= okey(y) ? x : y; }
__device__ __forceinline__ double imax(double x, double y) { return okey(x) >= okey(y) ? x : y; }
__device__ __forceinline__ bool ilt(double x, double y) { return okey(x) < okey(y); }
__device__ __forceinline__ double ineg(double x) { return from_bits(bits(x) ^ (long long)0x8000000000000000ULL); }

// neighbour towards +inf / -inf (integer steps on the bit pattern)
__device__ __forceinline__ double next_up(double y) {
    long long b = bits(y);
    if (b == 0x7FF0000000000000LL) return y;          // +inf stays
    if ((b << 1) == 0) return from_bits(1);           // +-0 -> smallest subnormal
    return from_bits(b >= 0 ? b + 1 : b - 1);
}
__device__ __forceinline__ double next_dn(double y) { return ineg(next_up(ineg(y))); }

}  // namespace ivb

#include "ivb_fp64x.cuh"
#include "ivb_emu.cuh"

// Which endpoint operations run as the integer-pipe emulation of
// ivb_emu.cuh (bit-identical to the FP64 instructions): bit 0 upper ends of
// products, bit 1 lower ends of products, bit 2 upper ends of sums and
// differences, bit 3 lower ends. The precompiled kernels use none; the
// tape-specialised kernels are compiled with the policy of their problem.
#ifndef IVB_EMU
#define IVB_EMU 0
#endif

// Inlining of the long primitives (reciprocal, division, square root, exp,
// log). Inline by default; a tape-specialised kernel compiled in compact mode
// calls them out of line, which keeps its code and its compile time small.
#ifndef IVB_HEAVY
#define IVB_HEAVY __forceinline__
#endif

namespace ivb {

// ---------------------------------------------------------------- endpoints
// templates on the emulation policy E; the plain names use IVB_EMU
template <int E> __device__ __forceinline__ double add_dn_t(double x, double y) {
    return (E & 8) ? add_rd_emu(x, y) : __dadd_rd(x, y);
}
template <int E> __device__ __forceinline__ double add_up_t(double x, double y) {
    return (E & 4) ? add_ru_emu(x, y) : __dadd_ru(x, y);
}
template <int E> __device__ __forceinline__ double sub_dn_t(double x, double y) {
    return (E & 8) ? add_rd_emu(x, ineg(y)) : __dsub_rd(x, y);
}
template <int E> __device__ __forceinline__ double sub_up_t(double x, double y) {
    return (E & 4) ? add_ru_emu(x, ineg(y)) : __dsub_ru(x, y);
}

// products with 0 * inf = 0 (interval factors are sets of reals)
__device__ __forceinline__ double prod_dir_emu(double x, double y, bool up) {
    const bool z = is0(x) || is0(y);
    bool ok;
    double p = mul_dir_emu_fast(x, y, up, ok);
    if (!ok && !z) p = up ? mul_ru_hw(x, y) : mul_rd_hw(x, y);
    return z ? 0.0 : p;
}
template <int E> __device__ __forceinline__ double prod_dn_t(double x, double y) {
    if (E & 2) return prod_dir_emu(x, y, false);
    double p = __dmul_rd(x, y);
    return (is0(x) || is0(y)) ? 0.0 : p;
}
template <int E> __device__ __forceinline__ double prod_up_t(double x, double y) {
    if (E & 1) return prod_dir_emu(x, y, true);
    double p = __dmul_ru(x, y);
    return (is0(x) || is0(y)) ? 0.0 : p;
}

__device__ __forceinline__ double add_dn(double x, double y) { return add_dn_t<IVB_EMU>(x, y); }
__device__ __forceinline__ double add_up(double x, double y) { return add_up_t<IVB_EMU>(x, y); }
__device__ __forceinline__ double sub_dn(double x, double y) { return sub_dn_t<IVB_EMU>(x, y); }
__device__ __forceinline__ double sub_up(double x, double y) { return sub_up_t<IVB_EMU>(x, y); }
__device__ __forceinline__ double prod_dn(double x, double y) { return prod_dn_t<IVB_EMU>(x, y); }
__device__ __forceinline__ double prod_up(double x, double y) { return prod_up_t<IVB_EMU>(x, y); }

// ---------------------------------------------------------------- intervals
__device__ __forceinline__ iv mk(double lo, double hi) { iv r; r.lo = lo; r.hi = hi; return r; }
__device__ __forceinline__ iv entire() { return mk(from_bits((long long)0xFFF0000000000000ULL), from_bits(0x7FF0000000000000LL)); }
__device__ __forceinline__ iv zero() { return mk(0.0, 0.0); }
__device__ __forceinline__ iv one() { return mk(1.0, 1.0); }
__device__ __forceinline__ bool has_inf(iv x) { return isinf_(x.lo) || isinf_(x.hi); }

template <int E> __device__ __forceinline__ iv iv_add_t(iv x, iv y) {
    return mk(add_dn_t<E>(x.lo, y.lo), add_up_t<E>(x.hi, y.hi));
}
template <int E> __device__ __forceinline__ iv iv_sub_t(iv x, iv y) {
    return mk(sub_dn_t<E>(x.lo, y.hi), sub_up_t<E>(x.hi, y.lo));
}
__device__ __forceinline__ iv iv_add(iv x, iv y) { return iv_add_t<IVB_EMU>(x, y); }
__device__ __forceinline__ iv iv_sub(iv x, iv y) { return iv_sub_t<IVB_EMU>(x, y); }
__device__ __forceinline__ iv iv_neg(iv x) { return mk(ineg(x.hi), ineg(x.lo)); }

// product: sign-case choice of the endpoint pairs that realise min and max of
// the four endpoint products (P: lo >= 0, N: hi <= 0, M: otherwise). The
// operands are picked with selects on the integer pipe, so every lane issues
// the same two directed multiplies; lanes where both factors straddle 0 need a
// second pair, issued only when some lane of the warp needs it (warp-uniform
// branch: no FP64 instruction runs with idle lanes for the common case).
struct MulPairs {
    double lx, ly, ux, uy;   // factors of the lower and of the upper end
    bool mm;                 // both straddle 0: second pair x.hi*y.lo | x.hi*y.hi
};
__device__ __forceinline__ MulPairs mul_pairs(iv x, iv y) {
    const bool xP = ge0(x.lo), xN = !xP && le0(x.hi), xM = !xP && !xN;
    const bool yP = ge0(y.lo), yN = !yP && le0(y.hi), yM = !yP && !yN;
    MulPairs q;
    q.mm = xM && yM;
    // endpoint pairs (lower | upper):
    //   P,P: lo*lo | hi*hi   P,M: hi*lo | hi*hi   P,N: hi*lo | lo*hi
    //   M,P: lo*hi | hi*hi   M,N: hi*lo | lo*lo   M,M: lo*hi, hi*lo | lo*lo, hi*hi
    //   N,P: lo*hi | hi*lo   N,M: lo*hi | lo*lo   N,N: hi*hi | lo*lo
    q.lx = q.mm ? x.lo : ((xP ? !yP : yN) ? x.hi : x.lo);
    q.ly = q.mm ? y.hi : ((xP || (xM && yN)) ? y.lo : y.hi);
    q.ux = q.mm ? x.lo : ((xP ? !yN : yP) ? x.hi : x.lo);
    q.uy = q.mm ? y.lo : ((xP || (xM && yP)) ? y.hi : y.lo);
    return q;
}
template <int E> __device__ __forceinline__ iv iv_mul_t(iv x, iv y) {
    const MulPairs q = mul_pairs(x, y);
    double lo = prod_dn_t<E>(q.lx, q.ly), hi = prod_up_t<E>(q.ux, q.uy);
    if (__any_sync(__activemask(), q.mm)) {
        const double lo2 = prod_dn_t<E>(q.mm ? x.hi : q.lx, q.mm ? y.lo : q.ly);
        const double hi2 = prod_up_t<E>(q.mm ? x.hi : q.ux, q.mm ? y.hi : q.uy);
        lo = imin(lo, lo2);
        hi = imax(hi, hi2);
    }
    return mk(lo, hi);
}
__device__ __forceinline__ iv iv_mul(iv x, iv y) { return iv_mul_t<IVB_EMU>(x, y); }

// acc + x*y with one directed rounding per end (fused multiply-add): each end
// adds the extreme endpoint product to the accumulator's end in one rounding,
// RD(acc.lo + min) and RU(acc.hi + max). Same pair selection as the product;
// a zero factor gives an exact zero product (0 * inf = 0), i.e. RD(acc.lo + 0)
// = acc.lo and RU(acc.hi + 0) = acc.hi with -0 turned into +0. One FP64 fma per
// end instead of a multiply and an add. Never emulated (the emulation policy
// covers stand-alone adds and multiplies only), so every policy gives the same
// bits.
__device__ __forceinline__ double fprod_dn(double x, double y, double c) {
    const double p = __fma_rd(x, y, c);
    return (is0(x) || is0(y)) ? c : p;
}
__device__ __forceinline__ double fprod_up(double x, double y, double c) {
    const double p = __fma_ru(x, y, c);
    return (is0(x) || is0(y)) ? (is0(c) ? 0.0 : c) : p;
}
__device__ __forceinline__ iv iv_fma(iv x, iv y, iv acc) {
    const MulPairs q = mul_pairs(x, y);
    double lo = fprod_dn(q.lx, q.ly, acc.lo), hi = fprod_up(q.ux, q.uy, acc.hi);
    if (__any_sync(__activemask(), q.mm)) {
        const double lo2 = fprod_dn(q.mm ? x.hi : q.lx, q.mm ? y.lo : q.ly, acc.lo);
        const double hi2 = fprod_up(q.mm ? x.hi : q.ux, q.mm ? y.hi : q.uy, acc.hi);
        lo = imin(lo, lo2);
        hi = imax(hi, hi2);
    }
    return mk(lo, hi);
}

// 2*x rounded toward -inf / +inf: exact (an exponent increment on the integer
// pipe, or a shift for zero and subnormals) unless |x| >= 2^1023, where the
// directed multiply decides between the largest double and infinity
__device__ __forceinline__ double twice_dir(double x, bool up) {
    const long long b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return from_bits((b & (long long)0x8000000000000000ULL) | ((b & 0x7FFFFFFFFFFFFFFFLL) << 1));
    if (E < 2046) return from_bits(b + (1LL << 52));
    return up ? __dmul_ru(2.0, x) : __dmul_rd(2.0, x);
}
__device__ __forceinline__ iv iv_twice(iv x) { return mk(twice_dir(x.lo, false), twice_dir(x.hi, true)); }

// square: [a^2, b^2] with b = max(|lo|, |hi|) and a = min(|lo|, |hi|), or
// a = 0 when the interval straddles 0 -- two directed multiplies, no branch
template <int E> __device__ __forceinline__ iv iv_sqr_t(iv x) {
    const long long ml = bits(x.lo) & 0x7FFFFFFFFFFFFFFFLL, mh = bits(x.hi) & 0x7FFFFFFFFFFFFFFFLL;
    const bool straddle = !ge0(x.lo) && !le0(x.hi);
    const double big = from_bits(ml > mh ? ml : mh);
    const double small = straddle ? 0.0 : from_bits(ml > mh ? mh : ml);
    return mk(prod_dn_t<E>(small, small), prod_up_t<E>(big, big));
}
__device__ __forceinline__ iv iv_sqr(iv x) { return iv_sqr_t<IVB_EMU>(x); }

// reciprocal of an interval without 0 (ENTIRE otherwise)
__device__ IVB_HEAVY iv iv_recip(iv y) {
    if (!(gt0(y.lo) || lt0(y.hi))) return entire();
    return mk(rcp_dn(y.hi), rcp_up(y.lo));
}
__device__ __forceinline__ iv iv_recip_pos(iv y) { return gt0(y.lo) ? iv_recip(y) : entire(); }

// quotient for 0 not in y and finite endpoints (ENTIRE otherwise)
__device__ IVB_HEAVY iv iv_div(iv x, iv y) {
    const bool ypos = gt0(y.lo), yneg = lt0(y.hi);
    if (!(ypos || yneg) || has_inf(x) || has_inf(y)) return entire();
    // for y < 0 use x/y = (-x)/(-y) with -y > 0 (negations are exact)
    double xl = x.lo, xh = x.hi, yl = y.lo, yh = y.hi;
    if (yneg) { xl = ineg(x.hi); xh = ineg(x.lo); yl = ineg(y.hi); yh = ineg(y.lo); }
    const double dl = ge0(xl) ? yh : yl;
    const double dh = ge0(xh) ? yl : yh;
    const double rl = rcp_refined(dl);
    const double rh = (bits(dh) == bits(dl)) ? rl : rcp_refined(dh);
    return mk(div_dir_pos(xl, dl, rl, false), div_dir_pos(xh, dh, rh, true));
}

__device__ IVB_HEAVY iv iv_sqrt(iv x) {
    if (lt0(x.lo)) return entire();
    return mk(sqrt_dir(x.lo, false), sqrt_dir(x.hi, true));
}

// exp / log: table-driven evaluation (ivb_fp64x.cuh) widened two neighbour
// steps outward; the lower end of exp is clamped at 0.
__device__ __forceinline__ double exp_dn(double x) {
    double r = exp_dir(x, false);
    return lt0(r) ? 0.0 : r;
}
__device__ __forceinline__ double exp_up(double x) { return exp_dir(x, true); }
__device__ __forceinline__ double log_dn(double x) { return log_dir(x, false); }
__device__ __forceinline__ double log_up(double x) { return log_dir(x, true); }

__device__ IVB_HEAVY iv iv_exp(iv x) { return mk(exp_dn(x.lo), exp_up(x.hi)); }
__device__ IVB_HEAVY iv iv_log(iv x) {
    if (!gt0(x.lo)) return entire();
    return mk(log_dn(x.lo), log_up(x.hi));
}

// intersection of two enclosures of the same quantity
__device__ __forceinline__ iv iv_meet(iv x, iv y) { return mk(imax(x.lo, y.lo), imin(x.hi, y.hi)); }

}  // namespace ivb
