// ivb_fp64x.cuh -- directed-rounding FP64 primitives built for a narrow FP64
// pipe (GB300: one FP64 warp instruction per 64 cycles per SM sub-partition,
// integer / FP32 / MUFU pipes many times wider).
//
// Division, reciprocal, square root (Markstein's method, IBM J. Res. Dev. 34,
// 1990: Newton-Raphson with fused multiply-add and a final remainder): a
// 23-bit seed from the FP32 MUFU approximations (rcp.approx / rsqrt.approx) of
// a float assembled from the double's bits on the integer pipe, FP64 Newton
// steps, then the sign of an exact FMA remainder decides which neighbour is
// the correctly rounded result toward -inf or +inf. The results are the
// correctly rounded directed values (identical to __ddiv_rd & co.); inputs
// outside the fast path's exponent range, and results that are powers of two
// (where the spacing of doubles changes), take the CUDA intrinsic. The sign of
// the remainder comes from the integer pipe: the remainder is below 2^56 in
// units of the last place of the significand product, so it equals the low
// 64 bits of that product (one 64-bit integer multiply) read as a signed
// integer, and no FP64 instruction is spent on it.
//
// exp and log (Tang's table-driven method, ACM TOMS 15(2) 1989 and 16(4)
// 1990): exp(x) = 2^m 2^(j/512) e^r with |r| < 0.00082, e^r - 1 = r + r^2/2
// in FP64 and the tail r^3/6 + r^4/24 + r^5/120 (below 2^-33) on the FP32
// pipe, where 24 bits of it are enough; log(x) = m ln2 - log(c_j) +
// log1p(x 2^-m c_j - 1) with 2048 reciprocal centres c_j and a degree-5
// polynomial whose r^4 and r^5 terms come from the FP32 pipe. Large tables
// (read through L1) buy short polynomials, i.e. fewer FP64 instructions.
// Tables are computed on the host in extended precision. Error before the
// final rounding below 0.6 ulp of the result; the interval ends are then
// moved two neighbour steps outward, which covers at least one ulp (of the
// binade above) on each side, so they enclose the true value.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ivb {

// tables, in device memory of this module (filled by init_math_tables, or
// copied from the library's tables into a tape-specialised module)
constexpr int kExpTab = 512, kLogTab = 2048;
struct ExpEntry { double hi; float hi_f, lo_f; };   // 2^(j/512) = hi + lo; hi and lo rounded to float
struct LogEntry { double c, hi, lo, pad; };    // reciprocal centre c_j, -log(c_j) as hi + lo
struct MathTables {
    ExpEntry exp[kExpTab];
    LogEntry log[kLogTab];
};
#if defined(__CUDACC_RTC__) && defined(IVB_JIT_EXTERN_TABLES)
extern __device__ MathTables g_math;   // defined by the kernel unit of a segmented module
#elif defined(__CUDACC_RTC__)
__device__ MathTables g_math;          // run-time compiled module: filled from the library's copy
#else
static __device__ MathTables g_math;
#endif

__device__ __forceinline__ float rcp_approx_f(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx_f(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ int bexp(double x) { return (int)((bits(x) >> 52) & 0x7FF); }
__device__ __forceinline__ bool mant_zero(double x) { return (bits(x) & 0x000FFFFFFFFFFFFFLL) == 0; }
__device__ __forceinline__ double up1(double y) {   // next toward +inf, y finite nonzero
    long long b = bits(y);
    return from_bits(b >= 0 ? b + 1 : b - 1);
}
__device__ __forceinline__ double dn1(double y) {   // next toward -inf, y finite nonzero
    long long b = bits(y);
    return from_bits(b >= 0 ? b - 1 : b + 1);
}

// significand of a normal double as the integer in [2^52, 2^53)
__device__ __forceinline__ unsigned long long sig53(double x) {
    return ((unsigned long long)bits(x) & 0x000FFFFFFFFFFFFFULL) | 0x0010000000000000ULL;
}
// Remainder signs from the integer pipe. Write the normal doubles a, b, c as
// A 2^ea, B 2^eb, C 2^ec with A, B, C their 53-bit significands (ea = biased
// exponent Ea - 1075). Then c - a b = 2^(ea+eb) (C 2^s - A B) with
// s = ec - ea - eb = Ec + 1075 - Ea - Eb. When c / (a b) is within 2^-50 of 1,
// A B lies in [2^104, 2^106), s in 52..54 and |C 2^s - A B| < 2^56, so
// C 2^s - A B equals the difference of the two products modulo 2^64 read as
// a signed integer: a shift and one 64-bit multiply, exact, no FP64 instruction.
__device__ __forceinline__ long long rem_sig(double a, double b, double c, int s) {
    return (long long)((sig53(c) << s) - sig53(a) * sig53(b));
}

// Slow paths out of line: inlined, the compiler would start parts of them
// speculatively on the fast path, which costs FP64 issue slots every call.
static __device__ __noinline__ double rcp_slow(double y, bool up) { return up ? __drcp_ru(y) : __drcp_rd(y); }
static __device__ __noinline__ double div_slow(double x, double y, bool up) { return up ? __ddiv_ru(x, y) : __ddiv_rd(x, y); }
static __device__ __noinline__ double sqrt_slow(double x, bool up) { return up ? __dsqrt_ru(x) : __dsqrt_rd(x); }
static __device__ __noinline__ double exp_slow(double x) { return exp(x); }
static __device__ __noinline__ double log_slow(double x) { return log(x); }

// 1/y seed for y > 0 with biased exponent E in [1, 2044]: relative error < 2^-21
__device__ __forceinline__ double rcp_seed(double y) {
    const long long b = bits(y);
    const int E = (int)((b >> 52) & 0x7FF);
    const float m = __int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF));   // y's mantissa in [1,2)
    const int rb = __float_as_int(rcp_approx_f(m));                              // (0.5, 1]
    const int fe = (rb >> 23) & 0xFF;
    const long long db = ((long long)(fe - 127 + 2046 - E) << 52) | ((long long)(rb & 0x7FFFFF) << 29);
    return from_bits(db);
}

// 1 - y r0 for a seed r0 of 24 significant bits with |1 - y r0| < 2^-20, from the
// integer pipe. With Y, R0 the significands (R0 of 24 bits), y r0 = Y R0 2^-K with
// K = 2121 - Ey - Er >= 75 and |2^K - Y R0| < 2^57, so 2^K - Y R0 is minus the
// low 64 bits of Y R0; it becomes a double by bit assembly with truncation
// (relative error below 2^-52, which the refinements below tolerate).
__device__ __forceinline__ double one_minus_prod24(double y, double r0) {
    const unsigned long long Y = sig53(y), R = sig53(r0) >> 29;
    const long long D = -(long long)(Y * R);
    const unsigned long long A = D < 0 ? 0ULL - (unsigned long long)D : (unsigned long long)D;
    const int lz = __clzll((long long)A);
    const unsigned long long N = A << (lz & 63);
    const int K = 2121 - bexp(y) - bexp(r0);
    const unsigned long long b = ((unsigned long long)(D < 0) << 63) |
                                 ((unsigned long long)(1023 + 63 - lz - K) << 52) | ((N >> 11) & 0x000FFFFFFFFFFFFFULL);
    return from_bits(A != 0ULL ? (long long)b : 0LL);
}

// fast-path exponent window: products, quotients and remainders stay normal
__device__ __forceinline__ bool safe_e(int E) { return E >= 64 && E <= 1980; }

// ---------------------------------------------------------------- reciprocal
// correctly rounded 1/y toward -inf (up = false) or +inf (up = true), y > 0.
// With e = 1 - y r0 (|e| < 2^-21, from the integer pipe), 1/y =
// r0 / (1 - e) = r0 (1 + e + e^2 + e^3 + ...): r0 + r0 (e + e^2) leaves e^3 <
// 2^-63, so one rounding puts r within 0.5 ulp + 2^-62 relative of 1/y, and the
// exact residual 1 - y r picks the directed neighbour.
__device__ __forceinline__ double rcp_dir_pos(double y, bool up) {
    if (safe_e(bexp(y))) {
        const double r0 = rcp_seed(y);
        const double e = one_minus_prod24(y, r0);
        const double r = __fma_rn(r0, __fma_rn(e, e, e), r0);
        if (!mant_zero(r)) {
            // sign(1 - y r); 1.0 has biased exponent 1023: s = 1023 + 1075 - Ey - Er
            const int s = 2098 - bexp(y) - bexp(r);
            const long long rho = rem_sig(y, r, 1.0, s);
            if (up) return rho <= 0 ? r : up1(r);
            return rho >= 0 ? r : dn1(r);
        }
    }
    return rcp_slow(y, up);
}

// ---------------------------------------------------------------- division
// seed-refined reciprocal of y > 0 (relative error < 2^-42), or 0 when y is
// outside the fast path
__device__ __forceinline__ double rcp_refined(double y) {
    if (!safe_e(bexp(y))) return 0.0;
    const double r = rcp_seed(y);
    return __fma_rn(r, one_minus_prod24(y, r), r);
}

// correctly rounded x/y toward -inf or +inf, y > 0, given r = rcp_refined(y)
__device__ __forceinline__ double div_dir_pos(double x, double y, double r, bool up) {
    const int Ex = bexp(x), Ey = bexp(y);
    const bool x0 = (bits(x) << 1) == 0;
    if (bits(r) != 0 && (x0 || (safe_e(Ex) && Ex - Ey <= 900 && Ey - Ex <= 900))) {
        if (x0) return x;                              // exact: +-0 / y = +-0 for y > 0
        const double q0 = x * r;
        const double q = __fma_rn(__fma_rn(-y, q0, x), r, q0);   // within 0.5 ulp + 2^-80 relative
        const int s = Ex + 1075 - Ey - bexp(q);        // 52..54 for q near x / y
        if (!mant_zero(q) && (unsigned)(s - 48) <= 8u) {
            // sign(x/y - q) = sign(x - y q): |X 2^s - Y Q| for the magnitudes, sign of x applied
            const long long t = rem_sig(y, q, x, s);
            const long long rho = bits(x) < 0 ? -t : t;
            if (up) return rho <= 0 ? q : up1(q);
            return rho >= 0 ? q : dn1(q);
        }
    }
    return div_slow(x, y, up);
}

// directed reciprocal for y of either sign (y != 0, finite or infinite)
__device__ __forceinline__ double rcp_dn(double y) {
    return bits(y) > 0 ? rcp_dir_pos(y, false) : ineg(rcp_dir_pos(ineg(y), true));
}
__device__ __forceinline__ double rcp_up(double y) {
    return bits(y) > 0 ? rcp_dir_pos(y, true) : ineg(rcp_dir_pos(ineg(y), false));
}

// ---------------------------------------------------------------- square root
// correctly rounded sqrt(x) toward -inf or +inf, x >= 0
__device__ __forceinline__ double sqrt_dir(double x, bool up) {
    const long long b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (safe_e(E)) {
        // x = m 2^e, e = E - 1023; seed for 1/sqrt of m' = m or 2m so that the exponent halves
        const int odd = (E + 1) & 1;                 // e odd
        const float mf = __int_as_float(((127 + odd) << 23) | (int)((b >> 29) & 0x7FFFFF));   // [1,4)
        const int rb = __float_as_int(rsqrt_approx_f(mf));
        const int fe = (rb >> 23) & 0xFF;
        const int h = (E - 1023 - odd) / 2;          // exact: E - 1023 - odd is even
        const double r0 = from_bits(((long long)(fe - 127 - h + 1023) << 52) | ((long long)(rb & 0x7FFFFF) << 29));
        double g = x * r0;                           // ~sqrt(x)
        const double hh = from_bits(bits(r0) - (1LL << 52));   // r0 / 2, exact
        const double eps = __fma_rn(-g, hh, 0.5);
        g = __fma_rn(g, eps, g);                     // relative error < 1.5 (2^-21)^2 < 2^-41
        // last step: the remainder x - g^2 is < 2^-40 x, so the seed-accurate 1/(2 sqrt x)
        // (2^-21) leaves < 2^-62 relative: within 0.5 ulp + 2^-62 after one rounding
        g = __fma_rn(__fma_rn(-g, g, x), hh, g);
        const int s = E + 1075 - 2 * bexp(g);          // 52..54 for g near sqrt(x)
        if (!mant_zero(g) && (unsigned)(s - 48) <= 8u) {
            const long long d = rem_sig(g, g, x, s);   // sign(x - g^2) = sign(sqrt(x) - g)
            if (up) return d <= 0 ? g : up1(g);
            return d >= 0 ? g : dn1(g);
        }
    }
    return sqrt_slow(x, up);
}

// ---------------------------------------------------------------- exp
// double whose value is the integer k (|k| < 2^31), assembled on the integer
// pipe: sign, biased exponent 1023 + floor(log2 |k|) from the leading-zero
// count, and |k| shifted under the hidden bit (exact)
__device__ __forceinline__ double int_to_double(int k) {
    const unsigned a = k < 0 ? 0u - (unsigned)k : (unsigned)k;
    const int msb = 31 - __clz((int)a);                       // a > 0: position of the leading one
    const unsigned long long mant = ((unsigned long long)a << (52 - msb)) & 0x000FFFFFFFFFFFFFULL;
    const unsigned long long b = ((unsigned long long)(k < 0) << 63) |
                                 ((unsigned long long)(1023 + msb) << 52) | mant;
    return from_bits(a != 0u ? (long long)b : 0LL);
}

// float nearest to a double v with 2^-126 <= |v| < 2^127 (ties away from
// zero), 0 for smaller |v|; integer pipe only
__device__ __forceinline__ float f32_near(double v) {
    const long long b = bits(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const long long m = (b & 0x7FFFFFFFFFFFFFFFLL) + (1LL << 28);   // round the 29 dropped bits
    const int fb = (int)((m >> 29) - ((long long)(1023 - 127) << 23));
    return __int_as_float(E > 1023 - 127 ? (fb | (int)((b >> 32) & 0x80000000)) : 0);
}
// the double equal to a normal float (0 for zero and subnormal floats); integer pipe only
__device__ __forceinline__ double f64_of(float f) {
    const unsigned fb = (unsigned)__float_as_int(f);
    const unsigned e = (fb >> 23) & 0xFFu;
    const unsigned long long db = ((unsigned long long)(fb >> 31) << 63) |
                                  ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                  ((unsigned long long)(fb & 0x7FFFFFu) << 29);
    return from_bits(e != 0u ? (long long)db : 0LL);
}

// exp(x) for |x| <= 700 (fast path). With k = round(x 512/ln2) (within 0.6 of
// x 512/ln2), j = k mod 512, m = k div 512 and r = x - k ln2/512 (|r| <= 0.6 ln2/512
// < 0.00082): exp(x) = 2^m 2^(j/512) (1 + r + r^2/2 + tau), tau = r^3/6 + r^4/24 +
// r^5/120 + ... < 2^-33.3. r + r^2/2 is one FP64 fma (r/2 is exact); tau and its
// product with the table entry go on the FP32 pipe: 24-bit arithmetic leaves tau
// within 2^-21 relative, i.e. 2^-54.3 absolute, and tl + th tau within 2^-53.3.
// Error before the final rounding below 2^-53.7 of the result (one final rounding
// on top; two-step outward widening needs less than 0.75 ulp of it at powers of
// two and 1.5 ulp elsewhere).
__device__ __forceinline__ double exp_core(double x, bool* ok) {
    const long long b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if ((b & 0x7FFFFFFFFFFFFFFFLL) > 0x4085E00000000000LL) { *ok = false; return 0.0; }   // |x| > 700
    *ok = true;
    // k = round(x 512/ln2), from a float copy of x (any k within one of the rounded value works)
    float xf = 0.0f;
    if (E >= 1023 - 100) xf = __int_as_float((int)((b >> 32) & 0x80000000) | ((E - 1023 + 127) << 23) | (int)((b >> 29) & 0x7FFFFF));
    const int k = __float2int_rn(xf * 738.65986f);
    const double kd = int_to_double(k);
    // r = x - k ln2/512 with ln2/512 = C1 + C2: C1 is ln2/512 rounded to 32 significant
    // bits (k C1 is exact for |k| < 2^19), C2 the remainder rounded to nearest
    const double C1 = 0x1.62e42ff000000p-10, C2 = -0x1.718432a1b0e26p-44;
    double r = __fma_rn(-kd, C1, x);
    r = __fma_rn(-kd, C2, r);
    // FP32: tau = r^3 (1/6 + r/24 + r^2/120)
    const float rf = f32_near(r);
    float q = __fmaf_rn(rf, 1.0f / 120.0f, 1.0f / 24.0f);
    q = __fmaf_rn(rf, q, 1.0f / 6.0f);
    const float tau = __fmul_rn(__fmul_rn(__fmul_rn(rf, rf), rf), q);
    const int j = k & (kExpTab - 1), m = k >> 9;
    const ExpEntry T = g_math.exp[j];
    const double e = f64_of(__fmaf_rn(T.hi_f, tau, T.lo_f));       // tl + th tau
    // FP64: 2^(j/512) (1 + r + r^2/2) + e with one final rounding
    const long long rb = bits(r);
    const double h = ((rb >> 52) & 0x7FF) >= 2 ? from_bits(rb - (1LL << 52)) : 0.0;   // r / 2
    const double p2 = __fma_rn(r, h, r);
    const double y = T.hi + __fma_rn(T.hi, p2, e);
    return from_bits(bits(y) + ((long long)m << 52));
}

// log(x) for normal x > 0 (fast path), error below 1.5 ulp of the result
__device__ __forceinline__ double log_core(double x, bool* ok) {
    const long long b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (b <= 0 || E == 0 || E == 0x7FF) { *ok = false; return 0.0; }
    *ok = true;
    int m = E - 1023;
    const long long mant = b & 0x000FFFFFFFFFFFFFLL;
    const int j = (int)(mant >> 41);                 // top 11 mantissa bits
    long long yb = 0x3FF0000000000000LL | mant;       // y in [1, 2)
    if (j >= kLogTab / 2) { yb -= (1LL << 52); m += 1; }   // y in [0.75, 1)
    const double y = from_bits(yb);
    const LogEntry& T = g_math.log[j];
    const double r = __fma_rn(y, T.c, -1.0);          // |r| <= 2^-11
    // log1p(r) = r + r^2 P(r), P = -1/2 + r/3 - r^2/4 + r^3/5: relative truncation
    // below 2^-57 (next to 1, where r = y - 1 exactly and the result is about r)
    // and below 2^-62 elsewhere, where the result is at least 2^-11.3 in
    // magnitude. delta = r^2 (-1/4 + r/5) is <= 0 and below 2^-22 in magnitude,
    // so it goes on the FP32 pipe (24 bits of it are enough: its error reaches
    // the result multiplied by r^2), and C = -1/2 + delta is assembled exactly on
    // the integer pipe from delta cut to units of 2^-53: P = r/3 + C, one FP64 fma.
    const float rf = f32_near(r);
    const float delta = __fmul_rn(__fmul_rn(rf, rf), __fmaf_rn(rf, 0.2f, -0.25f));
    const int db = __float_as_int(delta) & 0x7FFFFFFF;
    const int sh = (db >> 23) - 127 + 30;              // |delta| = M 2^(sh - 53), M of 24 bits
    const long long M = (long long)((db & 0x7FFFFF) | 0x800000);
    const long long D = db == 0 ? 0LL : (sh >= 0 ? (M << sh) : (sh > -40 ? (M >> -sh) : 0LL));
    const double C = from_bits((long long)0xBFE0000000000000ULL | D);   // -(1/2 + D 2^-53)
    const double P = __fma_rn(r, 1.0 / 3.0, C);
    const double md = int_to_double(m);
    // ln2 = LN2_HI + LN2_LO: LN2_HI is ln2 rounded to 42 significant bits (m LN2_HI is
    // exact for |m| < 2^11), LN2_LO the remainder rounded to nearest
    const double LN2_HI = 0x1.62e42fefa3800p-1, LN2_LO = 0x1.ef35793c76730p-45;
    const double hi = __fma_rn(md, LN2_HI, T.hi);
    const double lo = __fma_rn(md, LN2_LO, T.lo);
    const double s = __fma_rn(r * r, P, r) + lo;
    return hi + s;
}

__device__ __forceinline__ double exp_dir(double x, bool up) {
    bool ok;
    double y = exp_core(x, &ok);
    if (!ok) y = exp_slow(x);
    return up ? next_up(next_up(y)) : next_dn(next_dn(y));
}
__device__ __forceinline__ double log_dir(double x, bool up) {   // x > 0
    bool ok;
    double y = log_core(x, &ok);
    if (!ok) y = log_slow(x);
    return up ? next_up(next_up(y)) : next_dn(next_dn(y));
}

}  // namespace ivb
