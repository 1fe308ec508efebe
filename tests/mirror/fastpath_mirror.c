/*
 * fastpath_mirror.c -- host model of the fast paths of the kernels' directed
 * primitives (reciprocal, division, square root, exp, log), written out again
 * on the CPU from the same algorithms, to check their error analysis on many
 * operands: the integer remainder and seed-residual identities against exact
 * FMA remainders and fesetround division, and the exp / log errors against
 * binary128 evaluation. The hardware reciprocal / reciprocal-square-root seed
 * is modelled as the exact value cut to 24 significant bits and moved by up to
 * three units of its last place (the seeds' error bound). Test code: the GPU
 * tests check the device code itself against the oracle.
 *
 *   fastpath_mirror rcp|div|sqrt|exp|log N   ->  one line "key=value ..."
 */
#define _GNU_SOURCE
#include <fenv.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#pragma STDC FENV_ACCESS ON

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_EXP expq
#define Q_LOG logq
#define Q_EXP2 exp2q
#define Q_ABS fabsq
#define Q_LDEXP ldexpq
#elif defined(__aarch64__)
typedef long double qreal; /* IEEE binary128 on AArch64 Linux */
#define Q_EXP expl
#define Q_LOG logl
#define Q_EXP2 exp2l
#define Q_ABS fabsl
#define Q_LDEXP ldexpl
#else
#error "needs a binary128 type"
#endif

static inline int64_t bits(double x) { int64_t b; memcpy(&b, &x, 8); return b; }
static inline double from_bits(int64_t b) { double x; memcpy(&x, &b, 8); return x; }
static inline float f_of_bits(int32_t b) { float f; memcpy(&f, &b, 4); return f; }
static inline int32_t fbits(float f) { int32_t b; memcpy(&b, &f, 4); return b; }
static inline int bexp(double x) { return (int)((bits(x) >> 52) & 0x7FF); }
static inline int mant_zero(double x) { return (bits(x) & 0x000FFFFFFFFFFFFFLL) == 0; }
static inline double up1(double y) { int64_t b = bits(y); return from_bits(b >= 0 ? b + 1 : b - 1); }
static inline double dn1(double y) { int64_t b = bits(y); return from_bits(b >= 0 ? b - 1 : b + 1); }
static inline int sgn(double v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }
static inline int sgni(int64_t v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

/* ------------------------------------------------ integer-pipe identities */
static inline uint64_t sig53(double x) { return ((uint64_t)bits(x) & 0x000FFFFFFFFFFFFFULL) | 0x0010000000000000ULL; }
/* c - a b in units of the product's last place, modulo 2^64 */
static inline int64_t rem_sig(double a, double b, double c, int s) { return (int64_t)((sig53(c) << s) - sig53(a) * sig53(b)); }
/* 1 - y r0 for a seed of 24 significant bits, truncated to a double */
static double one_minus_prod24(double y, double r0) {
    const uint64_t Y = sig53(y), R = sig53(r0) >> 29;
    const int64_t D = -(int64_t)(Y * R);
    if (D == 0) return 0.0;
    const uint64_t A = D < 0 ? 0 - (uint64_t)D : (uint64_t)D;
    const int lz = __builtin_clzll(A);
    const uint64_t N = A << lz;
    const int K = 2121 - bexp(y) - bexp(r0);
    const uint64_t b = ((uint64_t)(D < 0) << 63) | ((uint64_t)(1023 + 63 - lz - K) << 52) | ((N >> 11) & 0x000FFFFFFFFFFFFFULL);
    return from_bits((int64_t)b);
}
/* FP32 / FP64 conversions on the integer pipe */
static float f32_near(double v) {
    const int64_t b = bits(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const int64_t m = (b & 0x7FFFFFFFFFFFFFFFLL) + (1LL << 28);
    const int32_t fb = (int32_t)((m >> 29) - ((int64_t)(1023 - 127) << 23));
    return f_of_bits(E > 1023 - 127 ? (fb | (int32_t)((b >> 32) & 0x80000000)) : 0);
}
static double f64_of(float f) {
    const uint32_t fb = (uint32_t)fbits(f), e = (fb >> 23) & 0xFFu;
    const uint64_t db = ((uint64_t)(fb >> 31) << 63) | ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)(fb & 0x7FFFFFu) << 29);
    return from_bits(e != 0u ? (int64_t)db : 0LL);
}

/* ------------------------------------------------------------ operands */
static uint64_t st[4] = {0x123456789abcdefULL, 0xfedcba9876543210ULL, 0x0f1e2d3c4b5a6978ULL, 0x1111222233334444ULL};
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t nxt(void) {   /* xoshiro256** */
    const uint64_t r = rotl(st[1] * 5, 7) * 9, t = st[1] << 17;
    st[2] ^= st[0]; st[3] ^= st[1]; st[1] ^= st[2]; st[0] ^= st[3]; st[2] ^= t; st[3] = rotl(st[3], 45);
    return r;
}
static double uni(void) { return (double)(nxt() >> 11) * 0x1.0p-53; }
/* double with biased exponent in [elo, ehi]; an eighth each with significand 1, all ones, or 24 bits */
static double rnd(int elo, int ehi) {
    const int64_t E = elo + (int64_t)(nxt() % (uint64_t)(ehi - elo + 1));
    int64_t m = (int64_t)(nxt() & 0x000FFFFFFFFFFFFFULL);
    const uint64_t k = nxt() % 8;
    if (k == 0) m = 0;
    else if (k == 1) m = 0x000FFFFFFFFFFFFFLL;
    else if (k == 2) m &= ~0xFFFFFFFLL;
    return from_bits((E << 52) | m);
}
/* seed model: the exact value cut to 24 significant bits, moved by up to three units */
static double seed_of(double exact) {
    int64_t b = bits(exact) & ~((1LL << 29) - 1);
    b += ((int64_t)(nxt() % 7) - 3) << 29;
    return from_bits(b);
}
__attribute__((noinline)) static double dir_div(double x_, double y_, int up) {
    volatile double x = x_, y = y_, q;
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    q = x / y;
    fesetround(FE_TONEAREST);
    return q;
}
__attribute__((noinline)) static double dir_sqrt(double x_, int up) {
    volatile double x = x_, q;
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    q = sqrt(x);
    fesetround(FE_TONEAREST);
    return q;
}

/* --------------------------------------------- reciprocal, division, sqrt
 * Each fast path as in the kernels: seed residual from the integer pipe, FP64
 * refinement, the remainder's sign from the integer pipe. Counted: fast-path
 * cases, directed results that differ from fesetround's, remainder signs that
 * differ from the exact FMA remainder's, shifts outside 52..54. */
static void check_rcp(long N) {
    long fast = 0, wrong = 0, sign_bad = 0, shift_bad = 0;
    for (long i = 0; i < N; ++i) {
        const double y = rnd(64, 1980);
        const double r0 = seed_of(1.0 / y);
        const double e = one_minus_prod24(y, r0);
        const double r = fma(r0, fma(e, e, e), r0);
        if (mant_zero(r)) continue;
        ++fast;
        const int s = 2098 - bexp(y) - bexp(r);
        const int64_t rho = rem_sig(y, r, 1.0, s);
        if (s < 52 || s > 54) ++shift_bad;
        if (sgni(rho) != sgn(fma(-y, r, 1.0))) ++sign_bad;
        if ((rho >= 0 ? r : dn1(r)) != dir_div(1.0, y, 0) || (rho <= 0 ? r : up1(r)) != dir_div(1.0, y, 1)) ++wrong;
    }
    printf("fast=%ld wrong=%ld sign_bad=%ld shift_bad=%ld\n", fast, wrong, sign_bad, shift_bad);
}

static void check_div(long N) {
    long fast = 0, exact = 0, wrong = 0, sign_bad = 0, shift_bad = 0;
    for (long i = 0; i < N; ++i) {
        const double y = rnd(200, 1800);
        double x;
        if (i % 4 == 0) {                                     /* exact quotients */
            x = (double)(1 + nxt() % 1000000) * y;
            if (!isfinite(x)) continue;
        } else x = rnd(200, 1800);
        if (nxt() & 1) x = -x;
        const int Ex = bexp(x), Ey = bexp(y);
        if (Ex < 64 || Ex > 1980 || Ex - Ey > 900 || Ey - Ex > 900) continue;
        const double rs = seed_of(1.0 / y);
        const double r = fma(rs, one_minus_prod24(y, rs), rs);
        const double q0 = x * r;
        const double q = fma(fma(-y, q0, x), r, q0);
        const int s = Ex + 1075 - Ey - bexp(q);
        if (mant_zero(q)) continue;
        ++fast;
        if (s < 52 || s > 54) { ++shift_bad; continue; }
        const int64_t t = rem_sig(y, q, x, s);
        const int64_t rho = bits(x) < 0 ? -t : t;
        const double fr = fma(-y, q, x);
        exact += fr == 0.0;
        if (sgni(rho) != sgn(fr)) ++sign_bad;
        if ((rho >= 0 ? q : dn1(q)) != dir_div(x, y, 0) || (rho <= 0 ? q : up1(q)) != dir_div(x, y, 1)) ++wrong;
    }
    printf("fast=%ld exact=%ld wrong=%ld sign_bad=%ld shift_bad=%ld\n", fast, exact, wrong, sign_bad, shift_bad);
}

static void check_sqrt(long N) {
    long fast = 0, exact = 0, wrong = 0, sign_bad = 0, shift_bad = 0;
    for (long i = 0; i < N; ++i) {
        double x;
        if (i % 4 == 0) {                                     /* exact squares: 26-bit roots */
            const double g = from_bits(bits(rnd(600, 1400)) & ~0x7FFFFFFLL);
            x = g * g;
        } else x = rnd(64, 1980);
        const int E = bexp(x);
        if (E < 64 || E > 1980) continue;
        const double r0 = seed_of(1.0 / sqrt(x));
        double g = x * r0;
        const double hh = r0 * 0.5;
        const double eps = fma(-g, hh, 0.5);
        g = fma(g, eps, g);
        g = fma(fma(-g, g, x), hh, g);
        if (mant_zero(g)) continue;
        ++fast;
        const int s = E + 1075 - 2 * bexp(g);
        if (s < 52 || s > 54) { ++shift_bad; continue; }
        const int64_t d = rem_sig(g, g, x, s);
        const double fr = fma(-g, g, x);
        exact += fr == 0.0;
        if (sgni(d) != sgn(fr)) ++sign_bad;
        if ((d >= 0 ? g : dn1(g)) != dir_sqrt(x, 0) || (d <= 0 ? g : up1(g)) != dir_sqrt(x, 1)) ++wrong;
    }
    printf("fast=%ld exact=%ld wrong=%ld sign_bad=%ld shift_bad=%ld\n", fast, exact, wrong, sign_bad, shift_bad);
}

/* ----------------------------------------------------------- exp and log
 * Tables as in the kernels (host extended precision); the fast paths return
 * the two summands of the final rounding so that the error before it can be
 * measured in binary128, and the result widened by two neighbour steps is
 * checked for containment of the binary128 value. Reported: worst error before
 * the final rounding in ulps of the result, worst where the rounded result is a
 * power of two, and the number of inputs whose widened result misses the value. */
static double exp_hi[512];
static float exp_hi_f[512], exp_lo_f[512];
typedef struct { double c, hi, lo; } log_entry;
static log_entry log_tab[2048];

static void tables(void) {
    for (int j = 0; j < 512; ++j) {
        const qreal v = Q_EXP2((qreal)j / 512);
        exp_hi[j] = (double)v;
        exp_hi_f[j] = (float)exp_hi[j];
        exp_lo_f[j] = (float)(double)(v - (qreal)exp_hi[j]);
    }
    for (int j = 0; j < 2048; ++j) {
        double c = 1.0;
        if (j != 0 && j != 2047) {
            const qreal F = (j < 1024) ? 1 + (j + (qreal)0.5) / 2048 : (1 + (j + (qreal)0.5) / 2048) / 2;
            c = (double)(1 / F);
        }
        const qreal L = -Q_LOG((qreal)c);
        log_tab[j].c = c;
        log_tab[j].hi = (double)L;
        log_tab[j].lo = (double)(L - (qreal)log_tab[j].hi);
    }
}

/* exp(x) = 2^m (hi + w) for |x| <= 700 */
static void exp_fast(double x, double* hi, double* w, int* m_out) {
    const int64_t b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    float xf = 0.0f;
    if (E >= 1023 - 100) xf = f_of_bits((int32_t)((b >> 32) & 0x80000000) | ((E - 1023 + 127) << 23) | (int32_t)((b >> 29) & 0x7FFFFF));
    const int k = (int)lrintf(xf * 738.65986f);
    const double kd = (double)k;
    const double C1 = 0x1.62e42ff000000p-10, C2 = -0x1.718432a1b0e26p-44;
    double r = fma(-kd, C1, x);
    r = fma(-kd, C2, r);
    const float rf = f32_near(r);
    float q = fmaf(rf, 1.0f / 120.0f, 1.0f / 24.0f);
    q = fmaf(rf, q, 1.0f / 6.0f);
    const float tau = ((rf * rf) * rf) * q;
    const int j = k & 511;
    const double e = f64_of(fmaf(exp_hi_f[j], tau, exp_lo_f[j]));
    const int64_t rb = bits(r);
    const double h = ((rb >> 52) & 0x7FF) >= 2 ? from_bits(rb - (1LL << 52)) : 0.0;
    const double p2 = fma(r, h, r);
    *hi = exp_hi[j];
    *w = fma(exp_hi[j], p2, e);
    *m_out = k >> 9;
}

/* log(x) = hi + s for normal x > 0 */
static void log_fast(double x, double* hi_out, double* s_out) {
    const int64_t b = bits(x);
    const int E = (int)((b >> 52) & 0x7FF);
    int m = E - 1023;
    const int64_t mant = b & 0x000FFFFFFFFFFFFFLL;
    const int j = (int)(mant >> 41);
    int64_t yb = 0x3FF0000000000000LL | mant;
    if (j >= 1024) { yb -= (1LL << 52); m += 1; }
    const double y = from_bits(yb);
    const log_entry* T = &log_tab[j];
    const double r = fma(y, T->c, -1.0);
    const float rf = f32_near(r);
    const float delta = (rf * rf) * fmaf(rf, 0.2f, -0.25f);
    const int32_t db = fbits(delta) & 0x7FFFFFFF;
    const int sh = (db >> 23) - 127 + 30;
    const int64_t M = (int64_t)((db & 0x7FFFFF) | 0x800000);
    const int64_t D = db == 0 ? 0 : (sh >= 0 ? (M << sh) : (sh > -40 ? (M >> -sh) : 0));
    const double C = from_bits((int64_t)0xBFE0000000000000ULL | D);
    const double P = fma(r, 1.0 / 3.0, C);
    const double md = (double)m;
    const double LN2_HI = 0x1.62e42fefa3800p-1, LN2_LO = 0x1.ef35793c76730p-45;
    *hi_out = fma(md, LN2_HI, T->hi);
    const double lo = fma(md, LN2_LO, T->lo);
    *s_out = fma(r * r, P, r) + lo;
}

static void report(long n, double worst, double worst_p2, long missed) {
    printf("inputs=%ld worst_ulp=%.4f worst_ulp_pow2=%.4f missed=%ld\n", n, worst, worst_p2, missed);
}
static void measure(double y, qreal pre, qreal truth, double scale_lo, double scale_hi, double* worst, double* worst_p2, long* missed) {
    if (y == 0.0) return;
    int ey;
    frexp(y, &ey);
    const double err = (double)(Q_ABS(pre - truth) / (qreal)ldexp(1.0, ey - 53));
    if (err > *worst) *worst = err;
    if (mant_zero(y) && err > *worst_p2) *worst_p2 = err;
    if (!((qreal)scale_lo <= truth && truth <= (qreal)scale_hi)) ++*missed;
}

static void check_exp(long N) {
    long n = 0, missed = 0;
    double worst = 0, worst_p2 = 0;
    const double L = 0.69314718055994530942;
    for (long i = 0; i < N; ++i) {
        double x;
        switch (i % 6) {
        case 0: x = -700 + 1400 * uni(); break;
        case 1: x = -1 + 2 * uni(); break;
        case 2: x = ldexp(2 * uni() - 1, -(int)(nxt() % 60)); break;
        case 3: x = (double)((long)(nxt() % 517000) - 258500) * (L / 512) + ldexp(2 * uni() - 1, -(int)(10 + nxt() % 50)); break;
        case 4: x = ((double)((long)(nxt() % 517000) - 258500) + 0.5) * (L / 512) + ldexp(2 * uni() - 1, -(int)(14 + nxt() % 40)); break;
        default: x = (double)((long)(nxt() % 2000) - 1000) * L + ldexp(2 * uni() - 1, -(int)(nxt() % 50)); break;
        }
        if (fabs(x) > 700) continue;
        ++n;
        double hi, w;
        int m;
        exp_fast(x, &hi, &w, &m);
        const double y = hi + w;
        const qreal truth = Q_EXP((qreal)x) / Q_LDEXP((qreal)1, m);
        measure(y, (qreal)hi + (qreal)w, truth, dn1(dn1(y)), up1(up1(y)), &worst, &worst_p2, &missed);
    }
    report(n, worst, worst_p2, missed);
}

static void check_log(long N) {
    long n = 0, missed = 0;
    double worst = 0, worst_p2 = 0;
    for (long i = 0; i < N; ++i) {
        double x;
        switch (i % 6) {
        case 0: x = ldexp(1 + uni(), (int)(nxt() % 2040) - 1020); break;
        case 1: x = 1 + ldexp(2 * uni() - 1, -(int)(nxt() % 50)); break;
        case 2: x = 0.5 + uni(); break;
        case 3: { const int j = (int)(nxt() % 2048); x = j < 1024 ? 1 + (j + uni()) / 2048.0 : (1 + (j + uni()) / 2048.0) / 2; } break;
        case 4: { const int j = 1 + (int)(nxt() % 8); x = 1 + (j + uni()) / 2048.0; if (nxt() & 1) x = 1 / x; } break;
        default: x = ldexp(1 + uni() * 1e-3, (int)(nxt() % 40) - 20); break;
        }
        if (!(x > 0x1p-1022) || !isfinite(x)) continue;
        double hi, s;
        log_fast(x, &hi, &s);
        const double y = hi + s;
        if (y == 0.0) continue;
        ++n;
        measure(y, (qreal)hi + (qreal)s, Q_LOG((qreal)x), dn1(dn1(y)), up1(up1(y)), &worst, &worst_p2, &missed);
    }
    report(n, worst, worst_p2, missed);
}

int main(int argc, char** argv) {
    if (argc < 3) { fprintf(stderr, "usage: %s rcp|div|sqrt|exp|log N\n", argv[0]); return 2; }
    const long N = atol(argv[2]);
    tables();
    if (!strcmp(argv[1], "rcp")) check_rcp(N);
    else if (!strcmp(argv[1], "div")) check_div(N);
    else if (!strcmp(argv[1], "sqrt")) check_sqrt(N);
    else if (!strcmp(argv[1], "exp")) check_exp(N);
    else if (!strcmp(argv[1], "log")) check_log(N);
    else return 2;
    return 0;
}
