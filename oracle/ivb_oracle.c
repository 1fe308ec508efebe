/*
 * ivb_oracle.c -- plain CPU oracle for GPU-parallel Subdomain Lower Bounding
 * with the interval Mean Value Form (Zhang, Kerkenhoff, Kichler, Dahmen,
 * Mitsos, Naumann, Bongartz: "Accelerating Deterministic Global Optimization
 * via GPU-parallel Interval Arithmetic").
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously correct reference that the
 * CUDA path is checked against. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it. It shares no code,
 * header, table or helper with the CUDA library and includes nothing from it.
 *
 * Outward rounding: every endpoint operation sets the FPU rounding mode with
 * fesetround() around one IEEE operation and restores round-to-nearest
 * afterwards (Section 2.3: on CPUs the global rounding mode must be switched
 * to obtain directed rounding). Operands pass through volatile locals so that
 * the compiler cannot move the arithmetic across the mode switches.
 *
 * Canonical semantics implemented here (the CUDA path implements the same
 * formulas independently; rational ops are then bit-identical because every
 * directed IEEE operation is correctly rounded on both sides):
 *   values   : Section 2.2 (natural interval extension of each intrinsic)
 *   tangents : Section 3.2 (tangent-mode AD over intervals)
 *   adjoints : reverse-mode interval AD (same local partials)
 *   MVF      : Section 2.2, Definition 5 (Mean Value Form), centre c = m(X)
 *   splitting: Section 2.2 (splitting technique, items i-iii)
 *   Steps 1-3 and pruning: Section 3.1 (Fig. 4), basic and adaptive
 *              partitioning: Sections 3.1.1 and 3.1.2
 */
#define _GNU_SOURCE
#include <fenv.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#pragma STDC FENV_ACCESS ON

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_EXP expq
#define Q_LOG logq
#define Q_EPS ((qreal)1.0 / ((qreal)(1ULL << 52) * (qreal)(1ULL << 52)))   /* 2^-104 */
#elif defined(__aarch64__)
typedef long double qreal; /* IEEE binary128 on AArch64 Linux */
_Static_assert(LDBL_MANT_DIG == 113, "long double must be binary128 on AArch64");
#define Q_EXP expl
#define Q_LOG logl
#define Q_EPS 0x1p-104L
#else
#error "oracle needs a binary128 type (x86-64 __float128 or AArch64 long double)"
#endif

/* opcodes and output kinds of the op tape (Section 3.2: the factorable
 * objective and constraints as one DAG, Fig. 5) */
enum { OP_VAR = 0, OP_CONST = 1, OP_ADD = 2, OP_SUB = 3, OP_MUL = 4, OP_DIV = 5,
       OP_SQR = 6, OP_SQRT = 7, OP_EXP = 8, OP_LOG = 9, OP_NEG = 10 };
enum { KIND_OBJ = 0, KIND_INEQ = 1, KIND_EQ = 2 };
enum { GRAD_FORWARD = 0, GRAD_ADJOINT = 1 };
enum { FORM_MVF = 0, FORM_NIE = 1, FORM_MVF_NIE = 2 };

typedef struct { double lo, hi; } iv;

typedef struct {
    int n_vars, n_ops, n_out;
    const uint8_t* op;
    const int32_t* a;
    const int32_t* b;
    const double* c;
    const int32_t* out_idx;
    const uint8_t* out_kind;
} tape_t;

static const iv ZERO = {0.0, 0.0};
static const iv ONE = {1.0, 1.0};
static const iv ENTIRE = {-INFINITY, INFINITY};

/* ---------------------------------------------------------------- rounding */

#define DIRECTED2(name, mode, expr)                                          \
    static double name(double x, double y) {                                 \
        volatile double vx = x, vy = y, r;                                   \
        fesetround(mode);                                                    \
        r = (expr);                                                          \
        fesetround(FE_TONEAREST);                                            \
        return r;                                                            \
    }

DIRECTED2(add_dn, FE_DOWNWARD, vx + vy)
DIRECTED2(add_up, FE_UPWARD, vx + vy)
DIRECTED2(sub_dn, FE_DOWNWARD, vx - vy)
DIRECTED2(sub_up, FE_UPWARD, vx - vy)
DIRECTED2(mul_dn, FE_DOWNWARD, vx * vy)
DIRECTED2(mul_up, FE_UPWARD, vx * vy)
DIRECTED2(div_dn, FE_DOWNWARD, vx / vy)
DIRECTED2(div_up, FE_UPWARD, vx / vy)

/* fused multiply-add rounded once, toward -inf / +inf: RD(x y + z), RU(x y + z)
 * (C99 fma is correctly rounded in the current rounding mode) */
static double fma_dn(double x, double y, double z) {
    volatile double vx = x, vy = y, vz = z, r;
    fesetround(FE_DOWNWARD);
    r = fma(vx, vy, vz);
    fesetround(FE_TONEAREST);
    return r;
}
static double fma_up(double x, double y, double z) {
    volatile double vx = x, vy = y, vz = z, r;
    fesetround(FE_UPWARD);
    r = fma(vx, vy, vz);
    fesetround(FE_TONEAREST);
    return r;
}

static double sqrt_dn(double x) {
    volatile double vx = x, r;
    fesetround(FE_DOWNWARD);
    r = sqrt(vx);
    fesetround(FE_TONEAREST);
    return r;
}
static double sqrt_up(double x) {
    volatile double vx = x, r;
    fesetround(FE_UPWARD);
    r = sqrt(vx);
    fesetround(FE_TONEAREST);
    return r;
}

/* products with the set-theoretic convention 0 * (+-inf) = 0: the interval
 * factors stand for sets of reals, so a zero factor gives an exact zero */
static double prod_dn(double x, double y) { return (x == 0.0 || y == 0.0) ? 0.0 : mul_dn(x, y); }
static double prod_up(double x, double y) { return (x == 0.0 || y == 0.0) ? 0.0 : mul_up(x, y); }

/* z + x y with one rounding and the same convention: a zero factor adds an
 * exact zero */
static double fprod_dn(double x, double y, double z) { return (x == 0.0 || y == 0.0) ? add_dn(z, 0.0) : fma_dn(x, y, z); }
static double fprod_up(double x, double y, double z) { return (x == 0.0 || y == 0.0) ? add_up(z, 0.0) : fma_up(x, y, z); }

static double min2(double x, double y) { return x < y ? x : y; }
static double max2(double x, double y) { return x > y ? x : y; }
static double min4(double p, double q, double r, double s) { return min2(min2(p, q), min2(r, s)); }
static double max4(double p, double q, double r, double s) { return max2(max2(p, q), max2(r, s)); }

/* k representable steps towards -inf / +inf */
static double step_dn(double y, int k) { while (k--) y = nextafter(y, -INFINITY); return y; }
static double step_up(double y, int k) { while (k--) y = nextafter(y, INFINITY); return y; }

/* largest double <= q, smallest double >= q (exact comparisons in binary128) */
static double q_to_dn(qreal q) { double d = (double)q; if ((qreal)d > q) d = nextafter(d, -INFINITY); return d; }
static double q_to_up(qreal q) { double d = (double)q; if ((qreal)d < q) d = nextafter(d, INFINITY); return d; }

/* Rigorous enclosures of exp and log at one point (Section 3.2: functions
 * without correctly rounded implementations are rounded in both directions).
 * tight=1: evaluate in binary128, widen by 2^-104 relative (far above the
 *          library's quad error), round outward to double: at most one ulp
 *          from the true value per side.
 * tight=0: round-to-nearest libm result widened by two ulps per side.
 * tight=k>1: the tight enclosure moved k-1 further representable steps
 *          outward on each side -- the outer end of the bracket that parity
 *          tests put around an implementation allowed k-1 steps beyond the
 *          tight ends per operation; every other operation is unchanged, so
 *          by inclusion isotonicity (Definition 2) a whole tape evaluated
 *          with such operations lies between the tight=1 and tight=k sweeps. */
static double exp_dn(double x, int tight) {
    if (isinf(x)) return x < 0 ? 0.0 : INFINITY;
    double r;
    if (tight) { qreal q = Q_EXP((qreal)x); r = q_to_dn(q - q * Q_EPS); if (tight > 1) r = step_dn(r, tight - 1); }
    else r = step_dn(exp(x), 2);
    return r < 0.0 ? 0.0 : r;
}
static double exp_up(double x, int tight) {
    if (isinf(x)) return x < 0 ? 0.0 : INFINITY;
    if (tight) { qreal q = Q_EXP((qreal)x); double r = q_to_up(q + q * Q_EPS); return tight > 1 ? step_up(r, tight - 1) : r; }
    return step_up(exp(x), 2);
}
static double log_dn(double x, int tight) { /* x > 0 */
    if (isinf(x)) return INFINITY;
    if (tight) {
        qreal q = Q_LOG((qreal)x); qreal m = q < 0 ? -q : q; double r = q_to_dn(q - m * Q_EPS);
        return tight > 1 ? step_dn(r, tight - 1) : r;
    }
    return step_dn(log(x), 2);
}
static double log_up(double x, int tight) { /* x > 0 */
    if (isinf(x)) return INFINITY;
    if (tight) {
        qreal q = Q_LOG((qreal)x); qreal m = q < 0 ? -q : q; double r = q_to_up(q + m * Q_EPS);
        return tight > 1 ? step_up(r, tight - 1) : r;
    }
    return step_up(log(x), 2);
}

/* ------------------------------------------------------ interval operations
 * Natural interval extensions of the intrinsics (Section 2.2). Domain rule:
 * an operation whose argument leaves the intrinsic's domain returns ENTIRE
 * (the paper assumes no domain violations; ENTIRE keeps the bound rigorous). */

static iv iv_add(iv x, iv y) { iv r = {add_dn(x.lo, y.lo), add_up(x.hi, y.hi)}; return r; }
static iv iv_sub(iv x, iv y) { iv r = {sub_dn(x.lo, y.hi), sub_up(x.hi, y.lo)}; return r; }
static iv iv_neg(iv x) { iv r = {-x.hi, -x.lo}; return r; }

/* product: hull of the four endpoint products */
static iv iv_mul(iv x, iv y) {
    iv r;
    r.lo = min4(prod_dn(x.lo, y.lo), prod_dn(x.lo, y.hi), prod_dn(x.hi, y.lo), prod_dn(x.hi, y.hi));
    r.hi = max4(prod_up(x.lo, y.lo), prod_up(x.lo, y.hi), prod_up(x.hi, y.lo), prod_up(x.hi, y.hi));
    return r;
}

/* min / max that skip NaN (NaN only when every argument is NaN) */
static double minnn(double x, double y) { return isnan(x) ? y : (isnan(y) ? x : (x < y ? x : y)); }
static double maxnn(double x, double y) { return isnan(x) ? y : (isnan(y) ? x : (x > y ? x : y)); }

/* acc + x y with one directed rounding per end (a fused multiply-add, which
 * the adjoint accumulation, the tangent rules and the Mean Value Form sum use):
 * lo = RD(acc.lo + min of the four endpoint products), hi = RU(acc.hi + max).
 * RD and RU are monotone, so the min (max) of the four fused candidates is
 * that value. A candidate is NaN only where an infinite addend meets the
 * opposite infinite product; such candidates are skipped unless all are NaN. */
static iv iv_fma(iv x, iv y, iv acc) {
    iv r;
    r.lo = minnn(minnn(fprod_dn(x.lo, y.lo, acc.lo), fprod_dn(x.lo, y.hi, acc.lo)),
                 minnn(fprod_dn(x.hi, y.lo, acc.lo), fprod_dn(x.hi, y.hi, acc.lo)));
    r.hi = maxnn(maxnn(fprod_up(x.lo, y.lo, acc.hi), fprod_up(x.lo, y.hi, acc.hi)),
                 maxnn(fprod_up(x.hi, y.lo, acc.hi), fprod_up(x.hi, y.hi, acc.hi)));
    return r;
}

static int iv_has_inf(iv x) { return isinf(x.lo) || isinf(x.hi); }

/* quotient: defined when 0 is not in y and all endpoints are finite */
static iv iv_div(iv x, iv y) {
    if (!(y.lo > 0.0 || y.hi < 0.0) || iv_has_inf(x) || iv_has_inf(y)) return ENTIRE;
    iv r;
    r.lo = min4(div_dn(x.lo, y.lo), div_dn(x.lo, y.hi), div_dn(x.hi, y.lo), div_dn(x.hi, y.hi));
    r.hi = max4(div_up(x.lo, y.lo), div_up(x.lo, y.hi), div_up(x.hi, y.lo), div_up(x.hi, y.hi));
    return r;
}

/* reciprocal 1/y for 0 not in y (ENTIRE otherwise) */
static iv iv_recip(iv y) {
    if (!(y.lo > 0.0 || y.hi < 0.0)) return ENTIRE;
    iv r = {div_dn(1.0, y.hi), div_up(1.0, y.lo)};
    return r;
}
/* reciprocal of a strictly positive interval (ENTIRE otherwise) */
static iv iv_recip_pos(iv y) { return y.lo > 0.0 ? iv_recip(y) : ENTIRE; }

/* 2*x, outward rounded (exact unless it overflows) */
static iv iv_twice(iv x) { iv r = {mul_dn(2.0, x.lo), mul_up(2.0, x.hi)}; return r; }

static iv iv_sqr(iv x) {
    iv r;
    if (x.lo >= 0.0) { r.lo = prod_dn(x.lo, x.lo); r.hi = prod_up(x.hi, x.hi); }
    else if (x.hi <= 0.0) { r.lo = prod_dn(x.hi, x.hi); r.hi = prod_up(x.lo, x.lo); }
    else { r.lo = 0.0; r.hi = max2(prod_up(x.lo, x.lo), prod_up(x.hi, x.hi)); }
    return r;
}

static iv iv_sqrt(iv x) {
    if (x.lo < 0.0) return ENTIRE;
    iv r = {sqrt_dn(x.lo), sqrt_up(x.hi)};
    return r;
}

static iv iv_exp(iv x, int tight) { iv r = {exp_dn(x.lo, tight), exp_up(x.hi, tight)}; return r; }

static iv iv_log(iv x, int tight) {
    if (!(x.lo > 0.0)) return ENTIRE;
    iv r = {log_dn(x.lo, tight), log_up(x.hi, tight)};
    return r;
}

/* ------------------------------------------------------------- tape sweeps */

static iv op_value(const tape_t* T, int t, const iv* V, const iv* X, int tight) {
    int a = T->a[t], b = T->b[t];
    switch (T->op[t]) {
    case OP_VAR: return X[a];
    case OP_CONST: { iv r = {T->c[t], T->c[t]}; return r; }
    case OP_ADD: return iv_add(V[a], V[b]);
    case OP_SUB: return iv_sub(V[a], V[b]);
    case OP_MUL: return iv_mul(V[a], V[b]);
    case OP_DIV: return iv_div(V[a], V[b]);
    case OP_SQR: return iv_sqr(V[a]);
    case OP_SQRT: return iv_sqrt(V[a]);
    case OP_EXP: return iv_exp(V[a], tight);
    case OP_LOG: return iv_log(V[a], tight);
    case OP_NEG: return iv_neg(V[a]);
    }
    return ENTIRE;
}

/* Natural interval extension of every tape node on the box X (Section 2.2);
 * with a degenerate box [c,c] this is the rigorous point value f(c). */
static void value_sweep(const tape_t* T, const iv* X, iv* V, int tight) {
    for (int t = 0; t < T->n_ops; ++t) V[t] = op_value(T, t, V, X, tight);
}

/* Tangent-mode interval AD (Section 3.2): D[t*n+d] encloses d(node t)/dx_d
 * over X, one vector sweep for all n directions. Local rules ("+ ... fused":
 * the product is added with one rounding per end, iv_fma):
 *   mul:  da*B + A*db, the second product fused
 *   div:  (da + (-V)*db fused) * (1/B)
 *   sqr:  (2A)*da                sqrt: da * (1/(2V))
 *   exp:  V*da                   log:  da * (1/A)                          */
static void tangent_sweep(const tape_t* T, const iv* V, iv* D) {
    const int n = T->n_vars;
    for (int t = 0; t < T->n_ops; ++t) {
        const int a = T->a[t], b = T->b[t];
        iv* Dt = D + (size_t)t * n;
        const iv* Da = D + (size_t)a * n;
        const iv* Db = D + (size_t)b * n;
        iv R;
        switch (T->op[t]) {
        case OP_VAR: for (int d = 0; d < n; ++d) Dt[d] = (d == a) ? ONE : ZERO; break;
        case OP_CONST: for (int d = 0; d < n; ++d) Dt[d] = ZERO; break;
        case OP_ADD: for (int d = 0; d < n; ++d) Dt[d] = iv_add(Da[d], Db[d]); break;
        case OP_SUB: for (int d = 0; d < n; ++d) Dt[d] = iv_sub(Da[d], Db[d]); break;
        case OP_NEG: for (int d = 0; d < n; ++d) Dt[d] = iv_neg(Da[d]); break;
        case OP_MUL:
            for (int d = 0; d < n; ++d) Dt[d] = iv_fma(V[a], Db[d], iv_mul(Da[d], V[b]));
            break;
        case OP_DIV:
            R = iv_recip(V[b]);
            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(iv_fma(iv_neg(V[t]), Db[d], Da[d]), R);
            break;
        case OP_SQR:
            R = iv_twice(V[a]);
            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(R, Da[d]);
            break;
        case OP_SQRT:
            R = iv_recip_pos(iv_twice(V[t]));
            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(Da[d], R);
            break;
        case OP_EXP:
            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(V[t], Da[d]);
            break;
        case OP_LOG:
            R = iv_recip_pos(V[a]);
            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(Da[d], R);
            break;
        default: for (int d = 0; d < n; ++d) Dt[d] = ENTIRE;
        }
    }
}

/* Reverse-mode interval AD for output node `out`: A[t] accumulates the
 * adjoint of node t, processed from `out` down to node 0; for each node the
 * first operand is updated before the second, a product contribution with
 * one rounding per end (iv_fma). G[i] encloses df/dx_i over X. */
static void adjoint_sweep(const tape_t* T, const iv* V, int out, iv* A, iv* G) {
    const int n = T->n_vars;
    for (int t = 0; t <= out; ++t) A[t] = ZERO;
    for (int i = 0; i < n; ++i) G[i] = ZERO;
    A[out] = ONE;
    for (int t = out; t >= 0; --t) {
        const int a = T->a[t], b = T->b[t];
        const iv w = A[t];
        iv R;
        switch (T->op[t]) {
        case OP_VAR: G[a] = iv_add(G[a], w); break;
        case OP_CONST: break;
        case OP_ADD: A[a] = iv_add(A[a], w); A[b] = iv_add(A[b], w); break;
        case OP_SUB: A[a] = iv_add(A[a], w); A[b] = iv_sub(A[b], w); break;
        case OP_NEG: A[a] = iv_sub(A[a], w); break;
        case OP_MUL:
            A[a] = iv_fma(w, V[b], A[a]);
            A[b] = iv_fma(w, V[a], A[b]);
            break;
        case OP_DIV:
            R = iv_recip(V[b]);
            A[a] = iv_fma(w, R, A[a]);
            A[b] = iv_fma(iv_neg(iv_mul(w, V[t])), R, A[b]);
            break;
        case OP_SQR: A[a] = iv_fma(w, iv_twice(V[a]), A[a]); break;
        case OP_SQRT: A[a] = iv_fma(w, iv_recip_pos(iv_twice(V[t])), A[a]); break;
        case OP_EXP: A[a] = iv_fma(w, V[t], A[a]); break;
        case OP_LOG: A[a] = iv_fma(w, iv_recip_pos(V[a]), A[a]); break;
        }
    }
}

/* ---------------------------------------------------- Step 1: partitioning
 * Subinterval j of [lo,hi] split into N parts (Section 2.2, splitting item i):
 * e_j = lo + j*w/N with w = hi-lo, evaluated as RN(lo + RN(j * RN(w/N))),
 * e_0 = lo, e_N = hi, clamped to [lo,hi] so neighbours share endpoints. */
static double endpoint(double lo, double hi, int64_t N, int64_t j) {
    if (j <= 0) return lo;
    if (j >= N) return hi;
    double h = (hi - lo) / (double)N;
    double e = lo + (double)j * h;
    if (e < lo) e = lo;
    if (e > hi) e = hi;
    return e;
}

/* subdomain k of a node, dimension 0 varying fastest (Section 3.1.1 worked
 * example), and its centre c_i = RN(RN(lo_i + hi_i) * 0.5) = m(X_k). */
static void decode(int n, const double* box, const int32_t* splits, int64_t k, iv* X, double* c) {
    for (int i = 0; i < n; ++i) {
        const int64_t N = splits[i];
        const int64_t j = k % N;
        k /= N;
        X[i].lo = endpoint(box[2 * i], box[2 * i + 1], N, j);
        X[i].hi = endpoint(box[2 * i], box[2 * i + 1], N, j + 1);
        c[i] = (X[i].lo + X[i].hi) * 0.5;
    }
}

/* ------------------------------------------- Step 2: per-subdomain bounds */

typedef struct {
    int grad_mode, form, tight, filter;
} opts_t;

typedef struct {
    iv *X, *P, *V, *Vc, *D, *A, *G;
    double* c;
} ws_t;

static int ws_alloc(ws_t* w, const tape_t* T) {
    const size_t n = (size_t)T->n_vars, m = (size_t)T->n_ops;
    w->X = malloc(n * sizeof(iv));
    w->P = malloc(n * sizeof(iv));
    w->V = malloc(m * sizeof(iv));
    w->Vc = malloc(m * sizeof(iv));
    w->D = malloc(m * n * sizeof(iv) + sizeof(iv));
    w->A = malloc(m * sizeof(iv));
    w->G = malloc(n * sizeof(iv) + sizeof(iv));
    w->c = malloc(n * sizeof(double));
    return w->X && w->P && w->V && w->Vc && w->D && w->A && w->G && w->c;
}
static void ws_free(ws_t* w) {
    free(w->X); free(w->P); free(w->V); free(w->Vc); free(w->D); free(w->A); free(w->G); free(w->c);
}

/* Enclosures of every output on subdomain k:
 *   Fc[o] : rigorous point value f_o(c) (interval sweep on [c,c])
 *   F[o]  : Mean Value Form f(c) + <G, X - c> (Definition 5), accumulated
 *           left to right over i, each term G_i (X_i - c_i) added with one
 *           rounding per end (iv_fma); or NIE, or MVF intersected with NIE
 *   G     : optional copy of the gradient enclosures [n_out][n]           */
static void enclose_one(const tape_t* T, const double* box, const int32_t* splits, int64_t k,
                        const opts_t* o, ws_t* w, iv* F, iv* Fc, iv* Gout) {
    const int n = T->n_vars;
    decode(n, box, splits, k, w->X, w->c);
    for (int i = 0; i < n; ++i) { w->P[i].lo = w->c[i]; w->P[i].hi = w->c[i]; }
    value_sweep(T, w->P, w->Vc, o->tight);
    value_sweep(T, w->X, w->V, o->tight);
    if (o->grad_mode == GRAD_FORWARD) tangent_sweep(T, w->V, w->D);
    for (int q = 0; q < T->n_out; ++q) {
        const int out = T->out_idx[q];
        const iv* G;
        if (o->grad_mode == GRAD_FORWARD) G = w->D + (size_t)out * n;
        else { adjoint_sweep(T, w->V, out, w->A, w->G); G = w->G; }
        if (Gout) memcpy(Gout + (size_t)q * n, G, n * sizeof(iv));
        iv mvf = w->Vc[out];
        for (int i = 0; i < n; ++i) {
            iv dx = {sub_dn(w->X[i].lo, w->c[i]), sub_up(w->X[i].hi, w->c[i])};
            mvf = iv_fma(G[i], dx, mvf);
        }
        const iv nie = w->V[out];
        iv r = mvf;
        if (o->form == FORM_NIE) r = nie;
        else if (o->form == FORM_MVF_NIE) { r.lo = max2(mvf.lo, nie.lo); r.hi = min2(mvf.hi, nie.hi); }
        if (isnan(r.lo) || isnan(r.hi)) r = ENTIRE;
        F[q] = r;
        if (Fc) Fc[q] = w->Vc[out];
    }
}

static tape_t make_tape(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a,
                        const int32_t* b, const double* c, const int32_t* out_idx, const uint8_t* out_kind) {
    tape_t T = {n_vars, n_ops, n_out, op, a, b, c, out_idx, out_kind};
    return T;
}

static int64_t n_subdomains(int n, const int32_t* splits) {
    int64_t S = 1;
    for (int i = 0; i < n; ++i) S *= splits[i];
    return S;
}

/* -------------------------------------------------------- exported: steps */

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Step 1 for one subdomain: X_k as [n][2] and its centre c[n]. */
void orc_decode(int n, const double* box, const int32_t* splits, int64_t k, double* X, double* c) {
    iv Xi[64];
    decode(n, box, splits, k, Xi, c);
    for (int i = 0; i < n; ++i) { X[2 * i] = Xi[i].lo; X[2 * i + 1] = Xi[i].hi; }
}

/* Interval value of every node on box X ([n][2]) -> V [n_ops][2]. */
int orc_value_sweep(int n_vars, int n_ops, const uint8_t* op, const int32_t* a, const int32_t* b,
                    const double* c, const double* X, int tight, double* V) {
    tape_t T = make_tape(n_vars, n_ops, 0, op, a, b, c, NULL, NULL);
    iv* Xi = malloc((size_t)n_vars * sizeof(iv));
    iv* Vi = malloc((size_t)n_ops * sizeof(iv));
    if (!Xi || !Vi) { free(Xi); free(Vi); return 2; }
    for (int i = 0; i < n_vars; ++i) { Xi[i].lo = X[2 * i]; Xi[i].hi = X[2 * i + 1]; }
    value_sweep(&T, Xi, Vi, tight);
    memcpy(V, Vi, (size_t)n_ops * sizeof(iv));
    free(Xi); free(Vi);
    return 0;
}

/* Gradient enclosures of every output on box X: G [n_out][n][2]. */
int orc_gradient(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                 const double* c, const int32_t* out_idx, const double* X, int grad_mode, int tight, double* G) {
    tape_t T = make_tape(n_vars, n_ops, n_out, op, a, b, c, out_idx, NULL);
    ws_t w;
    if (!ws_alloc(&w, &T)) { ws_free(&w); return 2; }
    for (int i = 0; i < n_vars; ++i) { w.X[i].lo = X[2 * i]; w.X[i].hi = X[2 * i + 1]; }
    value_sweep(&T, w.X, w.V, tight);
    if (grad_mode == GRAD_FORWARD) tangent_sweep(&T, w.V, w.D);
    for (int q = 0; q < n_out; ++q) {
        const iv* g;
        if (grad_mode == GRAD_FORWARD) g = w.D + (size_t)out_idx[q] * n_vars;
        else { adjoint_sweep(&T, w.V, out_idx[q], w.A, w.G); g = w.G; }
        memcpy(G + (size_t)q * n_vars * 2, g, (size_t)n_vars * sizeof(iv));
    }
    ws_free(&w);
    return 0;
}

/* Per-subdomain enclosures for subdomains first..first+count-1 of one node:
 * F [count][n_out][2]; optional Fc [count][n_out][2], G [count][n_out][n][2]. */
int orc_enclose(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                const double* c, const int32_t* out_idx, const double* box, const int32_t* splits,
                int64_t first, int64_t count, int grad_mode, int form, int tight,
                double* F, double* Fc, double* G) {
    tape_t T = make_tape(n_vars, n_ops, n_out, op, a, b, c, out_idx, NULL);
    opts_t o = {grad_mode, form, tight, 0};
    int err = 0;
#pragma omp parallel reduction(| : err)
    {
        ws_t w;
        if (!ws_alloc(&w, &T)) err = 2;
        else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t s = 0; s < count; ++s) {
                iv* Fs = (iv*)(F + (size_t)s * n_out * 2);
                iv* Fcs = Fc ? (iv*)(Fc + (size_t)s * n_out * 2) : NULL;
                iv* Gs = G ? (iv*)(G + (size_t)s * n_out * n_vars * 2) : NULL;
                enclose_one(&T, box, splits, first + s, &o, &w, Fs, Fcs, Gs);
            }
        }
        ws_free(&w);
    }
    return err;
}

/* ------------------------------------- Step 3: refinement and node results
 * For every node: per output the refinement hull over all subdomains
 * (Section 2.2 splitting item iii, Section 3.1 Step 3): minlo = min_k lo(F_k),
 * maxhi = max_k hi(F_k); lb = minlo of the objective; infeasible when an
 * inequality has minlo > 0 or an equality has 0 outside [minlo, maxhi]
 * (Section 3.1, feasibility check). ub: smallest upper end of f(c_k) over
 * subdomains whose centre is certified feasible (all inequalities with
 * hi(g(c_k)) <= 0; none when equalities exist), +inf if none.
 * With filter=1 the objective minimum skips subdomains that are certainly
 * infeasible (some inequality lo > 0 or equality excluding 0). */
int orc_bound_nodes(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                    const double* c, const int32_t* out_idx, const uint8_t* out_kind, int n_nodes,
                    const double* boxes, const int32_t* splits, int grad_mode, int form, int tight, int filter,
                    double* out_lb, uint8_t* out_inf, double* out_ub, double* out_minlo, double* out_maxhi) {
    tape_t T = make_tape(n_vars, n_ops, n_out, op, a, b, c, out_idx, out_kind);
    opts_t o = {grad_mode, form, tight, filter};
    int obj = -1, has_eq = 0;
    for (int q = 0; q < n_out; ++q) {
        if (out_kind[q] == KIND_OBJ) obj = q;
        if (out_kind[q] == KIND_EQ) has_eq = 1;
    }
    if (obj < 0) return 1;
    int err = 0;
    for (int nd = 0; nd < n_nodes; ++nd) {
        const double* box = boxes + (size_t)nd * n_vars * 2;
        const int32_t* sp = splits + (size_t)nd * n_vars;
        const int64_t S = n_subdomains(n_vars, sp);
        double* minlo = malloc((size_t)n_out * sizeof(double));
        double* maxhi = malloc((size_t)n_out * sizeof(double));
        double objmin = INFINITY, ub = INFINITY;
        for (int q = 0; q < n_out; ++q) { minlo[q] = INFINITY; maxhi[q] = -INFINITY; }
#pragma omp parallel reduction(| : err)
        {
            ws_t w;
            iv* F = malloc((size_t)n_out * sizeof(iv));
            iv* Fc = malloc((size_t)n_out * sizeof(iv));
            double* lmin = malloc((size_t)n_out * sizeof(double));
            double* lmax = malloc((size_t)n_out * sizeof(double));
            double lobj = INFINITY, lub = INFINITY;
            if (!ws_alloc(&w, &T) || !F || !Fc || !lmin || !lmax) err = 2;
            else {
                for (int q = 0; q < n_out; ++q) { lmin[q] = INFINITY; lmax[q] = -INFINITY; }
#pragma omp for schedule(dynamic, 64)
                for (int64_t k = 0; k < S; ++k) {
                    enclose_one(&T, box, sp, k, &o, &w, F, Fc, NULL);
                    int certainly_infeasible = 0, centre_feasible = !has_eq;
                    for (int q = 0; q < n_out; ++q) {
                        if (F[q].lo < lmin[q]) lmin[q] = F[q].lo;
                        if (F[q].hi > lmax[q]) lmax[q] = F[q].hi;
                        if (out_kind[q] == KIND_INEQ) {
                            if (F[q].lo > 0.0) certainly_infeasible = 1;
                            if (!(Fc[q].hi <= 0.0)) centre_feasible = 0;
                        } else if (out_kind[q] == KIND_EQ) {
                            if (F[q].lo > 0.0 || F[q].hi < 0.0) certainly_infeasible = 1;
                        }
                    }
                    if (!(filter && certainly_infeasible) && F[obj].lo < lobj) lobj = F[obj].lo;
                    if (centre_feasible && Fc[obj].hi < lub) lub = Fc[obj].hi;
                }
#pragma omp critical
                {
                    for (int q = 0; q < n_out; ++q) {
                        if (lmin[q] < minlo[q]) minlo[q] = lmin[q];
                        if (lmax[q] > maxhi[q]) maxhi[q] = lmax[q];
                    }
                    if (lobj < objmin) objmin = lobj;
                    if (lub < ub) ub = lub;
                }
            }
            ws_free(&w);
            free(F); free(Fc); free(lmin); free(lmax);
        }
        uint8_t inf = 0;
        for (int q = 0; q < n_out; ++q) {
            if (out_kind[q] == KIND_INEQ && minlo[q] > 0.0) inf = 1;
            if (out_kind[q] == KIND_EQ && (minlo[q] > 0.0 || maxhi[q] < 0.0)) inf = 1;
        }
        double lb = filter ? objmin : minlo[obj];
        if (filter && objmin == INFINITY) inf = 1;
        if (out_lb) out_lb[nd] = lb;
        if (out_inf) out_inf[nd] = inf;
        if (out_ub) out_ub[nd] = ub;
        if (out_minlo) memcpy(out_minlo + (size_t)nd * n_out, minlo, (size_t)n_out * sizeof(double));
        if (out_maxhi) memcpy(out_maxhi + (size_t)nd * n_out, maxhi, (size_t)n_out * sizeof(double));
        free(minlo); free(maxhi);
    }
    return err;
}

/* ------------------------------------------------------ point evaluations */

/* Round-to-nearest point value and reverse-mode gradient of every output at
 * x (same local partials as the interval rules, in plain double). */
int orc_point_grad(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                   const double* c, const int32_t* out_idx, const double* x, double* f, double* g) {
    double* v = malloc((size_t)n_ops * sizeof(double));
    double* w = malloc((size_t)n_ops * sizeof(double));
    if (!v || !w) { free(v); free(w); return 2; }
    for (int t = 0; t < n_ops; ++t) {
        const int ia = a[t], ib = b[t];
        switch (op[t]) {
        case OP_VAR: v[t] = x[ia]; break;
        case OP_CONST: v[t] = c[t]; break;
        case OP_ADD: v[t] = v[ia] + v[ib]; break;
        case OP_SUB: v[t] = v[ia] - v[ib]; break;
        case OP_MUL: v[t] = v[ia] * v[ib]; break;
        case OP_DIV: v[t] = v[ia] / v[ib]; break;
        case OP_SQR: v[t] = v[ia] * v[ia]; break;
        case OP_SQRT: v[t] = sqrt(v[ia]); break;
        case OP_EXP: v[t] = exp(v[ia]); break;
        case OP_LOG: v[t] = log(v[ia]); break;
        case OP_NEG: v[t] = -v[ia]; break;
        default: v[t] = NAN;
        }
    }
    for (int q = 0; q < n_out; ++q) {
        const int out = out_idx[q];
        f[q] = v[out];
        double* gq = g + (size_t)q * n_vars;
        for (int i = 0; i < n_vars; ++i) gq[i] = 0.0;
        for (int t = 0; t <= out; ++t) w[t] = 0.0;
        w[out] = 1.0;
        for (int t = out; t >= 0; --t) {
            const int ia = a[t], ib = b[t];
            const double s = w[t];
            switch (op[t]) {
            case OP_VAR: gq[ia] += s; break;
            case OP_ADD: w[ia] += s; w[ib] += s; break;
            case OP_SUB: w[ia] += s; w[ib] -= s; break;
            case OP_NEG: w[ia] -= s; break;
            case OP_MUL: w[ia] += s * v[ib]; w[ib] += s * v[ia]; break;
            case OP_DIV: { double r = 1.0 / v[ib]; w[ia] += s * r; w[ib] -= (s * v[t]) * r; } break;
            case OP_SQR: w[ia] += s * (2.0 * v[ia]); break;
            case OP_SQRT: w[ia] += s * (1.0 / (2.0 * v[t])); break;
            case OP_EXP: w[ia] += s * v[t]; break;
            case OP_LOG: w[ia] += s * (1.0 / v[ia]); break;
            }
        }
    }
    free(v); free(w);
    return 0;
}

/* Point value of every output at x in binary128, rounded to nearest double:
 * used for central differences whose rounding error must not swamp h^2. */
int orc_point_value_q(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                      const double* c, const int32_t* out_idx, const double* x, const double* dx, double* f) {
    (void)n_vars;
    qreal* v = malloc((size_t)n_ops * sizeof(qreal));
    if (!v) return 2;
    for (int t = 0; t < n_ops; ++t) {
        const int ia = a[t], ib = b[t];
        switch (op[t]) {
        case OP_VAR: v[t] = (qreal)x[ia] + (dx ? (qreal)dx[ia] : (qreal)0); break;
        case OP_CONST: v[t] = c[t]; break;
        case OP_ADD: v[t] = v[ia] + v[ib]; break;
        case OP_SUB: v[t] = v[ia] - v[ib]; break;
        case OP_MUL: v[t] = v[ia] * v[ib]; break;
        case OP_DIV: v[t] = v[ia] / v[ib]; break;
        case OP_SQR: v[t] = v[ia] * v[ia]; break;
#if defined(__x86_64__) || defined(__i386__)
        case OP_SQRT: v[t] = sqrtq(v[ia]); break;
#else
        case OP_SQRT: v[t] = sqrtl(v[ia]); break;
#endif
        case OP_EXP: v[t] = Q_EXP(v[ia]); break;
        case OP_LOG: v[t] = Q_LOG(v[ia]); break;
        case OP_NEG: v[t] = -v[ia]; break;
        default: v[t] = 0;
        }
    }
    for (int q = 0; q < n_out; ++q) f[q] = (double)v[out_idx[q]];
    free(v);
    return 0;
}

/* Central difference (f(x+h e_i) - f(x-h e_i)) / 2h evaluated in binary128
 * for every output and variable: g [n_out][n]. */
int orc_central_diff_q(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                       const double* c, const int32_t* out_idx, const double* x, const double* h, double* g) {
    qreal* vp = malloc((size_t)n_ops * sizeof(qreal));
    qreal* vm = malloc((size_t)n_ops * sizeof(qreal));
    if (!vp || !vm) { free(vp); free(vm); return 2; }
    for (int i = 0; i < n_vars; ++i) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            qreal* v = sgn ? vm : vp;
            for (int t = 0; t < n_ops; ++t) {
                const int ia = a[t], ib = b[t];
                switch (op[t]) {
                case OP_VAR: v[t] = (qreal)x[ia] + ((ia == i) ? (sgn ? -(qreal)h[i] : (qreal)h[i]) : (qreal)0); break;
                case OP_CONST: v[t] = c[t]; break;
                case OP_ADD: v[t] = v[ia] + v[ib]; break;
                case OP_SUB: v[t] = v[ia] - v[ib]; break;
                case OP_MUL: v[t] = v[ia] * v[ib]; break;
                case OP_DIV: v[t] = v[ia] / v[ib]; break;
                case OP_SQR: v[t] = v[ia] * v[ia]; break;
#if defined(__x86_64__) || defined(__i386__)
                case OP_SQRT: v[t] = sqrtq(v[ia]); break;
#else
                case OP_SQRT: v[t] = sqrtl(v[ia]); break;
#endif
                case OP_EXP: v[t] = Q_EXP(v[ia]); break;
                case OP_LOG: v[t] = Q_LOG(v[ia]); break;
                case OP_NEG: v[t] = -v[ia]; break;
                default: v[t] = 0;
                }
            }
        }
        for (int q = 0; q < n_out; ++q)
            g[(size_t)q * n_vars + i] = (double)((vp[out_idx[q]] - vm[out_idx[q]]) / (2 * (qreal)h[i]));
    }
    free(vp); free(vm);
    return 0;
}

/* Rigorous one-point enclosures of exp / log (for per-op ulp tests). */
void orc_exp_enclose(int64_t n, const double* x, int tight, double* lo, double* hi) {
    for (int64_t i = 0; i < n; ++i) { lo[i] = exp_dn(x[i], tight); hi[i] = exp_up(x[i], tight); }
}
void orc_log_enclose(int64_t n, const double* x, int tight, double* lo, double* hi) {
    for (int64_t i = 0; i < n; ++i) {
        if (x[i] > 0) { lo[i] = log_dn(x[i], tight); hi[i] = log_up(x[i], tight); }
        else { lo[i] = -INFINITY; hi[i] = INFINITY; }
    }
}

/* One interval operation on arrays of operands (for closed-form op tests):
 * opcode from the tape alphabet (100: reciprocal, 105: fused r + x y with r
 * the addend on entry), x/y/r as [count][2]. */
void orc_iv_op(int opcode, int64_t count, const double* x, const double* y, int tight, double* r) {
    for (int64_t i = 0; i < count; ++i) {
        iv X = {x[2 * i], x[2 * i + 1]}, Y = {0, 0}, R;
        if (y) { Y.lo = y[2 * i]; Y.hi = y[2 * i + 1]; }
        switch (opcode) {
        case OP_ADD: R = iv_add(X, Y); break;
        case OP_SUB: R = iv_sub(X, Y); break;
        case OP_MUL: R = iv_mul(X, Y); break;
        case OP_DIV: R = iv_div(X, Y); break;
        case OP_SQR: R = iv_sqr(X); break;
        case OP_SQRT: R = iv_sqrt(X); break;
        case OP_EXP: R = iv_exp(X, tight); break;
        case OP_LOG: R = iv_log(X, tight); break;
        case OP_NEG: R = iv_neg(X); break;
        case 100: R = iv_recip(X); break;   /* interval reciprocal */
        case 105: {                         /* r + x y, fused: r holds the addend on entry */
            iv Z = {r[2 * i], r[2 * i + 1]};
            R = iv_fma(X, Y, Z);
        } break;
        default: R = ENTIRE;
        }
        r[2 * i] = R.lo;
        r[2 * i + 1] = R.hi;
    }
}

/* ------------------------------------------------- partitioning strategies
 * strategy 0 uniform (Section 3.1.1): N = floor(target^(1/n)) on every dim.
 * strategy 1 largest (Section 3.1.1): only the widest dim, into target parts.
 * strategy 2 adaptive (Section 3.1.2): start from uniform, then repeatedly
 *   add one subinterval to the dimension with the largest relative width per
 *   subinterval (w_i/ref_i)/N_i whose increment keeps the product <= target
 *   (ties: lowest index); stop when no dimension can grow.
 * ref (optional) holds reference widths for "relative" width; NULL = 1.    */
int orc_pick_splits(int n, const double* box, const double* ref, int64_t target, int strategy, int32_t* out) {
    if (n <= 0 || target < 1) return 1;
    double* rw = malloc((size_t)n * sizeof(double));
    if (!rw) return 2;
    for (int i = 0; i < n; ++i) {
        double w = box[2 * i + 1] - box[2 * i];
        rw[i] = ref ? (ref[i] > 0 ? w / ref[i] : 0.0) : w;
    }
    if (strategy == 1) {
        int wi = 0;
        for (int i = 1; i < n; ++i) if (rw[i] > rw[wi]) wi = i;
        for (int i = 0; i < n; ++i) out[i] = 1;
        out[wi] = (int32_t)(target > 2147483647 ? 2147483647 : target);
        free(rw);
        return 0;
    }
    /* largest N with N^n <= target, by exact integer search */
    int64_t N = 1;
    for (;;) {
        int64_t p = 1, M = N + 1;
        int over = 0;
        for (int i = 0; i < n; ++i) { if (p > target / M) { over = 1; break; } p *= M; }
        if (over || p > target) break;
        N = M;
    }
    for (int i = 0; i < n; ++i) out[i] = (int32_t)N;
    if (strategy == 2) {
        int64_t prod = 1;
        for (int i = 0; i < n; ++i) prod *= out[i];
        for (;;) {
            int best = -1;
            double bestv = -1.0;
            for (int i = 0; i < n; ++i) {
                if (prod / out[i] > target / (out[i] + 1)) continue;          /* would overflow the target */
                if ((prod / out[i]) * (out[i] + 1) > target) continue;
                double v = rw[i] / out[i];
                if (v > bestv) { bestv = v; best = i; }
            }
            if (best < 0) break;
            prod = (prod / out[best]) * (out[best] + 1);
            out[best] += 1;
        }
    }
    free(rw);
    return 0;
}

/* ------------------------------------------------- constraint propagation
 * Forward-backward bound tightening of a node box (host side of the B&B,
 * next to the paper's constraint propagation in its B&B framework): the
 * natural interval extension gives every entry an interval on the box; the
 * outputs are intersected with what a solution must satisfy (inequality
 * g <= 0, equality h = 0, objective f <= ub); then each entry, from the last
 * to the first, passes its interval back to its operands through the
 * inverse of its operation (HC4-style projections), each intersected with
 * what the operand had:
 *   z = a + b : a in z - b, then b in z - a      z = a - b : a in z + b, then b in a - z
 *   z = a * b : a in z / b if 0 not in b, then b in z / a if 0 not in a
 *   z = a / b : a in z * b, then b in a / z if 0 not in z
 *   z = a^2   : |a| <= sqrt(z.hi), and |a| >= sqrt(z.lo) when a has one sign
 *   z = sqrt a: a in [z.lo^2, z.hi^2] (lower end -inf unless z.lo > 0)
 *   z = exp a : a in [log z.lo, log z.hi] (lower end -inf unless z.lo > 0)
 *   z = log a : a in [exp z.lo, exp z.hi]         z = -a : a in -z
 *   variable  : the box's dimension is intersected with z
 *   constant  : z must contain it
 * NaN endpoints mean no information. A round repeats the forward sweep on the
 * tightened box; at most `passes` rounds, stopping early when a round leaves
 * the box bit-for-bit unchanged. Returns 1 when an intersection is empty. */
static int meet_iv(iv* x, iv y) {
    if (isnan(y.lo) || isnan(y.hi)) return 1;
    if (y.lo > x->lo) x->lo = y.lo;
    if (y.hi < x->hi) x->hi = y.hi;
    return x->lo <= x->hi;
}
static int straddles0(iv x) { return !(x.lo > 0.0 || x.hi < 0.0); }

static int propagate_box(const tape_t* T, double* box, double ub, int passes, int tight, iv* X, iv* V,
                         double* before) {
    const int n = T->n_vars;
    for (int pass = 0; pass < passes; ++pass) {
        memcpy(before, box, (size_t)2 * n * sizeof(double));
        for (int i = 0; i < n; ++i) { X[i].lo = box[2 * i]; X[i].hi = box[2 * i + 1]; }
        value_sweep(T, X, V, tight);
        for (int t = 0; t < T->n_ops; ++t)
            if (isnan(V[t].lo) || isnan(V[t].hi)) V[t] = ENTIRE;
        for (int q = 0; q < T->n_out; ++q) {
            iv* z = &V[T->out_idx[q]];
            int ok = 1;
            if (T->out_kind[q] == KIND_INEQ) { iv g = {-INFINITY, 0.0}; ok = meet_iv(z, g); }
            else if (T->out_kind[q] == KIND_EQ) ok = meet_iv(z, ZERO);
            else if (ub < INFINITY) { iv f = {-INFINITY, ub}; ok = meet_iv(z, f); }
            if (!ok) return 1;
        }
        for (int t = T->n_ops - 1; t >= 0; --t) {
            const int a = T->a[t], b = T->b[t];
            const iv z = V[t];
            int ok = 1;
            switch (T->op[t]) {
            case OP_VAR: {
                iv x = {box[2 * a], box[2 * a + 1]};
                ok = meet_iv(&x, z);
                box[2 * a] = x.lo;
                box[2 * a + 1] = x.hi;
            } break;
            case OP_CONST: ok = z.lo <= T->c[t] && T->c[t] <= z.hi; break;
            case OP_ADD: ok = meet_iv(&V[a], iv_sub(z, V[b])) && meet_iv(&V[b], iv_sub(z, V[a])); break;
            case OP_SUB: ok = meet_iv(&V[a], iv_add(z, V[b])) && meet_iv(&V[b], iv_sub(V[a], z)); break;
            case OP_NEG: ok = meet_iv(&V[a], iv_neg(z)); break;
            case OP_MUL:
                if (!straddles0(V[b])) ok = meet_iv(&V[a], iv_div(z, V[b]));
                if (ok && !straddles0(V[a])) ok = meet_iv(&V[b], iv_div(z, V[a]));
                break;
            case OP_DIV:
                ok = meet_iv(&V[a], iv_mul(z, V[b]));
                if (ok && !straddles0(z)) ok = meet_iv(&V[b], iv_div(V[a], z));
                break;
            case OP_SQR: {
                if (z.hi < 0.0) { ok = 0; break; }
                const double r_hi = sqrt_up(z.hi);
                const double r_lo = z.lo > 0.0 ? sqrt_dn(z.lo) : 0.0;
                iv r;
                if (V[a].lo >= 0.0) { r.lo = r_lo; r.hi = r_hi; }
                else if (V[a].hi <= 0.0) { r.lo = -r_hi; r.hi = -r_lo; }
                else { r.lo = -r_hi; r.hi = r_hi; }
                ok = meet_iv(&V[a], r);
            } break;
            case OP_SQRT: {
                if (z.hi < 0.0) { ok = 0; break; }
                iv r = {z.lo > 0.0 ? prod_dn(z.lo, z.lo) : -INFINITY, prod_up(z.hi, z.hi)};
                ok = meet_iv(&V[a], r);
            } break;
            case OP_EXP: {
                if (!(z.hi > 0.0)) { ok = 0; break; }
                iv r = {z.lo > 0.0 ? log_dn(z.lo, tight) : -INFINITY, log_up(z.hi, tight)};
                ok = meet_iv(&V[a], r);
            } break;
            case OP_LOG: {
                iv r = {exp_dn(z.lo, tight), exp_up(z.hi, tight)};
                ok = meet_iv(&V[a], r);
            } break;
            }
            if (!ok) return 1;
        }
        if (memcmp(before, box, (size_t)2 * n * sizeof(double)) == 0) break;
    }
    return 0;
}

/* boxes [count][n][2] tightened in place; infeasible[count] */
int orc_propagate(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
                  const double* c, const int32_t* out_idx, const uint8_t* out_kind, int64_t count, double* boxes,
                  double ub, int passes, int tight, uint8_t* infeasible) {
    tape_t T = make_tape(n_vars, n_ops, n_out, op, a, b, c, out_idx, out_kind);
    iv* X = malloc((size_t)n_vars * sizeof(iv));
    iv* V = malloc((size_t)n_ops * sizeof(iv));
    double* before = malloc((size_t)2 * n_vars * sizeof(double));
    if (!X || !V || !before) { free(X); free(V); free(before); return 2; }
    for (int64_t k = 0; k < count; ++k)
        infeasible[k] = (uint8_t)propagate_box(&T, boxes + (size_t)k * 2 * n_vars, ub, passes, tight, X, V, before);
    free(X); free(V); free(before);
    return 0;
}

/* ---------------------------------------------------------- branch & bound
 * Best-first spatial B&B (Section 3, Fig. 3) with the oracle's bounding as
 * lower-bounding solver. Each iteration pops the open node of lowest lower
 * bound, bisects it along the dimension of largest width relative to the
 * root box, bounds both children (Steps 1-3), and updates the incumbent from
 * the children's rigorous centre-point upper bounds and, with corner_ub, from
 * a descent corner of the child with the smallest centre value: the corner
 * that the sign of the objective's gradient enclosure over the child's box
 * points to (centre where the sign is unknown), else the midpoint between
 * that corner and the centre, used when certified feasible. Only then are
 * children dropped that are infeasible or satisfy
 * lb >= UB - max(eps_abs, eps_rel*|UB|). It stops when
 * UB - min(open lb) <= that tolerance, the heap is empty, or a node / time
 * limit is reached; the final lower bound is min(open lb, lb of nodes
 * dropped by the bound test). Splits per node: the fixed vector `splits` if
 * target <= 0, else orc_pick_splits(target, strategy). With propagate > 0
 * each box (root and children) is first tightened by that many rounds of
 * constraint propagation against the constraints and f <= UB (the UB before
 * the batch); a box proven empty is dropped unbounded and takes no part in
 * the incumbent update. */
typedef struct { double lb; double* box; } bb_node;

static void heap_push(bb_node* h, int64_t* n, bb_node x) {
    int64_t i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].lb <= h[i].lb) break;
        bb_node t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}
static bb_node heap_pop(bb_node* h, int64_t* n) {
    bb_node top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *n && h[l].lb < h[m].lb) m = l;
        if (r < *n && h[r].lb < h[m].lb) m = r;
        if (m == i) break;
        bb_node t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* rigorous objective value at point x, +inf unless certified feasible */
static double bb_point_value(const tape_t* T, const double* x, int tight) {
    const int n = T->n_vars;
    iv* X = malloc((size_t)n * sizeof(iv));
    iv* V = malloc((size_t)T->n_ops * sizeof(iv));
    double r = INFINITY;
    if (X && V) {
        for (int i = 0; i < n; ++i) { X[i].lo = x[i]; X[i].hi = x[i]; }
        value_sweep(T, X, V, tight);
        int feas = 1, obj = 0;
        for (int q = 0; q < T->n_out; ++q) {
            const iv v = V[T->out_idx[q]];
            if (T->out_kind[q] == KIND_OBJ) obj = q;
            if (T->out_kind[q] == KIND_EQ) feas = 0;
            if (T->out_kind[q] == KIND_INEQ && !(v.hi <= 0.0)) feas = 0;
        }
        if (feas) r = V[T->out_idx[obj]].hi;
    }
    free(X); free(V);
    return r;
}

/* descent corner of a box (see above) */
static double bb_corner_value(const tape_t* T, const double* box, int grad_mode, int tight) {
    const int n = T->n_vars;
    int obj = 0;
    for (int q = 0; q < T->n_out; ++q) if (T->out_kind[q] == KIND_OBJ) obj = q;
    ws_t w;
    double r = INFINITY;
    double* cp = malloc((size_t)n * sizeof(double));
    double* mp = malloc((size_t)n * sizeof(double));
    if (ws_alloc(&w, T) && cp && mp) {
        for (int i = 0; i < n; ++i) { w.X[i].lo = box[2 * i]; w.X[i].hi = box[2 * i + 1]; }
        value_sweep(T, w.X, w.V, tight);
        const iv* G;
        if (grad_mode == GRAD_FORWARD) { tangent_sweep(T, w.V, w.D); G = w.D + (size_t)T->out_idx[obj] * n; }
        else { adjoint_sweep(T, w.V, T->out_idx[obj], w.A, w.G); G = w.G; }
        for (int i = 0; i < n; ++i) {
            const double lo = box[2 * i], hi = box[2 * i + 1], c = (lo + hi) * 0.5;
            cp[i] = G[i].lo > 0.0 ? lo : (G[i].hi < 0.0 ? hi : c);
            mp[i] = (cp[i] + c) * 0.5;
        }
        r = bb_point_value(T, cp, tight);
        if (!(r < INFINITY)) r = bb_point_value(T, mp, tight);
    }
    ws_free(&w);
    free(cp); free(mp);
    return r;
}

/* stats: [0] lb, [1] ub, [2] iterations, [3] nodes bounded, [4] subdomains,
 *        [5] seconds, [6] converged (1/0), [7] open nodes left */
int orc_bnb(int n_vars, int n_ops, int n_out, const uint8_t* op, const int32_t* a, const int32_t* b,
            const double* c, const int32_t* out_idx, const uint8_t* out_kind, const double* root,
            const int32_t* splits, int64_t target, int strategy, int grad_mode, int form, int tight,
            double eps_abs, double eps_rel, int64_t max_nodes, double time_limit, int corner_ub, int propagate,
            double* stats) {
    const int n = n_vars;
    tape_t T = make_tape(n_vars, n_ops, n_out, op, a, b, c, out_idx, out_kind);
    int64_t cap = 1024, n_open = 0;
    bb_node* heap = malloc((size_t)cap * sizeof(bb_node));
    double* ref = malloc((size_t)n * sizeof(double));
    int32_t* sp = malloc((size_t)n * sizeof(int32_t));
    iv* pX = malloc((size_t)n * sizeof(iv));
    iv* pV = malloc((size_t)n_ops * sizeof(iv));
    double* pB = malloc((size_t)2 * n * sizeof(double));
    if (!heap || !ref || !sp || !pX || !pV || !pB) {
        free(heap); free(ref); free(sp); free(pX); free(pV); free(pB);
        return 2;
    }
    for (int i = 0; i < n; ++i) ref[i] = root[2 * i + 1] - root[2 * i];
    double UB = INFINITY, t0 = now_s();
    int64_t iters = 0, bounded = 0, subs = 0;
    int converged = 0, err = 0;
    double lb_global = -INFINITY, lb_pruned = INFINITY;
    double* kbox[2];
    double klb[2], kub[2];
    uint8_t kinf[2], kdrop[2];

    /* bound one box: lb, infeasible flag, centre ub; with propagation the box
     * is first tightened against the constraints and f <= UB, and a box
     * proven empty is marked infeasible without being bounded */
    #define BOUND(BOX, LB, INF, UBV, DROP)                                                         \
        do {                                                                                       \
            (DROP) = 0;                                                                            \
            if (propagate > 0 && propagate_box(&T, (BOX), UB, propagate, tight, pX, pV, pB)) {    \
                (LB) = INFINITY; (INF) = 1; (UBV) = INFINITY; (DROP) = 1; break;                  \
            }                                                                                      \
            if (target > 0) orc_pick_splits(n, (BOX), ref, target, strategy, sp);                 \
            else memcpy(sp, splits, (size_t)n * sizeof(int32_t));                                 \
            err |= orc_bound_nodes(n, n_ops, n_out, op, a, b, c, out_idx, out_kind, 1, (BOX), sp, \
                                   grad_mode, form, tight, 0, &(LB), &(INF), &(UBV), NULL, NULL);  \
            bounded++; subs += n_subdomains(n, sp);                                               \
        } while (0)
    /* incumbent update from a batch of bounded boxes, then push or drop each;
     * boxes emptied by propagation take no part */
    #define ABSORB(CNT)                                                                            \
        do {                                                                                       \
            int best_ = -1;                                                                        \
            for (int k_ = 0; k_ < (CNT); ++k_) {                                                   \
                if (kdrop[k_]) continue;                                                           \
                if (kub[k_] < UB) UB = kub[k_];                                                    \
                if (best_ < 0 || kub[k_] < kub[best_]) best_ = k_;                                 \
            }                                                                                      \
            if (corner_ub && best_ >= 0) {                                                         \
                double v_ = bb_corner_value(&T, kbox[best_], grad_mode, tight);                   \
                if (v_ < UB) UB = v_;                                                              \
            }                                                                                      \
            for (int k_ = 0; k_ < (CNT); ++k_) {                                                   \
                double tol_ = fmax(eps_abs, eps_rel * fabs(UB));                                  \
                if (!kinf[k_] && !(klb[k_] >= UB - tol_)) {                                       \
                    if (n_open == cap) { cap *= 2; heap = realloc(heap, (size_t)cap * sizeof(bb_node)); } \
                    heap_push(heap, &n_open, (bb_node){klb[k_], kbox[k_]});                       \
                } else {                                                                           \
                    if (!kinf[k_] && klb[k_] < lb_pruned) lb_pruned = klb[k_];                    \
                    free(kbox[k_]);                                                                \
                }                                                                                  \
            }                                                                                      \
        } while (0)

    kbox[0] = malloc((size_t)n * 2 * sizeof(double));
    memcpy(kbox[0], root, (size_t)n * 2 * sizeof(double));
    BOUND(kbox[0], klb[0], kinf[0], kub[0], kdrop[0]);
    ABSORB(1);
    while (n_open > 0) {
        const double tol = fmax(eps_abs, eps_rel * fabs(UB));
        lb_global = heap[0].lb;
        if (UB - lb_global <= tol) { converged = 1; break; }
        if ((max_nodes > 0 && bounded >= max_nodes) || (time_limit > 0 && now_s() - t0 > time_limit)) break;
        bb_node nd = heap_pop(heap, &n_open);
        if (nd.lb >= UB - tol) { if (nd.lb < lb_pruned) lb_pruned = nd.lb; free(nd.box); continue; }
        iters++;
        int bi = 0;
        double bw = -1.0;
        for (int i = 0; i < n; ++i) {
            double w = (nd.box[2 * i + 1] - nd.box[2 * i]) / ref[i];
            if (w > bw) { bw = w; bi = i; }
        }
        const double lo = nd.box[2 * bi], hi = nd.box[2 * bi + 1];
        const double mid = lo + (hi - lo) * 0.5;
        kbox[0] = malloc((size_t)n * 2 * sizeof(double));
        kbox[1] = nd.box;
        memcpy(kbox[0], nd.box, (size_t)n * 2 * sizeof(double));
        kbox[0][2 * bi + 1] = mid;
        kbox[1][2 * bi] = mid;
        BOUND(kbox[0], klb[0], kinf[0], kub[0], kdrop[0]);
        BOUND(kbox[1], klb[1], kinf[1], kub[1], kdrop[1]);
        ABSORB(2);
    }
    #undef BOUND
    #undef ABSORB
    if (n_open == 0) { converged = 1; lb_global = UB; }
    else lb_global = heap[0].lb;
    if (lb_pruned < lb_global) lb_global = lb_pruned;
    stats[0] = lb_global; stats[1] = UB; stats[2] = (double)iters; stats[3] = (double)bounded;
    stats[4] = (double)subs; stats[5] = now_s() - t0; stats[6] = converged; stats[7] = (double)n_open;
    for (int64_t i = 0; i < n_open; ++i) free(heap[i].box);
    free(heap); free(ref); free(sp); free(pX); free(pV); free(pB);
    return err;
}
