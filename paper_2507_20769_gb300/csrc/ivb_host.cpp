// ivb_host.cpp -- host-side interval evaluation for the branch and bound:
// point upper bounds, the descent corner heuristic and forward-backward
// constraint propagation (see ivb_host.h).
//
// Directed rounding without changing the FPU mode: every operation is done
// in round-to-nearest and its exact error term decides the neighbour --
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2) for sums, the FMA residual for products,
// quotients and square roots (exact unless the result is within 2^-960 of
// zero, where the result is widened by one step instead). exp and log are
// the C library's (within one ulp) widened by two steps, as in the kernels.
// The fused accumulation (acc + x*y with one rounding per end) switches the
// rounding mode around one fma in a function of its own. Same value, tangent
// and adjoint rules as the kernels (Section 3.2): ENTIRE on domain
// violations, 0 * inf = 0 in products.
#include "ivb_host.h"

#include <cfenv>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "ivb_internal.h"

namespace ivb {

namespace {

constexpr double kTiny = 0x1p-960;   // below this the FMA residual may lose its sign
const double INF = HUGE_VAL;

inline double nup(double x) { return std::nextafter(x, INF); }
inline double ndn(double x) { return std::nextafter(x, -INF); }

// round-to-nearest sum and its exact error (TwoSum)
inline double two_sum(double a, double b, double& e) {
    const double s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
double add_dir(double a, double b, bool up) {
    double e;
    const double s = two_sum(a, b, e);
    if (!std::isfinite(s)) {
        if (std::isfinite(a) && std::isfinite(b))   // overflow of a finite sum
            return s > 0 ? (up ? s : DBL_MAX) : (up ? -DBL_MAX : s);
        return s;
    }
    if (up) return e > 0 ? nup(s) : s;
    return e < 0 ? ndn(s) : s;
}
inline double sub_dir(double a, double b, bool up) { return add_dir(a, -b, up); }

double mul_dir(double a, double b, bool up) {
    if (a == 0.0 || b == 0.0) return 0.0;   // 0 * inf = 0 (interval factors are sets of reals)
    const double p = a * b;
    if (!std::isfinite(p)) {
        if (std::isfinite(a) && std::isfinite(b)) return p > 0 ? (up ? p : DBL_MAX) : (up ? -DBL_MAX : p);
        return p;
    }
    if (std::fabs(p) < kTiny) return up ? nup(p) : ndn(p);
    const double e = std::fma(a, b, -p);
    if (up) return e > 0 ? nup(p) : p;
    return e < 0 ? ndn(p) : p;
}

// a / b for finite a and b != 0
double div_dir(double a, double b, bool up) {
    const double q = a / b;
    if (a == 0.0) return q;                  // exact (+-0)
    if (!std::isfinite(q)) return q > 0 ? (up ? q : DBL_MAX) : (up ? -DBL_MAX : q);
    if (std::fabs(q) < kTiny || std::fabs(a) < kTiny) return up ? nup(q) : ndn(q);
    // a - q b, exact: its sign (times the sign of b) says on which side of q the quotient lies
    const double r = std::fma(-q, b, a);
    const bool above = (r > 0) == (b > 0) && r != 0;   // true quotient > q
    const bool below = (r < 0) == (b > 0) && r != 0;
    if (up) return above ? nup(q) : q;
    return below ? ndn(q) : q;
}

double sqrt_dir(double a, bool up) {
    const double s = std::sqrt(a);
    if (a == 0.0 || !std::isfinite(s)) return s;
    if (a < kTiny) return up ? nup(s) : ndn(s);
    const double r = std::fma(-s, s, a);   // a - s^2, exact
    if (up) return r > 0 ? nup(s) : s;
    return r < 0 ? ndn(s) : s;
}

inline double widen(double v, bool up) { return up ? nup(nup(v)) : ndn(ndn(v)); }
double exp_dir(double x, bool up) {
    if (std::isinf(x)) return x > 0 ? INF : 0.0;
    const double r = widen(std::exp(x), up);
    return (!up && r < 0) ? 0.0 : r;
}
double log_dir(double x, bool up) {
    if (std::isinf(x)) return x;
    return widen(std::log(x), up);
}

// a b + c rounded once toward -inf (up = false) or +inf: the rounding mode is
// switched around one fma; volatile operands and result keep the arithmetic
// between the two switches
__attribute__((noinline, optimize("rounding-math"))) double fma_dir(double a, double b, double c, bool up) {
    volatile double va = a, vb = b, vc = c, r;
    const int mode = std::fegetround();
    std::fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    r = std::fma(va, vb, vc);
    std::fesetround(mode);
    return r;
}
// c + a b with one rounding, a zero factor adding an exact zero
double fprod_dir(double a, double b, double c, bool up) {
    return (a == 0.0 || b == 0.0) ? add_dir(c, 0.0, up) : fma_dir(a, b, c, up);
}

inline hiv mk(double lo, double hi) { return hiv{lo, hi}; }
inline hiv entire() { return mk(-INF, INF); }
inline hiv zero() { return mk(0.0, 0.0); }
inline hiv one() { return mk(1.0, 1.0); }
inline bool has_inf(hiv x) { return std::isinf(x.lo) || std::isinf(x.hi); }

hiv iv_add(hiv x, hiv y) { return mk(add_dir(x.lo, y.lo, false), add_dir(x.hi, y.hi, true)); }
hiv iv_sub(hiv x, hiv y) { return mk(sub_dir(x.lo, y.hi, false), sub_dir(x.hi, y.lo, true)); }
hiv iv_neg(hiv x) { return mk(-x.hi, -x.lo); }
hiv iv_mul(hiv x, hiv y) {
    const double p[4] = {mul_dir(x.lo, y.lo, false), mul_dir(x.lo, y.hi, false), mul_dir(x.hi, y.lo, false),
                         mul_dir(x.hi, y.hi, false)};
    const double q[4] = {mul_dir(x.lo, y.lo, true), mul_dir(x.lo, y.hi, true), mul_dir(x.hi, y.lo, true),
                         mul_dir(x.hi, y.hi, true)};
    return mk(std::fmin(std::fmin(p[0], p[1]), std::fmin(p[2], p[3])),
              std::fmax(std::fmax(q[0], q[1]), std::fmax(q[2], q[3])));
}
// acc + x*y with one directed rounding per end: the extreme of the four
// fused candidates (fmin / fmax skip NaN, as the kernels' pair selection does)
hiv iv_fma(hiv x, hiv y, hiv acc) {
    const double p[4] = {fprod_dir(x.lo, y.lo, acc.lo, false), fprod_dir(x.lo, y.hi, acc.lo, false),
                         fprod_dir(x.hi, y.lo, acc.lo, false), fprod_dir(x.hi, y.hi, acc.lo, false)};
    const double q[4] = {fprod_dir(x.lo, y.lo, acc.hi, true), fprod_dir(x.lo, y.hi, acc.hi, true),
                         fprod_dir(x.hi, y.lo, acc.hi, true), fprod_dir(x.hi, y.hi, acc.hi, true)};
    return mk(std::fmin(std::fmin(p[0], p[1]), std::fmin(p[2], p[3])),
              std::fmax(std::fmax(q[0], q[1]), std::fmax(q[2], q[3])));
}
// exact doubling with the same overflow rule as a directed product
hiv iv_twice(hiv x) { return mk(mul_dir(2.0, x.lo, false), mul_dir(2.0, x.hi, true)); }
hiv iv_sqr(hiv x) {
    const double a = std::fabs(x.lo), b = std::fabs(x.hi);
    const double big = std::fmax(a, b);
    const double small = (x.lo < 0 && x.hi > 0) ? 0.0 : std::fmin(a, b);
    return mk(mul_dir(small, small, false), mul_dir(big, big, true));
}
hiv iv_recip(hiv y) {
    if (!(y.lo > 0 || y.hi < 0)) return entire();
    // 1/y with infinite ends: 1/inf = 0
    const double lo = std::isinf(y.hi) ? 0.0 : div_dir(1.0, y.hi, false);
    const double hi = std::isinf(y.lo) ? 0.0 : div_dir(1.0, y.lo, true);
    return mk(lo, hi);
}
hiv iv_recip_pos(hiv y) { return y.lo > 0 ? iv_recip(y) : entire(); }
hiv iv_div(hiv x, hiv y) {
    if (!(y.lo > 0 || y.hi < 0) || has_inf(x) || has_inf(y)) return entire();
    const double c[4][2] = {{x.lo, y.lo}, {x.lo, y.hi}, {x.hi, y.lo}, {x.hi, y.hi}};
    double lo = INF, hi = -INF;
    for (const auto& v : c) {
        lo = std::fmin(lo, div_dir(v[0], v[1], false));
        hi = std::fmax(hi, div_dir(v[0], v[1], true));
    }
    return mk(lo, hi);
}
hiv iv_sqrt(hiv x) {
    if (x.lo < 0) return entire();
    return mk(sqrt_dir(x.lo, false), sqrt_dir(x.hi, true));
}
hiv iv_exp(hiv x) { return mk(exp_dir(x.lo, false), exp_dir(x.hi, true)); }
hiv iv_log(hiv x) {
    if (!(x.lo > 0)) return entire();
    return mk(log_dir(x.lo, false), log_dir(x.hi, true));
}
hiv nan_to_entire(hiv x) { return (std::isnan(x.lo) || std::isnan(x.hi)) ? entire() : x; }

hiv eval(int op, hiv A, hiv B) {
    switch (op) {
    case OP_ADD: return iv_add(A, B);
    case OP_SUB: return iv_sub(A, B);
    case OP_MUL: return iv_mul(A, B);
    case OP_DIV: return iv_div(A, B);
    case OP_SQR: return iv_sqr(A);
    case OP_SQRT: return iv_sqrt(A);
    case OP_EXP: return iv_exp(A);
    case OP_LOG: return iv_log(A);
    case OP_NEG: return iv_neg(A);
    }
    return entire();
}

bool binary(int op) { return op == OP_ADD || op == OP_SUB || op == OP_MUL || op == OP_DIV; }
bool unary(int op) { return op == OP_SQR || op == OP_SQRT || op == OP_EXP || op == OP_LOG || op == OP_NEG; }

// intersection; returns false when empty
inline bool meet(hiv& x, hiv y) {
    if (std::isnan(y.lo) || std::isnan(y.hi)) return true;   // no information
    x.lo = std::fmax(x.lo, y.lo);
    x.hi = std::fmin(x.hi, y.hi);
    return x.lo <= x.hi;
}

}  // namespace

void host_tape(const ivb_tape* t, HostTape& H) {
    H.n = t->n_vars;
    H.T = t->n_ops;
    H.no = t->n_outputs;
    H.ops.assign(t->ops, t->ops + t->n_ops);
    H.out_idx.assign(t->out_idx, t->out_idx + t->n_outputs);
    H.out_kind.assign(t->out_kind, t->out_kind + t->n_outputs);
    H.has_eq = false;
    for (int o = 0; o < H.no; ++o) {
        if (H.out_kind[o] == IVB_OUT_OBJ) H.obj = o;
        if (H.out_kind[o] == IVB_OUT_EQ) H.has_eq = true;
    }
}

void host_values(const HostTape& H, const double* box, hiv* V) {
    for (int t = 0; t < H.T; ++t) {
        const ivb_op& e = H.ops[t];
        if (e.op == OP_VAR) V[t] = mk(box[2 * e.a], box[2 * e.a + 1]);
        else if (e.op == OP_CONST) V[t] = mk(e.c, e.c);
        else V[t] = eval(e.op, V[e.a], binary(e.op) ? V[e.b] : V[e.a]);
    }
}

void host_gradient(const HostTape& H, const double* box, int o, int grad_mode, hiv* G) {
    const int n = H.n, T = H.T, out = H.out_idx[o];
    std::vector<hiv> V(T);
    host_values(H, box, V.data());
    for (int i = 0; i < n; ++i) G[i] = zero();
    if (grad_mode == IVB_GRAD_FORWARD) {
        // tangent rules (Section 3.2): D[t][d] = d v_t / d x_d
        std::vector<hiv> D((size_t)(out + 1) * n, zero());
        for (int t = 0; t <= out; ++t) {
            const ivb_op& e = H.ops[t];
            hiv* Dt = &D[(size_t)t * n];
            if (e.op == OP_VAR) { Dt[e.a] = one(); continue; }
            if (e.op == OP_CONST) continue;
            const hiv* Da = &D[(size_t)e.a * n];
            const hiv* Db = binary(e.op) ? &D[(size_t)e.b * n] : Da;
            const hiv A = V[e.a], B = binary(e.op) ? V[e.b] : A;
            for (int d = 0; d < n; ++d) {
                switch (e.op) {
                case OP_ADD: Dt[d] = iv_add(Da[d], Db[d]); break;
                case OP_SUB: Dt[d] = iv_sub(Da[d], Db[d]); break;
                case OP_NEG: Dt[d] = iv_neg(Da[d]); break;
                case OP_MUL: Dt[d] = iv_fma(A, Db[d], iv_mul(Da[d], B)); break;
                case OP_DIV: Dt[d] = iv_mul(iv_fma(iv_neg(V[t]), Db[d], Da[d]), iv_recip(B)); break;
                case OP_SQR: Dt[d] = iv_mul(iv_twice(A), Da[d]); break;
                case OP_SQRT: Dt[d] = iv_mul(Da[d], iv_recip_pos(iv_twice(V[t]))); break;
                case OP_EXP: Dt[d] = iv_mul(V[t], Da[d]); break;
                case OP_LOG: Dt[d] = iv_mul(Da[d], iv_recip_pos(A)); break;
                }
            }
        }
        for (int i = 0; i < n; ++i) G[i] = D[(size_t)out * n + i];
        return;
    }
    // reverse sweep from the output, operand a before b
    std::vector<hiv> W(out + 1, zero());
    W[out] = one();
    for (int t = out; t >= 0; --t) {
        const ivb_op& e = H.ops[t];
        const hiv w = W[t];
        if (e.op == OP_VAR) { G[e.a] = iv_add(G[e.a], w); continue; }
        if (e.op == OP_CONST) continue;
        switch (e.op) {
        case OP_ADD: W[e.a] = iv_add(W[e.a], w); W[e.b] = iv_add(W[e.b], w); break;
        case OP_SUB: W[e.a] = iv_add(W[e.a], w); W[e.b] = iv_sub(W[e.b], w); break;
        case OP_NEG: W[e.a] = iv_sub(W[e.a], w); break;
        case OP_MUL:
            W[e.a] = iv_fma(w, V[e.b], W[e.a]);
            W[e.b] = iv_fma(w, V[e.a], W[e.b]);
            break;
        case OP_DIV: {
            const hiv R = iv_recip(V[e.b]);
            W[e.a] = iv_fma(w, R, W[e.a]);
            W[e.b] = iv_fma(iv_neg(iv_mul(w, V[t])), R, W[e.b]);
        } break;
        case OP_SQR: W[e.a] = iv_fma(w, iv_twice(V[e.a]), W[e.a]); break;
        case OP_SQRT: W[e.a] = iv_fma(w, iv_recip_pos(iv_twice(V[t])), W[e.a]); break;
        case OP_EXP: W[e.a] = iv_fma(w, V[t], W[e.a]); break;
        case OP_LOG: W[e.a] = iv_fma(w, iv_recip_pos(V[e.a]), W[e.a]); break;
        }
    }
}

double host_point_value(const HostTape& H, const double* x) {
    if (H.has_eq) return INF;
    std::vector<double> box(2 * H.n);
    for (int i = 0; i < H.n; ++i) { box[2 * i] = x[i]; box[2 * i + 1] = x[i]; }
    std::vector<hiv> V(H.T);
    host_values(H, box.data(), V.data());
    for (int o = 0; o < H.no; ++o)
        if (H.out_kind[o] == IVB_OUT_INEQ && !(V[H.out_idx[o]].hi <= 0.0)) return INF;
    const double v = V[H.out_idx[H.obj]].hi;
    return std::isnan(v) ? INF : v;
}

double host_corner_value(const HostTape& H, const double* box, int grad_mode) {
    const int n = H.n;
    std::vector<hiv> G(n);
    host_gradient(H, box, H.obj, grad_mode, G.data());
    std::vector<double> cp(n), mp(n);
    for (int i = 0; i < n; ++i) {
        const double lo = box[2 * i], hi = box[2 * i + 1], c = (lo + hi) * 0.5;
        cp[i] = G[i].lo > 0.0 ? lo : (G[i].hi < 0.0 ? hi : c);
        mp[i] = (cp[i] + c) * 0.5;
    }
    const double v = host_point_value(H, cp.data());
    if (v < INF) return v;
    return host_point_value(H, mp.data());
}

int host_propagate(const HostTape& H, double* box, double ub, int passes) {
    const int T = H.T, n = H.n;
    std::vector<hiv> V(T);
    std::vector<double> before(2 * n);
    for (int pass = 0; pass < passes; ++pass) {
        std::memcpy(before.data(), box, 2 * n * sizeof(double));
        host_values(H, box, V.data());
        for (int t = 0; t < T; ++t) V[t] = nan_to_entire(V[t]);
        // targets of the outputs
        for (int o = 0; o < H.no; ++o) {
            hiv& z = V[H.out_idx[o]];
            bool ok = true;
            if (H.out_kind[o] == IVB_OUT_INEQ) ok = meet(z, mk(-INF, 0.0));
            else if (H.out_kind[o] == IVB_OUT_EQ) ok = meet(z, zero());
            else if (ub < INF) ok = meet(z, mk(-INF, ub));
            if (!ok) return 1;
        }
        // projections onto the operands, consumers before producers
        for (int t = T - 1; t >= 0; --t) {
            const ivb_op& e = H.ops[t];
            const hiv z = V[t];
            bool ok = true;
            switch (e.op) {
            case OP_VAR: {
                hiv x = mk(box[2 * e.a], box[2 * e.a + 1]);
                ok = meet(x, z);
                box[2 * e.a] = x.lo;
                box[2 * e.a + 1] = x.hi;
            } break;
            case OP_CONST: ok = z.lo <= e.c && e.c <= z.hi; break;
            case OP_ADD:   // z = a + b
                ok = meet(V[e.a], iv_sub(z, V[e.b])) && meet(V[e.b], iv_sub(z, V[e.a]));
                break;
            case OP_SUB:   // z = a - b
                ok = meet(V[e.a], iv_add(z, V[e.b])) && meet(V[e.b], iv_sub(V[e.a], z));
                break;
            case OP_NEG: ok = meet(V[e.a], iv_neg(z)); break;
            case OP_MUL:   // z = a b: a in z / b where 0 is not in b
                if (V[e.b].lo > 0 || V[e.b].hi < 0) ok = meet(V[e.a], iv_div(z, V[e.b]));
                if (ok && (V[e.a].lo > 0 || V[e.a].hi < 0)) ok = meet(V[e.b], iv_div(z, V[e.a]));
                break;
            case OP_DIV:   // z = a / b: a in z b, b in a / z
                ok = meet(V[e.a], iv_mul(z, V[e.b]));
                if (ok && (z.lo > 0 || z.hi < 0)) ok = meet(V[e.b], iv_div(V[e.a], z));
                break;
            case OP_SQR: {   // z = a^2: |a| <= sqrt(z.hi), and |a| >= sqrt(z.lo) on a one-signed a
                if (z.hi < 0) { ok = false; break; }
                const double r_hi = sqrt_dir(z.hi, true);
                const double r_lo = z.lo > 0 ? sqrt_dir(z.lo, false) : 0.0;
                hiv& a = V[e.a];
                if (a.lo >= 0) ok = meet(a, mk(r_lo, r_hi));
                else if (a.hi <= 0) ok = meet(a, mk(-r_hi, -r_lo));
                else ok = meet(a, mk(-r_hi, r_hi));
            } break;
            case OP_SQRT: {   // z = sqrt(a), z >= 0: a in z^2
                if (z.hi < 0) { ok = false; break; }
                const double lo = z.lo > 0 ? mul_dir(z.lo, z.lo, false) : -INF;
                ok = meet(V[e.a], mk(lo, mul_dir(z.hi, z.hi, true)));
            } break;
            case OP_EXP: {   // z = exp(a), z > 0: a in log(z)
                if (!(z.hi > 0)) { ok = false; break; }
                const double lo = z.lo > 0 ? log_dir(z.lo, false) : -INF;
                ok = meet(V[e.a], mk(lo, log_dir(z.hi, true)));
            } break;
            case OP_LOG:   // z = log(a): a in exp(z)
                ok = meet(V[e.a], mk(exp_dir(z.lo, false), exp_dir(z.hi, true)));
                break;
            }
            if (!ok) return 1;
        }
        if (std::memcmp(before.data(), box, 2 * n * sizeof(double)) == 0) break;
    }
    return 0;
}

}  // namespace ivb
