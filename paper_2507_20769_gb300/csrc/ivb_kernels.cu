// ivb_kernels.cu -- sm_103a kernels for Subdomain Lower Bounding (Section 3.1),
// tape interpreter (tile loop, decoding and reductions in ivb_bound_common.cuh):
//   Step 1: subdomain boxes decoded from the thread's global index (never
//           stored), dimension 0 fastest (Section 3.1.1)
//   Step 2: Mean Value Form (Definition 5) per subdomain: rigorous f(c) by an
//           interval sweep on [c,c], gradient enclosure by forward tangents or
//           by a reverse (adjoint) interval sweep
//   Step 3: refinement hull (Section 2.2 item iii) by warp shuffles and
//           ordered-integer atomicMin / atomicMax per node and output
// One persistent kernel serves any number of nodes: blocks grab tiles of the
// global subdomain index space from a device counter and map indices to nodes
// through the node queue's prefix sums.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ivb_bound_common.cuh"
#include "ivb_internal.h"
#include "ivb_iv.cuh"
#include "ivb_kernels.h"

namespace ivb {

// ------------------------------------------------------------------ frame
struct Frame {
    double* p;  // this thread's element 0
    int s;      // stride between consecutive units
    __device__ __forceinline__ double ld(int u) const { return p[(size_t)u * s]; }
    __device__ __forceinline__ void st(int u, double v) const { p[(size_t)u * s] = v; }
    __device__ __forceinline__ iv get(int u) const { return mk(ld(u), ld(u + 1)); }
    __device__ __forceinline__ void put(int u, iv v) const { st(u, v.lo); st(u + 1, v.hi); }
};

struct SweepCtx {
    Frame F;
    const double* consts;
    int x_base, c_base;
    bool point;  // VAR operands read [c,c] instead of X
};

__device__ __forceinline__ iv load_val(const SweepCtx& C, uint32_t kind, uint32_t idx, int base, int rec) {
    if (kind == K_SLOT) return C.F.get(base + (int)idx * rec);
    if (kind == K_VAR) {
        if (C.point) { double c = C.F.ld(C.c_base + (int)idx); return mk(c, c); }
        return C.F.get(C.x_base + 2 * (int)idx);
    }
    const double k = __ldg(C.consts + idx);
    return mk(k, k);
}

__device__ __forceinline__ iv eval_value(uint32_t op, iv A, iv B) {
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

// interval values of a straight-line program; records of 2 units at `base`
__device__ void run_values(const Ins* __restrict__ ins, int count, const SweepCtx& C, int base) {
    for (int i = 0; i < count; ++i) {
        const Ins I = ins[i];
        const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
        const iv A = load_val(C, ak, I.w1 & 0xFFFFu, base, 2);
        const iv B = (bk != K_NONE) ? load_val(C, bk, I.w1 >> 16, base, 2) : A;
        C.F.put(base + 2 * (int)dst, eval_value(op, A, B));
    }
}

// tangent of an operand in direction d
__device__ __forceinline__ iv load_tan(const SweepCtx& C, uint32_t kind, uint32_t idx, int base, int rec, int d) {
    if (kind == K_SLOT) return C.F.get(base + (int)idx * rec + 2 + 2 * d);
    if (kind == K_VAR) return ((int)idx == d) ? one() : zero();
    return zero();
}

// forward-mode sweep: value + n tangent intervals per record (Section 3.2).
// Terms whose tangent is exactly zero (constant operands) are skipped: adding
// [0,0] and multiplying by [0,0] are exact, so the values do not change.
__device__ void run_tangents(const Ins* __restrict__ ins, int count, const SweepCtx& C, int base, int n) {
    const int rec = 2 * (1 + n);
    for (int i = 0; i < count; ++i) {
        const Ins I = ins[i];
        const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
        const uint32_t ai = I.w1 & 0xFFFFu, bi = I.w1 >> 16;
        const iv A = load_val(C, ak, ai, base, rec);
        const iv B = (bk != K_NONE) ? load_val(C, bk, bi, base, rec) : A;
        const iv V = eval_value(op, A, B);
        const int o = base + (int)dst * rec;
        const bool az = (ak == K_CONST), bz = (bk == K_CONST || bk == K_NONE);
        switch (op) {
        case OP_ADD:
            for (int d = 0; d < n; ++d) {
                iv t = az ? load_tan(C, bk, bi, base, rec, d)
                          : bz ? load_tan(C, ak, ai, base, rec, d)
                               : iv_add(load_tan(C, ak, ai, base, rec, d), load_tan(C, bk, bi, base, rec, d));
                C.F.put(o + 2 + 2 * d, t);
            }
            break;
        case OP_SUB:
            for (int d = 0; d < n; ++d) {
                iv t = az ? iv_neg(load_tan(C, bk, bi, base, rec, d))
                          : bz ? load_tan(C, ak, ai, base, rec, d)
                               : iv_sub(load_tan(C, ak, ai, base, rec, d), load_tan(C, bk, bi, base, rec, d));
                C.F.put(o + 2 + 2 * d, t);
            }
            break;
        case OP_NEG:
            for (int d = 0; d < n; ++d) C.F.put(o + 2 + 2 * d, iv_neg(load_tan(C, ak, ai, base, rec, d)));
            break;
        case OP_MUL:
            for (int d = 0; d < n; ++d) {
                iv t;
                if (az) t = iv_mul(A, load_tan(C, bk, bi, base, rec, d));
                else if (bz) t = iv_mul(load_tan(C, ak, ai, base, rec, d), B);
                else t = iv_fma(A, load_tan(C, bk, bi, base, rec, d), iv_mul(load_tan(C, ak, ai, base, rec, d), B));
                C.F.put(o + 2 + 2 * d, t);
            }
            break;
        case OP_DIV: {
            const iv R = iv_recip(B);
            for (int d = 0; d < n; ++d) {
                iv t;
                if (bz) t = iv_mul(load_tan(C, ak, ai, base, rec, d), R);
                else if (az) t = iv_mul(iv_neg(iv_mul(V, load_tan(C, bk, bi, base, rec, d))), R);
                else t = iv_mul(iv_fma(iv_neg(V), load_tan(C, bk, bi, base, rec, d), load_tan(C, ak, ai, base, rec, d)), R);
                C.F.put(o + 2 + 2 * d, t);
            }
        } break;
        case OP_SQR: {
            const iv D = iv_twice(A);
            for (int d = 0; d < n; ++d) C.F.put(o + 2 + 2 * d, iv_mul(D, load_tan(C, ak, ai, base, rec, d)));
        } break;
        case OP_SQRT: {
            const iv R = iv_recip_pos(iv_twice(V));
            for (int d = 0; d < n; ++d) C.F.put(o + 2 + 2 * d, iv_mul(load_tan(C, ak, ai, base, rec, d), R));
        } break;
        case OP_EXP:
            for (int d = 0; d < n; ++d) C.F.put(o + 2 + 2 * d, iv_mul(V, load_tan(C, ak, ai, base, rec, d)));
            break;
        case OP_LOG: {
            const iv R = iv_recip_pos(A);
            for (int d = 0; d < n; ++d) C.F.put(o + 2 + 2 * d, iv_mul(load_tan(C, ak, ai, base, rec, d), R));
        } break;
        }
        C.F.put(o, V);
    }
}

// reverse sweep of one output (reverse-mode interval AD): adjoint slots at
// `abase` (2 units each), forward values in tape records at `tbase`, gradient
// accumulators at `gbase`. Operand a is updated before operand b. A product
// contribution x*y to a slot already written is accumulated with one directed
// rounding per end (iv_fma); the first write stores the product.
__device__ void run_reverse(const RIns* __restrict__ rins, int count, const SweepCtx& C, int abase, int tbase,
                            int gbase) {
    for (int i = 0; i < count; ++i) {
        const RIns R = rins[i];
        const uint32_t op = R.w0 & 31u, wslot = R.w0 >> 16;
        const iv W = C.F.get(abase + 2 * (int)wslot);
        if (op == OP_VAR) {
            const int g = gbase + 2 * (int)R.w1;
            C.F.put(g, iv_add(C.F.get(g), W));
            continue;
        }
        const bool a_init = (R.w0 >> 5) & 1u, b_init = (R.w0 >> 6) & 1u;
        const bool a_none = (R.w0 >> 7) & 1u, b_none = (R.w0 >> 8) & 1u;
        const uint32_t Ak = (R.w3 >> 16) & 3u, Bk = (R.w3 >> 18) & 3u;
        // contribution to operand a: ax * ay (a_prod) or +-W; to operand b likewise
        iv ax = W, ay = W, bx = W, by = W;
        bool a_prod = true, b_prod = true, sub_b = false, sub_a = false;
        switch (op) {
        case OP_ADD: a_prod = b_prod = false; break;
        case OP_SUB: a_prod = b_prod = false; sub_b = true; break;
        case OP_NEG: a_prod = false; sub_a = true; break;
        case OP_MUL: {
            ay = load_val(C, Bk, R.w2 >> 16, tbase, 2);
            by = load_val(C, Ak, R.w2 & 0xFFFFu, tbase, 2);
        } break;
        case OP_DIV: {
            const iv B = load_val(C, Bk, R.w2 >> 16, tbase, 2);
            const iv V = C.F.get(tbase + 2 * (int)(R.w3 & 0xFFFFu));
            ay = iv_recip(B);
            bx = iv_neg(iv_mul(W, V));            // b gets -(W V) / B
            by = ay;
        } break;
        case OP_SQR: ay = iv_twice(load_val(C, Ak, R.w2 & 0xFFFFu, tbase, 2)); break;
        case OP_SQRT: ay = iv_recip_pos(iv_twice(C.F.get(tbase + 2 * (int)(R.w3 & 0xFFFFu)))); break;
        case OP_EXP: ay = C.F.get(tbase + 2 * (int)(R.w3 & 0xFFFFu)); break;
        case OP_LOG: ay = iv_recip_pos(load_val(C, Ak, R.w2 & 0xFFFFu, tbase, 2)); break;
        default: a_prod = b_prod = false; ax = bx = entire();
        }
        if (!a_none) {
            const int u = abase + 2 * (int)(R.w1 & 0xFFFFu);
            iv v;
            if (a_prod) v = a_init ? iv_mul(ax, ay) : iv_fma(ax, ay, C.F.get(u));
            else if (a_init) v = sub_a ? iv_neg(ax) : ax;
            else v = sub_a ? iv_sub(C.F.get(u), ax) : iv_add(C.F.get(u), ax);
            C.F.put(u, v);
        }
        if (!b_none) {
            const int u = abase + 2 * (int)(R.w1 >> 16);
            iv v;
            if (b_prod) v = b_init ? iv_mul(bx, by) : iv_fma(bx, by, C.F.get(u));
            else if (b_init) v = sub_b ? iv_neg(bx) : bx;
            else v = sub_b ? iv_sub(C.F.get(u), bx) : iv_add(C.F.get(u), bx);
            C.F.put(u, v);
        }
    }
}

// --------------------------------------------------------------- the kernel
template <int MODE>
__global__ void __launch_bounds__(512) k_bound(const KParams P) {
    extern __shared__ double smem[];
    const ProgDesc& G = *P.prog;
    const int n = G.n, n_out = G.n_out;
    const FrameLayout L = G.L;
    SweepCtx C;
    if (P.frame_in_smem) C.F.p = smem + threadIdx.x;
    else C.F.p = P.gframe + (size_t)blockIdx.x * P.frame_units * blockDim.x + threadIdx.x;
    C.F.s = blockDim.x;
    C.consts = G.consts;
    C.x_base = L.x_base;
    C.c_base = L.c_base;

    tile_loop(P, [&](const Sub& s) {
        const long long g = s.g;
        const bool valid = s.valid;
        if (valid) {
            // ---- Step 1: decode X_k and c
            unsigned int kk = s.k;
            for (int i = 0; i < n; ++i) {
                iv X;
                double c;
                decode_dim(s.rec, n, i, kk, X, c);
                C.F.put(L.x_base + 2 * i, X);
                C.F.st(L.c_base + i, c);
            }
            // ---- Step 2a: rigorous point value f(c) of every output
            C.point = true;
            run_values(G.ins + G.pt_begin, G.pt_count, C, L.phase_base);
            for (int o = 0; o < n_out; ++o)
                C.F.put(L.fc_base + 2 * o, load_val(C, G.pt_out_kind[o], G.pt_out_ref[o], L.phase_base, 2));
            C.point = false;
        }
        // ---- Step 2b: gradient enclosures and the Mean Value Form, output by output.
        // With the natural interval extension alone (form 1) a reduce launch needs no
        // gradients: only the value sweep over X_k.
        const bool nie_only = (MODE == KM_FWD_REDUCE || MODE == KM_ADJ_REDUCE) && P.form == 1;
        bool cert_infeasible = false;
        double obj_lo = from_bits(0x7FF0000000000000LL);
        if (MODE == KM_FWD_REDUCE || MODE == KM_FWD_STORE) {
            if (valid) {
                if (nie_only) run_values(G.ins + G.tan_begin, G.tan_count, C, L.phase_base);
                else run_tangents(G.ins + G.tan_begin, G.tan_count, C, L.phase_base, n);
            }
        }
        for (int o = 0; o < n_out; ++o) {
            iv F = zero(), Fc = zero();
            if (valid && nie_only) {
                Fc = C.F.get(L.fc_base + 2 * o);
                iv nie;
                if (MODE == KM_FWD_REDUCE) {
                    nie = load_val(C, G.tan_out_kind[o], G.tan_out_ref[o], L.phase_base, 2);
                } else {
                    const AdjProgram& A = G.adj[o];
                    const int tb = L.phase_base + 2 * n + 2 * A.adj_slots;
                    run_values(G.ins + A.fw_begin, A.fw_count, C, tb);
                    nie = load_val(C, A.out_kind_ref, A.out_ref, tb, 2);
                }
                F = final_form(1, nie, nie);
                if (excludes_feasible(G.out_kind[o], F)) cert_infeasible = true;
                if (o == G.obj) obj_lo = F.lo;
            } else if (valid) {
                Fc = C.F.get(L.fc_base + 2 * o);
                iv nie;
                int gunit, gstride;  // gradient of this output: unit of G_0 and stride (0: constant/variable)
                if (MODE == KM_FWD_REDUCE || MODE == KM_FWD_STORE) {
                    const int rec = L.tan_rec;
                    const uint32_t kind = G.tan_out_kind[o], ref = G.tan_out_ref[o];
                    nie = load_val(C, kind, ref, L.phase_base, rec);
                    if (kind == K_SLOT) { gunit = L.phase_base + (int)ref * rec + 2; gstride = 2; }
                    else { gunit = (kind == K_VAR) ? (int)ref : -1; gstride = 0; }
                } else {
                    const AdjProgram& A = G.adj[o];
                    const int gb = L.phase_base, ab = gb + 2 * n, tb = ab + 2 * A.adj_slots;
                    run_values(G.ins + A.fw_begin, A.fw_count, C, tb);
                    for (int i = 0; i < n; ++i) C.F.put(gb + 2 * i, zero());
                    if (A.out_wslot >= 0) C.F.put(ab + 2 * A.out_wslot, one());
                    run_reverse(G.rins + A.rv_begin, A.rv_count, C, ab, tb, gb);
                    nie = load_val(C, A.out_kind_ref, A.out_ref, tb, 2);
                    gunit = gb;
                    gstride = 2;
                }
                // Mean Value Form (Definition 5): f(c) + sum_i G_i (X_i - c_i), left to right
                iv mvf = Fc;
                for (int i = 0; i < n; ++i) {
                    const iv Gi = gstride ? C.F.get(gunit + 2 * i) : ((gunit == i) ? one() : zero());
                    mvf = mvf_term(mvf, Gi, C.F.get(L.x_base + 2 * i), C.F.ld(L.c_base + i));
                    if ((MODE == KM_FWD_STORE || MODE == KM_ADJ_STORE) && P.outG) {
                        const long long q0 = g - P.store_first_g;
                        double* q = P.outG + ((size_t)q0 * n_out + o) * n * 2 + 2 * i;
                        q[0] = Gi.lo;
                        q[1] = Gi.hi;
                    }
                }
                F = final_form(P.form, mvf, nie);
                if (excludes_feasible(G.out_kind[o], F)) cert_infeasible = true;
                if (o == G.obj) obj_lo = F.lo;
            }
            if (MODE == KM_FWD_STORE || MODE == KM_ADJ_STORE) {
                if (valid) {
                    const long long q0 = g - P.store_first_g;
                    P.outF[((size_t)q0 * n_out + o) * 2] = F.lo;
                    P.outF[((size_t)q0 * n_out + o) * 2 + 1] = F.hi;
                    if (P.outFc) {
                        P.outFc[((size_t)q0 * n_out + o) * 2] = Fc.lo;
                        P.outFc[((size_t)q0 * n_out + o) * 2 + 1] = Fc.hi;
                    }
                }
            } else {
                // ---- Step 3: refinement hull per node and output
                reduce_output(P, s, n_out, o, F);
            }
        }
        if (MODE == KM_FWD_REDUCE || MODE == KM_ADJ_REDUCE) {
            double ub = from_bits(0x7FF0000000000000LL);
            if (valid) {
                bool feas = !G.has_eq;
                for (int o = 0; o < n_out; ++o)
                    if (G.out_kind[o] == OUT_INEQ && !le0(C.F.ld(L.fc_base + 2 * o + 1))) feas = false;
                if (feas) ub = C.F.ld(L.fc_base + 2 * G.obj + 1);
                if (cert_infeasible) obj_lo = from_bits(0x7FF0000000000000LL);
            }
            reduce_extras(P, s, n_out, ub, obj_lo);
        }
    });
}

}  // namespace ivb
namespace ivb {

// ------------------------------------------------------------ node results
__global__ void k_init_keys(unsigned long long* keys, const char* queue, int n_out) {
    const int n_nodes = (int)reinterpret_cast<const long long*>(queue)[0];
    const int K = 2 * n_out + 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes * K; i += gridDim.x * blockDim.x) {
        const int slot = i % K;
        const bool is_max = slot >= n_out && slot < 2 * n_out;
        keys[i] = is_max ? 0ULL : ~0ULL;
    }
}

// Section 3.1 Step 3 and pruning: lb = lower end of the objective's
// refinement (or the filtered minimum), infeasible when an inequality's lower
// end is > 0 or an equality's refinement excludes 0.
__global__ void k_finalize(const FinalizeParams F) {
    const int nd = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_nodes = (int)reinterpret_cast<const long long*>(F.queue)[0];
    if (nd >= n_nodes) return;
    const int K = 2 * F.n_out + 2;
    const unsigned long long* k = F.keys + (size_t)nd * K;
    uint8_t inf = 0;
    for (int o = 0; o < F.n_out; ++o) {
        const double lo = unkey(k[o]), hi = unkey(k[F.n_out + o]);
        if (F.out_kind[o] == OUT_INEQ && gt0(lo)) inf = 1;
        if (F.out_kind[o] == OUT_EQ && (gt0(lo) || lt0(hi))) inf = 1;
        if (F.minlo) F.minlo[(size_t)nd * F.n_out + o] = lo;
        if (F.maxhi) F.maxhi[(size_t)nd * F.n_out + o] = hi;
    }
    double lb = unkey(k[F.obj]);
    if (F.filter) {
        lb = unkey(k[2 * F.n_out + 1]);
        if (isinf_(lb) && gt0(lb)) inf = 1;
    }
    if (F.lb) F.lb[nd] = lb;
    if (F.inf) F.inf[nd] = inf;
    if (F.ub) F.ub[nd] = unkey(k[2 * F.n_out]);
}

// ------------------------------------------------- round-to-nearest gradients
// Point value and reverse-mode gradient of every output at x (plain double,
// same local partials as the interval rules), one thread per point. Uses the
// adjoint programs: forward values into tape records, adjoints into slots.
__device__ __forceinline__ double pload(const Frame& F, uint32_t kind, uint32_t idx, int base,
                                        const double* x, const double* consts) {
    if (kind == K_SLOT) return F.ld(base + (int)idx);
    if (kind == K_VAR) return x[idx];
    return __ldg(consts + idx);
}

__global__ void __launch_bounds__(256) k_point_grad(const ProgDesc* __restrict__ prog, long long n_points,
                                                   const double* __restrict__ X, double* f, double* grad,
                                                   double* gframe, int frame_units) {
    const ProgDesc& G = *prog;
    const int n = G.n, n_out = G.n_out;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n_points;
         p += (long long)gridDim.x * blockDim.x) {
        Frame F;
        F.p = gframe + (size_t)blockIdx.x * frame_units * blockDim.x + threadIdx.x;
        F.s = blockDim.x;
        const double* x = X + (size_t)p * n;
        for (int o = 0; o < n_out; ++o) {
            const AdjProgram& A = G.adj[o];
            const int gb = 0, ab = n, tb = ab + A.adj_slots;
            for (int i = 0; i < A.fw_count; ++i) {
                const Ins I = G.ins[A.fw_begin + i];
                const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
                const double a = pload(F, ak, I.w1 & 0xFFFFu, tb, x, G.consts);
                const double b = (bk != K_NONE) ? pload(F, bk, I.w1 >> 16, tb, x, G.consts) : a;
                double v;
                switch (op) {
                case OP_ADD: v = __dadd_rn(a, b); break;
                case OP_SUB: v = __dsub_rn(a, b); break;
                case OP_MUL: v = __dmul_rn(a, b); break;
                case OP_DIV: v = __ddiv_rn(a, b); break;
                case OP_SQR: v = __dmul_rn(a, a); break;
                case OP_SQRT: v = __dsqrt_rn(a); break;
                case OP_EXP: v = exp(a); break;
                case OP_LOG: v = log(a); break;
                case OP_NEG: v = -a; break;
                default: v = __longlong_as_double(0x7FF8000000000000LL);
                }
                F.st(tb + (int)dst, v);
            }
            f[(size_t)p * n_out + o] = pload(F, A.out_kind_ref, A.out_ref, tb, x, G.consts);
            if (!grad) continue;
            for (int i = 0; i < n; ++i) F.st(gb + i, 0.0);
            if (A.out_wslot >= 0) F.st(ab + A.out_wslot, 1.0);
            for (int i = 0; i < A.rv_count; ++i) {
                const RIns R = G.rins[A.rv_begin + i];
                const uint32_t op = R.w0 & 31u, wslot = R.w0 >> 16;
                const double w = F.ld(ab + (int)wslot);
                if (op == OP_VAR) { F.st(gb + (int)R.w1, __dadd_rn(F.ld(gb + (int)R.w1), w)); continue; }
                const bool a_init = (R.w0 >> 5) & 1u, b_init = (R.w0 >> 6) & 1u;
                const bool a_none = (R.w0 >> 7) & 1u, b_none = (R.w0 >> 8) & 1u;
                const uint32_t Ak = (R.w3 >> 16) & 3u, Bk = (R.w3 >> 18) & 3u;
                double ca = 0.0, cb = 0.0;
                bool sub_a = false, sub_b = false;
                switch (op) {
                case OP_ADD: ca = w; cb = w; break;
                case OP_SUB: ca = w; cb = w; sub_b = true; break;
                case OP_NEG: ca = w; sub_a = true; break;
                case OP_MUL:
                    ca = __dmul_rn(w, pload(F, Bk, R.w2 >> 16, tb, x, G.consts));
                    cb = __dmul_rn(w, pload(F, Ak, R.w2 & 0xFFFFu, tb, x, G.consts));
                    break;
                case OP_DIV: {
                    const double r = __ddiv_rn(1.0, pload(F, Bk, R.w2 >> 16, tb, x, G.consts));
                    const double v = F.ld(tb + (int)(R.w3 & 0xFFFFu));
                    ca = __dmul_rn(w, r);
                    cb = __dmul_rn(__dmul_rn(w, v), r);
                    sub_b = true;
                } break;
                case OP_SQR: ca = __dmul_rn(w, __dmul_rn(2.0, pload(F, Ak, R.w2 & 0xFFFFu, tb, x, G.consts))); break;
                case OP_SQRT:
                    ca = __dmul_rn(w, __ddiv_rn(1.0, __dmul_rn(2.0, F.ld(tb + (int)(R.w3 & 0xFFFFu)))));
                    break;
                case OP_EXP: ca = __dmul_rn(w, F.ld(tb + (int)(R.w3 & 0xFFFFu))); break;
                case OP_LOG: ca = __dmul_rn(w, __ddiv_rn(1.0, pload(F, Ak, R.w2 & 0xFFFFu, tb, x, G.consts))); break;
                }
                if (!a_none) {
                    const int u = ab + (int)(R.w1 & 0xFFFFu);
                    const double c = sub_a ? -ca : ca;
                    F.st(u, a_init ? c : (sub_a ? __dsub_rn(F.ld(u), ca) : __dadd_rn(F.ld(u), ca)));
                }
                if (!b_none) {
                    const int u = ab + (int)(R.w1 >> 16);
                    const double c = sub_b ? -cb : cb;
                    F.st(u, b_init ? c : (sub_b ? __dsub_rn(F.ld(u), cb) : __dadd_rn(F.ld(u), cb)));
                }
            }
            for (int i = 0; i < n; ++i) grad[((size_t)p * n_out + o) * n + i] = F.ld(gb + i);
        }
    }
}

// ------------------------------------------------------------ test hook
// opcode: tape opcodes of the interval operations, 100 for the reciprocal,
// 101..104 for +, -, *, sqr with every endpoint operation emulated on the
// integer pipes (policy 15 of ivb_iv.cuh)
__device__ __forceinline__ iv eval_hook(int opcode, iv X, iv Y) {
    switch (opcode) {
    case 100: return iv_recip(X);
    case 101: return iv_add_t<15>(X, Y);
    case 102: return iv_sub_t<15>(X, Y);
    case 103: return iv_mul_t<15>(X, Y);
    case 104: return iv_sqr_t<15>(X);
    }
    return eval_value((uint32_t)opcode, X, Y);
}

__global__ void k_eval_op(int opcode, long long n, const double* __restrict__ x, const double* __restrict__ y,
                          double* r) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const iv X = mk(x[2 * i], x[2 * i + 1]);
        const iv Y = y ? mk(y[2 * i], y[2 * i + 1]) : X;
        const iv R = opcode == 105 ? iv_fma(X, Y, mk(r[2 * i], r[2 * i + 1])) : eval_hook(opcode, X, Y);
        r[2 * i] = R.lo;
        r[2 * i + 1] = R.hi;
    }
}

cudaError_t launch_eval_op(int opcode, long long n, const double* x, const double* y, double* r, cudaStream_t s) {
    const int block = 256;
    const long long g = (n + block - 1) / block;
    k_eval_op<<<(int)(g < 4096 ? g : 4096), block, 0, s>>>(opcode, n, x, y, r);
    return cudaGetLastError();
}

// ------------------------------------------------------------ own-primitive probe
// throughput of this library's directed primitives (ivb_fp64x.cuh), the
// same shape as ivb_probe.cu: 8 independent chains per thread
template <int W>
__global__ void k_own_probe(double* out, double seed, int iters) {
    double x[8];
    const double y = seed + threadIdx.x * 1e-12;
    for (int j = 0; j < 8; ++j) x[j] = 1.5 + j * 1e-3 + threadIdx.x * 1e-9;
    for (int i = 0; i < iters; ++i) {
        // factors and addends that keep the multiply / add chains near 1.5
        const double f = (i & 1) ? 1.0000001192092896 : 0.99999988079071045;
        const double d = (i & 1) ? 0.0009765625 : -0.0009765625;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (W == 0) x[j] = rcp_dir_pos(x[j], false);
            if (W == 1) x[j] = div_dir_pos(y, x[j], rcp_refined(x[j]), false);
            if (W == 2) x[j] = sqrt_dir(x[j] * 3.1, false);   // one multiply keeps x off powers of two
            if (W == 3) x[j] = exp_dir(-x[j], false);
            if (W == 4) x[j] = __dadd_rn(log_dir(x[j], false), 2.0);
            // integer-pipe emulation (ivb_emu.cuh) alone, and beside the FP64 pipe (half the chains each)
            if (W == 5) x[j] = mul_ru_emu(x[j], f);
            if (W == 6) x[j] = (j & 1) ? mul_ru_emu(x[j], f) : __dmul_ru(x[j], f);
            if (W == 7) x[j] = add_ru_emu(x[j], d);
            if (W == 8) x[j] = (j & 1) ? add_ru_emu(x[j], d) : __dadd_ru(x[j], d);
        }
    }
    double acc = 0.0;
    for (int j = 0; j < 8; ++j) acc += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int W>
static cudaError_t own_probe_run(double* out, int grid, int block, int iters, float* ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_own_probe<W><<<grid, block>>>(out, 1.0000001, iters / 4 + 1);
    cudaEventRecord(a);
    k_own_probe<W><<<grid, block>>>(out, 1.0000001, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t run_own_probe(int which, double* out, int grid, int block, int iters, float* ms) {
    cudaError_t e = init_math_tables();
    if (e != cudaSuccess) return e;
    switch (which) {
    case 0: return own_probe_run<0>(out, grid, block, iters, ms);
    case 1: return own_probe_run<1>(out, grid, block, iters, ms);
    case 2: return own_probe_run<2>(out, grid, block, iters, ms);
    case 3: return own_probe_run<3>(out, grid, block, iters, ms);
    case 4: return own_probe_run<4>(out, grid, block, iters, ms);
    case 5: return own_probe_run<5>(out, grid, block, iters, ms);
    case 6: return own_probe_run<6>(out, grid, block, iters, ms);
    case 7: return own_probe_run<7>(out, grid, block, iters, ms);
    default: return own_probe_run<8>(out, grid, block, iters, ms);
    }
}

// exp/log tables in extended precision on the host (long double: 64-bit
// significand on x86-64, binary128 on AArch64), split into double hi + lo
// (the exp table keeps hi, and hi and lo rounded to float)
cudaError_t math_tables_address(void** ptr, size_t* bytes) {
    *bytes = sizeof(MathTables);
    return cudaGetSymbolAddress(ptr, g_math);
}

cudaError_t init_math_tables() {
    static bool done[256] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 256 && done[dev]) return cudaSuccess;
    static MathTables h;
    for (int j = 0; j < kExpTab; ++j) {
        const long double v = exp2l((long double)j / kExpTab);
        h.exp[j].hi = (double)v;
        h.exp[j].hi_f = (float)h.exp[j].hi;
        h.exp[j].lo_f = (float)(v - (long double)h.exp[j].hi);
    }
    const long double T = kLogTab;
    for (int j = 0; j < kLogTab; ++j) {
        // y in [1 + j/T, 1 + (j+1)/T); the upper half is folded to y/2 in [0.75, 1);
        // the two intervals next to 1 use c = 1 so that r = y - 1 is exact
        double c = 1.0;
        if (j != 0 && j != kLogTab - 1) {
            const long double F = (j < kLogTab / 2) ? 1.0L + (j + 0.5L) / T : (1.0L + (j + 0.5L) / T) / 2.0L;
            c = (double)(1.0L / F);
        }
        const long double L = -logl((long double)c);
        h.log[j].c = c;
        h.log[j].hi = (double)L;
        h.log[j].lo = (double)(L - (long double)h.log[j].hi);
        h.log[j].pad = 0.0;
    }
    e = cudaMemcpyToSymbol(g_math, &h, sizeof(h));
    if (e == cudaSuccess && dev >= 0 && dev < 256) done[dev] = true;
    return e;
}

// ------------------------------------------------------------ host wrappers
static const void* bound_fn(int mode) {
    switch (mode) {
    case KM_FWD_REDUCE: return (const void*)k_bound<KM_FWD_REDUCE>;
    case KM_ADJ_REDUCE: return (const void*)k_bound<KM_ADJ_REDUCE>;
    case KM_FWD_STORE: return (const void*)k_bound<KM_FWD_STORE>;
    default: return (const void*)k_bound<KM_ADJ_STORE>;
    }
}

cudaError_t set_bound_smem_limit(int mode, int bytes) {
    return cudaFuncSetAttribute(bound_fn(mode), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int occupancy_blocks(int mode, int block, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bound_fn(mode), block, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_bound(int mode, const KParams& P, int grid, int block, size_t smem, cudaStream_t s) {
    switch (mode) {
    case KM_FWD_REDUCE: k_bound<KM_FWD_REDUCE><<<grid, block, smem, s>>>(P); break;
    case KM_ADJ_REDUCE: k_bound<KM_ADJ_REDUCE><<<grid, block, smem, s>>>(P); break;
    case KM_FWD_STORE: k_bound<KM_FWD_STORE><<<grid, block, smem, s>>>(P); break;
    default: k_bound<KM_ADJ_STORE><<<grid, block, smem, s>>>(P); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_keys(unsigned long long* keys, const char* queue, int max_nodes, int n_out, cudaStream_t s) {
    const int total = max_nodes * (2 * n_out + 2);
    const int block = 256, grid = (total + block - 1) / block < 1024 ? (total + block - 1) / block : 1024;
    k_init_keys<<<grid, block, 0, s>>>(keys, queue, n_out);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeParams& F, cudaStream_t s) {
    const int block = 128, grid = (F.max_nodes + block - 1) / block;
    k_finalize<<<grid, block, 0, s>>>(F);
    return cudaGetLastError();
}

cudaError_t launch_point_grad(const ProgDesc* prog, int n, int n_out, int frame_units, long long n_points,
                              const double* x, double* f, double* grad, double* gframe, int grid, int block,
                              cudaStream_t s) {
    (void)n; (void)n_out;
    k_point_grad<<<grid, block, 0, s>>>(prog, n_points, x, f, grad, gframe, frame_units);
    return cudaGetLastError();
}

}  // namespace ivb
