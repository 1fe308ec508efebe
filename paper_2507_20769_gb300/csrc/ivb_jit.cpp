// ivb_jit.cpp -- tape-specialised bounding kernels.
//
// The tape interpreter (ivb_kernels.cu) fetches, decodes and dispatches every
// instruction at run time and keeps every interval in per-thread frame memory.
// At problem creation, when asked to, this file writes the very programs the
// interpreter runs (the point sweep on [c,c], then per output either the
// tangent sweep or the forward sweep plus reverse adjoint sweep of Section
// 3.2) out as straight-line CUDA C++ -- one statement per instruction, frame
// records turned into named local variables -- around the shared tile loop,
// decoding, Mean Value Form sum and reductions of ivb_bound_common.cuh,
// compiles it with NVRTC for sm_103a and loads it as a CUDA library.
//
// Every statement calls the same interval primitive on the same operands as
// the interpreter does, in the same order wherever the order changes a
// rounded result (fused adjoint accumulation, the MVF sum), so the bounds are
// bit-identical to the interpreter's. What changes: no instruction stream,
// operands in registers, and the compiler is free to interleave independent
// operations, which hides the latency of the narrow FP64 pipe.
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_internal.h"
#include "ivb_jit.h"
#include "ivb_kernels.h"

// device headers as strings (written by the build from csrc/)
#include "ivb_jit_headers.inc"

namespace ivb {

namespace {

// exact hexadecimal literal of a finite double
std::string lit(double v) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%a", v);
    return std::string("(") + buf + ")";
}

std::string S(long long v) { return std::to_string(v); }

struct Gen {
    const HostProgram& P;
    const Ins* ins;
    const RIns* rins;
    const double* consts;
    int n, no;
    bool nie_only = false;   // form 1 (natural interval extension alone): no gradients needed
    std::string out;

    void line(int ind, const std::string& s) {
        out.append((size_t)ind * 2, ' ');
        out += s;
        out += '\n';
    }

    std::string konst(uint32_t idx) const { return "mk(" + lit(consts[idx]) + ", " + lit(consts[idx]) + ")"; }

    // value operand: role 'p' point sweep (variables read [c,c]), 't' tangent
    // records, 'r' adjoint tape records (variables read X)
    std::string val(char role, uint32_t kind, uint32_t idx) const {
        if (kind == K_SLOT) return std::string(1, role) + S(idx);
        if (kind == K_VAR) return role == 'p' ? "mk(c" + S(idx) + ", c" + S(idx) + ")" : "X" + S(idx);
        return konst(idx);
    }

    static std::string eval(uint32_t op, const std::string& A, const std::string& B) {
        switch (op) {
        case OP_ADD: return "iv_add(" + A + ", " + B + ")";
        case OP_SUB: return "iv_sub(" + A + ", " + B + ")";
        case OP_MUL: return "iv_mul(" + A + ", " + B + ")";
        case OP_DIV: return "iv_div(" + A + ", " + B + ")";
        case OP_SQR: return "iv_sqr(" + A + ")";
        case OP_SQRT: return "iv_sqrt(" + A + ")";
        case OP_EXP: return "iv_exp(" + A + ")";
        case OP_LOG: return "iv_log(" + A + ")";
        case OP_NEG: return "iv_neg(" + A + ")";
        }
        return "entire()";
    }

    void decls(int ind, const char* prefix, int count) {
        for (int i = 0; i < count; i += 8) {
            std::string s = "iv ";
            for (int j = i; j < count && j < i + 8; ++j) s += (j > i ? ", " : "") + std::string(prefix) + S(j) + " = zero()";
            line(ind, s + ";");
        }
    }

    // straight-line value sweep (run_values): dst record of each instruction
    void values(int ind, char role, int begin, int count) {
        for (int i = begin; i < begin + count; ++i) {
            const Ins I = ins[i];
            const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
            const std::string A = val(role, ak, I.w1 & 0xFFFFu);
            const std::string B = bk != K_NONE ? val(role, bk, I.w1 >> 16) : A;
            line(ind, std::string(1, role) + S(dst) + " = " + eval(op, A, B) + ";");
        }
    }

    // tangent of an operand in direction d (load_tan)
    std::string tan(uint32_t kind, uint32_t idx, int d) const {
        if (kind == K_SLOT) return "t" + S(idx) + "_" + S(d);
        if (kind == K_VAR) return (int)idx == d ? "one()" : "zero()";
        return "zero()";
    }

    // forward-mode sweep (run_tangents), records t<k> and t<k>_<d>
    void tangents(int ind) {
        for (int i = P.tan_begin; i < P.tan_begin + P.tan_count; ++i) {
            const Ins I = ins[i];
            const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
            const uint32_t ai = I.w1 & 0xFFFFu, bi = I.w1 >> 16;
            const bool az = ak == K_CONST, bz = bk == K_CONST || bk == K_NONE;
            line(ind, "{");
            const int j = ind + 1;
            line(j, "const iv A = " + val('t', ak, ai) + ";");
            line(j, std::string("const iv B = ") + (bk != K_NONE ? val('t', bk, bi) : "A") + ";");
            line(j, "const iv V = " + eval(op, "A", "B") + ";");
            const std::string T = "t" + S(dst) + "_";
            switch (op) {
            case OP_ADD:
                for (int d = 0; d < n; ++d)
                    line(j, T + S(d) + " = " +
                                (az ? tan(bk, bi, d) : bz ? tan(ak, ai, d)
                                                          : "iv_add(" + tan(ak, ai, d) + ", " + tan(bk, bi, d) + ")") + ";");
                break;
            case OP_SUB:
                for (int d = 0; d < n; ++d)
                    line(j, T + S(d) + " = " +
                                (az ? "iv_neg(" + tan(bk, bi, d) + ")"
                                    : bz ? tan(ak, ai, d) : "iv_sub(" + tan(ak, ai, d) + ", " + tan(bk, bi, d) + ")") + ";");
                break;
            case OP_NEG:
                for (int d = 0; d < n; ++d) line(j, T + S(d) + " = iv_neg(" + tan(ak, ai, d) + ");");
                break;
            case OP_MUL:
                for (int d = 0; d < n; ++d) {
                    std::string t;
                    if (az) t = "iv_mul(A, " + tan(bk, bi, d) + ")";
                    else if (bz) t = "iv_mul(" + tan(ak, ai, d) + ", B)";
                    else t = "iv_fma(A, " + tan(bk, bi, d) + ", iv_mul(" + tan(ak, ai, d) + ", B))";
                    line(j, T + S(d) + " = " + t + ";");
                }
                break;
            case OP_DIV:
                line(j, "const iv R = iv_recip(B);");
                for (int d = 0; d < n; ++d) {
                    std::string t;
                    if (bz) t = "iv_mul(" + tan(ak, ai, d) + ", R)";
                    else if (az) t = "iv_mul(iv_neg(iv_mul(V, " + tan(bk, bi, d) + ")), R)";
                    else t = "iv_mul(iv_fma(iv_neg(V), " + tan(bk, bi, d) + ", " + tan(ak, ai, d) + "), R)";
                    line(j, T + S(d) + " = " + t + ";");
                }
                break;
            case OP_SQR:
                line(j, "const iv D = iv_twice(A);");
                for (int d = 0; d < n; ++d) line(j, T + S(d) + " = iv_mul(D, " + tan(ak, ai, d) + ");");
                break;
            case OP_SQRT:
                line(j, "const iv R = iv_recip_pos(iv_twice(V));");
                for (int d = 0; d < n; ++d) line(j, T + S(d) + " = iv_mul(" + tan(ak, ai, d) + ", R);");
                break;
            case OP_EXP:
                for (int d = 0; d < n; ++d) line(j, T + S(d) + " = iv_mul(V, " + tan(ak, ai, d) + ");");
                break;
            case OP_LOG:
                line(j, "const iv R = iv_recip_pos(A);");
                for (int d = 0; d < n; ++d) line(j, T + S(d) + " = iv_mul(" + tan(ak, ai, d) + ", R);");
                break;
            }
            line(j, "t" + S(dst) + " = V;");
            line(ind, "}");
        }
    }

    // reverse sweep of one output (run_reverse): adjoint slots w<k>, tape
    // records r<k>, gradient accumulators g<i>
    void reverse(int ind, const AdjProgram& A) {
        for (int i = A.rv_begin; i < A.rv_begin + A.rv_count; ++i) {
            const RIns R = rins[i];
            const uint32_t op = R.w0 & 31u, wslot = R.w0 >> 16;
            const std::string W = "w" + S(wslot);
            if (op == OP_VAR) {
                const std::string g = "g" + S(R.w1);
                line(ind, g + " = iv_add(" + g + ", " + W + ");");
                continue;
            }
            const bool a_init = (R.w0 >> 5) & 1u, b_init = (R.w0 >> 6) & 1u;
            const bool a_none = (R.w0 >> 7) & 1u, b_none = (R.w0 >> 8) & 1u;
            const uint32_t Ak = (R.w3 >> 16) & 3u, Bk = (R.w3 >> 18) & 3u;
            const std::string Av = val('r', Ak, R.w2 & 0xFFFFu), Bv = val('r', Bk, R.w2 >> 16);
            const std::string V = "r" + S(R.w3 & 0xFFFFu);
            // contribution to operand a: ax * ay (a_prod) or +-W; to operand b likewise
            std::string ax = "W", ay, bx = "W", by;
            bool a_prod = true, b_prod = true, sub_a = false, sub_b = false;
            line(ind, "{");
            const int j = ind + 1;
            line(j, "const iv W = " + W + ";");
            switch (op) {
            case OP_ADD: a_prod = b_prod = false; break;
            case OP_SUB: a_prod = b_prod = false; sub_b = true; break;
            case OP_NEG: a_prod = false; sub_a = true; break;
            case OP_MUL: ay = Bv; by = Av; break;
            case OP_DIV:
                line(j, "const iv Rb = iv_recip(" + Bv + ");");
                ay = "Rb";
                if (!b_none) {
                    line(j, "const iv nb = iv_neg(iv_mul(W, " + V + "));");   // b gets -(W V) / B
                    bx = "nb";
                }
                by = "Rb";
                break;
            case OP_SQR: ay = "iv_twice(" + Av + ")"; break;
            case OP_SQRT: ay = "iv_recip_pos(iv_twice(" + V + "))"; break;
            case OP_EXP: ay = V; break;
            case OP_LOG: ay = "iv_recip_pos(" + Av + ")"; break;
            default: a_prod = b_prod = false; ax = bx = "entire()";
            }
            // the factors are formed before either slot is written
            if (!a_none && a_prod) line(j, "const iv ya = " + ay + ";");
            if (!b_none && b_prod) line(j, "const iv yb = " + by + ";");
            if (!a_none) {
                const std::string u = "w" + S(R.w1 & 0xFFFFu);
                std::string v;
                if (a_prod) v = a_init ? "iv_mul(" + ax + ", ya)" : "iv_fma(" + ax + ", ya, " + u + ")";
                else if (a_init) v = sub_a ? "iv_neg(" + ax + ")" : ax;
                else v = sub_a ? "iv_sub(" + u + ", " + ax + ")" : "iv_add(" + u + ", " + ax + ")";
                line(j, u + " = " + v + ";");
            }
            if (!b_none) {
                const std::string u = "w" + S(R.w1 >> 16);
                std::string v;
                if (b_prod) v = b_init ? "iv_mul(" + bx + ", yb)" : "iv_fma(" + bx + ", yb, " + u + ")";
                else if (b_init) v = sub_b ? "iv_neg(" + bx + ")" : bx;
                else v = sub_b ? "iv_sub(" + u + ", " + bx + ")" : "iv_add(" + u + ", " + bx + ")";
                line(j, u + " = " + v + ";");
            }
            line(ind, "}");
        }
    }

    // MVF, form and tests of output o (gradient expressions G_i, NIE expression)
    void finish(int ind, int o, const std::vector<std::string>& Gi, const std::string& nie) {
        line(ind, "{");
        const int j = ind + 1;
        if (nie_only) {
            line(j, "F" + S(o) + " = final_form(1, " + nie + ", " + nie + ");");
        } else {
            line(j, "iv mvf = fc" + S(o) + ";");
            for (int i = 0; i < n; ++i) line(j, "mvf = mvf_term(mvf, " + Gi[i] + ", X" + S(i) + ", c" + S(i) + ");");
            line(j, "F" + S(o) + " = final_form(P.form, mvf, " + nie + ");");
        }
        line(j, "if (excludes_feasible(" + S(P.out_kind[o]) + "u, F" + S(o) + ")) cert = true;");
        if (o == P.obj) line(j, "obj_lo = F" + S(o) + ".lo;");
        line(ind, "}");
    }

    std::string kernel(int mode, int block_max, int min_blocks, int emulate, bool compact, int form) {
        out.clear();
        nie_only = form == 1;
        line(0, "#define IVB_EMU " + S(emulate));
        if (compact) line(0, "#define IVB_HEAVY __noinline__");
        line(0, "typedef signed char int8_t; typedef unsigned char uint8_t;");
        line(0, "typedef short int16_t; typedef unsigned short uint16_t;");
        line(0, "typedef int int32_t; typedef unsigned int uint32_t;");
        line(0, "typedef long long int64_t; typedef unsigned long long uint64_t;");
        line(0, "#include \"ivb_bound_common.cuh\"");
        // compact adjoint mode: the point sweep and each output's sweeps in functions of their own
        const bool split = compact && mode == KM_ADJ_REDUCE;
        if (split) {
            line(0, "namespace ivb {");
            line(0, "__device__ __noinline__ void jit_point(const double* __restrict__ cv, iv* __restrict__ fc) {");
            for (int i = 0; i < n; ++i) line(1, "const double c" + S(i) + " = cv[" + S(i) + "];");
            decls(1, "p", P.pt_slots);
            values(1, 'p', P.pt_begin, P.pt_count);
            for (int o = 0; o < no; ++o)
                line(1, "fc[" + S(o) + "] = " + val('p', (uint32_t)P.pt_out_kind[o], (uint32_t)P.pt_out_ref[o]) + ";");
            line(0, "}");
            for (int o = 0; o < no; ++o) {
                const AdjProgram& A = P.adj[o];
                line(0, "__device__ __noinline__ iv jit_out" + S(o) +
                            "(const iv* __restrict__ Xv, const double* __restrict__ cv, iv fc, int form) {");
                for (int i = 0; i < n; ++i)
                    line(1, "const iv X" + S(i) + " = Xv[" + S(i) + "]; const double c" + S(i) + " = cv[" + S(i) + "];");
                decls(1, "r", A.tape_records);
                values(1, 'r', A.fw_begin, A.fw_count);
                const std::string nie = val('r', (uint32_t)A.out_kind_ref, (uint32_t)A.out_ref);
                if (nie_only) {
                    line(1, "return final_form(1, " + nie + ", " + nie + ");");
                } else {
                    decls(1, "w", A.adj_slots);
                    decls(1, "g", n);
                    if (A.out_wslot >= 0) line(1, "w" + S(A.out_wslot) + " = one();");
                    reverse(1, A);
                    line(1, "iv mvf = fc;");
                    for (int i = 0; i < n; ++i)
                        line(1, "mvf = mvf_term(mvf, g" + S(i) + ", X" + S(i) + ", c" + S(i) + ");");
                    line(1, "return final_form(form, mvf, " + nie + ");");
                }
                line(0, "}");
            }
            line(0, "}  // namespace ivb");
        }
        line(0, "extern \"C\" __global__ void __launch_bounds__(" + S(block_max) + ", " + S(min_blocks) +
                    ") ivb_jit_bound(const ivb::KParams P) {");
        line(1, "using namespace ivb;");
        line(1, "tile_loop(P, [&](const Sub& s) {");
        int d = 2;
        {
            std::string f = "iv ";
            for (int o = 0; o < no; ++o) f += (o ? ", F" : "F") + S(o) + " = zero()";
            line(d, f + ";");
        }
        line(d, "bool cert = false;");
        line(d, "double obj_lo = from_bits(0x7FF0000000000000LL);");
        line(d, "double ub = from_bits(0x7FF0000000000000LL);");
        line(d, "if (s.valid) {");
        d = 3;
        // Step 1
        decls(d, "X", n);
        for (int i = 0; i < n; ++i) line(d, "double c" + S(i) + " = 0.0;");
        line(d, "unsigned int kk = s.k;");
        for (int i = 0; i < n; ++i) line(d, "decode_dim(s.rec, " + S(n) + ", " + S(i) + ", kk, X" + S(i) + ", c" + S(i) + ");");
        // Step 2a: point sweep
        decls(d, "fc", no);
        if (split) {
            std::string xs = "const iv Xv[" + S(n) + "] = {", cs = "const double cv[" + S(n) + "] = {";
            for (int i = 0; i < n; ++i) { xs += (i ? ", X" : "X") + S(i); cs += (i ? ", c" : "c") + S(i); }
            line(d, xs + "};");
            line(d, cs + "};");
            line(d, "iv fcv[" + S(no) + "];");
            line(d, "jit_point(cv, fcv);");
            for (int o = 0; o < no; ++o) line(d, "fc" + S(o) + " = fcv[" + S(o) + "];");
            // Step 2b: one call per output; the tests of finish() on its result
            for (int o = 0; o < no; ++o) {
                line(d, "F" + S(o) + " = jit_out" + S(o) + "(Xv, cv, fc" + S(o) + ", P.form);");
                line(d, "if (excludes_feasible(" + S(P.out_kind[o]) + "u, F" + S(o) + ")) cert = true;");
                if (o == P.obj) line(d, "obj_lo = F" + S(o) + ".lo;");
            }
        } else {
        line(d, "{");
        decls(d + 1, "p", P.pt_slots);
        values(d + 1, 'p', P.pt_begin, P.pt_count);
        for (int o = 0; o < no; ++o)
            line(d + 1, "fc" + S(o) + " = " + val('p', (uint32_t)P.pt_out_kind[o], (uint32_t)P.pt_out_ref[o]) + ";");
        line(d, "}");
        }
        // Step 2b
        if (split) {
        } else if (mode == KM_FWD_REDUCE) {
            line(d, "{");
            const int e = d + 1;
            for (int k = 0; k < P.tan_slots; ++k) {
                line(e, "iv t" + S(k) + " = zero();");
                if (!nie_only) decls(e, ("t" + S(k) + "_").c_str(), n);
            }
            if (nie_only) values(e, 't', P.tan_begin, P.tan_count);
            else tangents(e);
            for (int o = 0; o < no; ++o) {
                const uint32_t kind = (uint32_t)P.tan_out_kind[o], ref = (uint32_t)P.tan_out_ref[o];
                std::vector<std::string> G(n);
                for (int i = 0; i < n; ++i)
                    G[i] = kind == K_SLOT ? "t" + S(ref) + "_" + S(i)
                                          : (kind == K_VAR && (int)ref == i) ? "one()" : "zero()";
                finish(e, o, G, val('t', kind, ref));
            }
            line(d, "}");
        } else {
            for (int o = 0; o < no; ++o) {
                const AdjProgram& A = P.adj[o];
                line(d, "{  // output " + S(o) + ": forward sweep over its cone, then the reverse sweep");
                const int e = d + 1;
                decls(e, "r", A.tape_records);
                values(e, 'r', A.fw_begin, A.fw_count);
                if (!nie_only) {
                    decls(e, "w", A.adj_slots);
                    decls(e, "g", n);
                    if (A.out_wslot >= 0) line(e, "w" + S(A.out_wslot) + " = one();");
                    reverse(e, A);
                }
                std::vector<std::string> G(n);
                for (int i = 0; i < n; ++i) G[i] = "g" + S(i);
                finish(e, o, G, val('r', (uint32_t)A.out_kind_ref, (uint32_t)A.out_ref));
                line(d, "}");
            }
        }
        // certified-feasible centre upper bound; filtered objective
        line(d, std::string("bool feas = ") + (P.has_eq ? "false" : "true") + ";");
        for (int o = 0; o < no; ++o)
            if (P.out_kind[o] == OUT_INEQ) line(d, "if (!le0(fc" + S(o) + ".hi)) feas = false;");
        line(d, "if (feas) ub = fc" + S(P.obj) + ".hi;");
        line(d, "if (cert) obj_lo = from_bits(0x7FF0000000000000LL);");
        line(2, "}");
        for (int o = 0; o < no; ++o) line(2, "reduce_output(P, s, " + S(no) + ", " + S(o) + ", F" + S(o) + ");");
        line(2, "reduce_extras(P, s, " + S(no) + ", ub, obj_lo);");
        line(1, "});");
        line(0, "}");
        return out;
    }
};

}  // namespace

std::string jit_source(const HostProgram& P, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                       const std::vector<double>& consts, int mode, int block_max, int min_blocks, int emulate,
                       bool compact, int form) {
    Gen g{P, ins.data(), rins.data(), consts.data(), P.n_vars, P.n_out};
    return g.kernel(mode, block_max, min_blocks, emulate, compact, form);
}

std::string jit_compile(const std::string& src, std::vector<char>& cubin, std::string& tables_name, double* seconds,
                        int* registers, int* spill_bytes) {
    const auto t0 = std::chrono::steady_clock::now();
    nvrtcProgram prog;
    const int nh = (int)(sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]));
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "ivb_jit_bound.cu", nh, kJitHeaderSources, kJitHeaderNames);
    if (r != NVRTC_SUCCESS) return std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
    nvrtcAddNameExpression(prog, "&ivb::g_math");
    const bool verbose = registers || spill_bytes;
    const char* opts[] = {"-arch=sm_103a", "--fmad=false", "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
    r = nvrtcCompileProgram(prog, verbose ? 5 : 4, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &log[0]);
    std::string err;
    if (r != NVRTC_SUCCESS) {
        err = std::string("NVRTC compilation of the tape-specialised kernel failed: ") + nvrtcGetErrorString(r) +
              "\n" + log.substr(0, 4000);
    } else {
        // ptxas info lines: "Used N registers", "M bytes spill stores"
        auto number_before = [&](const char* key) -> int {
            const size_t at = log.find(key);
            if (at == std::string::npos) return 0;
            size_t b = at;
            while (b > 0 && log[b - 1] == ' ') --b;
            size_t e = b;
            while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
            return b < e ? std::atoi(log.substr(b, e - b).c_str()) : 0;
        };
        auto number_after = [&](const char* key) -> int {
            const size_t at = log.find(key);
            return at == std::string::npos ? -1 : std::atoi(log.c_str() + at + std::strlen(key));
        };
        if (registers) *registers = number_after("Used ");
        if (spill_bytes) *spill_bytes = number_before(" bytes spill stores");
        size_t cs = 0;
        nvrtcGetCUBINSize(prog, &cs);
        cubin.resize(cs);
        nvrtcGetCUBIN(prog, cubin.data());
        const char* low = nullptr;
        nvrtcGetLoweredName(prog, "&ivb::g_math", &low);
        tables_name = low ? low : "";
        if (tables_name.empty()) err = "NVRTC: no lowered name for the math tables";
    }
    nvrtcDestroyProgram(&prog);
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return err;
}

cudaError_t jit_load(const std::vector<char>& cubin, const std::string& tables_name, JitKernel& K) {
    cudaError_t e = cudaLibraryLoadData(&K.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return e;
    e = cudaLibraryGetKernel(&K.kern, K.lib, "ivb_jit_bound");
    if (e != cudaSuccess) return e;
    // the module's own copy of the exp / log tables, from the library's
    void* dst = nullptr;
    size_t bytes = 0;
    e = cudaLibraryGetGlobal(&dst, &bytes, K.lib, tables_name.c_str());
    if (e != cudaSuccess) return e;
    void* src = nullptr;
    size_t sbytes = 0;
    e = math_tables_address(&src, &sbytes);
    if (e != cudaSuccess) return e;
    if (bytes != sbytes) return cudaErrorInvalidValue;
    e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes a{};
    e = cudaFuncGetAttributes(&a, (const void*)K.kern);
    if (e != cudaSuccess) return e;
    K.regs = a.numRegs;
    K.local_bytes = (int)a.localSizeBytes;
    K.max_threads = a.maxThreadsPerBlock;
    return cudaSuccess;
}

static cudaKernel_t pick(const JitKernel& K, int tpsub, bool sync) {
    const int i = tpsub_index(tpsub);
    if (i < 0) return nullptr;
    if (sync) return K.kern_sync[i];
    if (i > 0) return K.kern_t[i];
    return K.kern;
}

cudaError_t jit_launch(const JitKernel& K, const KParams& P, int grid, int block, cudaStream_t s, int tpsub,
                       bool sync) {
    const cudaKernel_t k = pick(K, tpsub, sync);
    if (!k) return cudaErrorInvalidValue;
    KParams p = P;
    void* args[] = {&p};
    return cudaLaunchKernel((const void*)k, dim3(grid), dim3(block), args, 0, s);
}

int jit_occupancy(const JitKernel& K, int block, int tpsub, bool sync) {
    const cudaKernel_t k = pick(K, tpsub, sync);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

void jit_unload(JitKernel& K) {
    if (K.lib) cudaLibraryUnload(K.lib);
    K = JitKernel{};
}

}  // namespace ivb
