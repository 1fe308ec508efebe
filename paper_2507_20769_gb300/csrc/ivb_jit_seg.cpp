// ivb_jit_seg.cpp -- segmented tape-specialised bounding kernels for large tapes.
//
// The compact generator of ivb_jit.cpp writes one function per output holding
// the output's whole forward sweep and reverse (adjoint) sweep. For the deep
// tapes of the full-scale workloads (cones of ~750 interval operations per
// output) every forward value of the cone is then live until the reverse sweep
// reads it: the register allocator spills them in an order of its own and the
// compile time of such a function grows to minutes.
//
// Here the same statements -- the point sweep on [c,c], then per output the
// forward sweep on X_k, the reverse sweep of Section 3.2's derivative
// propagation (run backwards) and the Mean Value Form of Definition 5 -- are
// cut into short chunks, each a function of its own, with a bound on the
// estimated work and on the values each chunk keeps in registers:
//  * a value that crosses a chunk boundary lives in a per-thread state area
//    in global memory (element u of thread t at state[u * blockDim + t],
//    coalesced across a warp), stored right after the statement that writes
//    it and loaded where the next chunk first reads it;
//  * with a recomputation policy a reverse chunk does not read the forward
//    values of its own segment from memory: it recomputes them from the
//    segment's checkpoints (the values that enter the segment from earlier
//    statements) before running its reverse statements -- tape recomputation
//    instead of storing the whole forward sweep. Policy 1 recomputes the cheap
//    operations (+ - * sqr neg) and keeps the values of the long ones
//    (/ sqrt exp log) in the state area; policy 2 recomputes every operation
//    of the segment; policy 0 (the default: on a narrow FP64 pipe the
//    recomputed work costs more than the state traffic it saves) stores every
//    forward value the reverse sweep reads.
// Every statement calls the same interval primitive on the same operands as
// the interpreter, a recomputed value is the same function of the same
// operands, and the adjoint accumulations and the Mean Value Form sum keep
// their order, so the bounds are bit-identical to the interpreter's.
//
// The chunks are spread over several NVRTC programs compiled in parallel as
// relocatable code and linked with nvJitLink, which keeps the compile time of
// a 11 x 1000-entry problem at seconds instead of minutes.
#include <cuda_runtime.h>
#include <nvJitLink.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_internal.h"
#include "ivb_jit.h"
#include "ivb_kernels.h"

// device headers as strings (written by the build from csrc/)
#include "ivb_jit_headers.inc"

namespace ivb {

namespace {

std::string lit(double v) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%a", v);
    return std::string("(") + buf + ")";
}
std::string S(long long v) { return std::to_string(v); }

enum VarType { V_IV = 0, V_DBL = 1 };

// one statement of the straight-line per-subdomain program
struct Stmt {
    std::string code;
    std::vector<int> reads;    // variables read (before this statement writes any)
    std::vector<int> writes;   // variables written
    int out = -1;              // output whose adjoint program it belongs to (-1: point sweep)
    int phase = 0;             // 0 point sweep, 1 forward sweep, 2 reverse sweep, 3 Mean Value Form
    int fk = -1;               // forward statement of the output's cone: record written
    int rk = -1;               // reverse statement: record of the entry it differentiates
    uint32_t op = 0;           // operation of a value statement
    double cost = 0.0;         // estimated FP64 issue slots (chunk sizing only)
};

// estimated FP64 issue slots per interval operation (for chunk sizing)
double op_cost(uint32_t op) {
    switch (op) {
    case OP_ADD: case OP_SUB: case OP_MUL: case OP_SQR: return 2.0;
    case OP_DIV: return 8.0;
    case OP_SQRT: return 10.0;
    case OP_EXP: return 12.0;
    case OP_LOG: return 16.0;
    }
    return 0.0;
}
bool cheap_op(uint32_t op) { return op == OP_ADD || op == OP_SUB || op == OP_MUL || op == OP_SQR || op == OP_NEG; }

struct Builder {
    const HostProgram& P;
    const Ins* ins;
    const RIns* rins;
    const double* consts;
    int n, no, form;
    bool nie_only;
    std::vector<std::string> vname;
    std::vector<int> vtype;
    std::map<std::string, int> vid;

    int var(const std::string& nm, int type = V_IV) {
        auto it = vid.find(nm);
        if (it != vid.end()) return it->second;
        const int id = (int)vname.size();
        vname.push_back(nm);
        vtype.push_back(type);
        vid[nm] = id;
        return id;
    }

    std::string konst(uint32_t idx) const { return "mk(" + lit(consts[idx]) + ", " + lit(consts[idx]) + ")"; }

    // value operand of role 'p' (point sweep: variables read [c,c]) or 'r'
    // (forward records of an adjoint program: variables read X)
    std::string val(char role, uint32_t kind, uint32_t idx, std::vector<int>& reads) {
        if (kind == K_SLOT) {
            const std::string nm = std::string(1, role) + S(idx);
            reads.push_back(var(nm));
            return nm + "$";
        }
        if (kind == K_VAR) {
            if (role == 'p' || role == 'q') {
                reads.push_back(var("c" + S(idx), V_DBL));
                return "mk(c" + S(idx) + "$, c" + S(idx) + "$)";
            }
            reads.push_back(var("X" + S(idx)));
            return "X" + S(idx) + "$";
        }
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

    Stmt value_stmt(char role, const Ins& I) {
        Stmt s;
        const uint32_t op = I.w0 & 31u, ak = (I.w0 >> 5) & 3u, bk = (I.w0 >> 7) & 3u, dst = I.w0 >> 16;
        const std::string A = val(role, ak, I.w1 & 0xFFFFu, s.reads);
        const std::string B = bk != K_NONE ? val(role, bk, I.w1 >> 16, s.reads) : A;
        const std::string D = std::string(1, role) + S(dst);
        s.writes.push_back(var(D));
        s.code = D + "$ = " + eval(op, A, B) + ";";
        s.cost = op_cost(op);
        s.op = op;
        s.phase = role == 'r' ? 1 : 0;
        if (role == 'r') s.fk = (int)dst;
        return s;
    }

    // reverse statement of one entry (the interpreter's run_reverse, unrolled)
    Stmt reverse_stmt(const RIns& R) {
        Stmt s;
        s.phase = 2;
        const uint32_t op = R.w0 & 31u, wslot = R.w0 >> 16;
        const std::string W = "w" + S(wslot) + "$";
        s.reads.push_back(var("w" + S(wslot)));
        if (op == OP_VAR) {
            const std::string g = "g" + S(R.w1);
            s.reads.push_back(var(g));
            s.writes.push_back(var(g));
            s.code = g + "$ = iv_add(" + g + "$, " + W + ");";
            s.cost = 2.0;
            return s;
        }
        s.rk = (int)(R.w3 & 0xFFFFu);
        const bool a_init = (R.w0 >> 5) & 1u, b_init = (R.w0 >> 6) & 1u;
        const bool a_none = (R.w0 >> 7) & 1u, b_none = (R.w0 >> 8) & 1u;
        const uint32_t Ak = (R.w3 >> 16) & 3u, Bk = (R.w3 >> 18) & 3u;
        auto rv = [&](uint32_t kind, uint32_t idx) { return val('r', kind, idx, s.reads); };
        auto V = [&]() { return rv(K_SLOT, R.w3 & 0xFFFFu); };
        std::string ax = "W", ay, bx = "W", by;
        bool a_prod = true, b_prod = true, sub_a = false, sub_b = false;
        std::string body = "const auto W = " + W + "; ";
        double cost = 0.0;
        switch (op) {
        case OP_ADD: a_prod = b_prod = false; break;
        case OP_SUB: a_prod = b_prod = false; sub_b = true; break;
        case OP_NEG: a_prod = false; sub_a = true; break;
        case OP_MUL:
            if (!a_none) ay = rv(Bk, R.w2 >> 16);
            if (!b_none) by = rv(Ak, R.w2 & 0xFFFFu);
            break;
        case OP_DIV:
            body += "const auto Rb = iv_recip(" + rv(Bk, R.w2 >> 16) + "); ";
            cost += 4.0;
            ay = "Rb";
            if (!b_none) {
                body += "const auto nb = iv_neg(iv_mul(W, " + V() + ")); ";   // b gets -(W V) / B
                bx = "nb";
                cost += 2.0;
            }
            by = "Rb";
            break;
        case OP_SQR: if (!a_none) ay = "iv_twice(" + rv(Ak, R.w2 & 0xFFFFu) + ")"; break;
        case OP_SQRT: if (!a_none) { ay = "iv_recip_pos(iv_twice(" + V() + "))"; cost += 4.0; } break;
        case OP_EXP: if (!a_none) ay = V(); break;
        case OP_LOG: if (!a_none) { ay = "iv_recip_pos(" + rv(Ak, R.w2 & 0xFFFFu) + ")"; cost += 4.0; } break;
        default: a_prod = b_prod = false; ax = bx = "entire()";
        }
        if (!a_none && a_prod) body += "const auto ya = " + ay + "; ";
        if (!b_none && b_prod) body += "const auto yb = " + by + "; ";
        std::string upd;
        if (!a_none) {
            const std::string un = "w" + S(R.w1 & 0xFFFFu), u = un + "$";
            std::string v;
            if (a_prod) v = a_init ? "iv_mul(" + ax + ", ya)" : "iv_fma(" + ax + ", ya, " + u + ")";
            else if (a_init) v = sub_a ? "iv_neg(" + ax + ")" : ax;
            else v = sub_a ? "iv_sub(" + u + ", " + ax + ")" : "iv_add(" + u + ", " + ax + ")";
            if (!a_init) s.reads.push_back(var(un));
            upd += u + " = " + v + "; ";
            cost += (a_prod || !a_init) ? 2.0 : 0.0;
        }
        if (!b_none) {
            const std::string un = "w" + S(R.w1 >> 16), u = un + "$";
            std::string v;
            if (b_prod) v = b_init ? "iv_mul(" + bx + ", yb)" : "iv_fma(" + bx + ", yb, " + u + ")";
            else if (b_init) v = sub_b ? "iv_neg(" + bx + ")" : bx;
            else v = sub_b ? "iv_sub(" + u + ", " + bx + ")" : "iv_add(" + u + ", " + bx + ")";
            if (!b_init) s.reads.push_back(var(un));
            upd += u + " = " + v + "; ";
            cost += (b_prod || !b_init) ? 2.0 : 0.0;
        }
        // the factors are formed before either slot is written (operand a may be operand b)
        if (!a_none) s.writes.push_back(var("w" + S(R.w1 & 0xFFFFu)));
        if (!b_none) s.writes.push_back(var("w" + S(R.w1 >> 16)));
        s.code = "{ " + body + upd + "}";
        s.cost = cost;
        return s;
    }

    // One program per output (and, when the outputs' cones share entries, a
    // point-sweep program for all of them first). An output's program runs
    // the point sweep of its cone on [c,c] (unless shared), the forward sweep
    // on X_k, the reverse sweep and the Mean Value Form; programs read X, c
    // (and a shared point value) and leave F_o and f(c)_o in fixed slots, so
    // any grouping of outputs over threads runs the same programs.
    struct Prog {
        std::vector<Stmt> st;
        int out = -1;          // -1: the shared point sweep
        double cost = 0.0;
    };
    std::vector<Prog> progs;
    bool shared_point = false;

    Stmt copy_stmt(const std::string& dst, char role, uint32_t kind, uint32_t ref, int o, int phase) {
        Stmt s;
        s.out = o;
        s.phase = phase;
        const std::string v = val(role, kind, ref, s.reads);
        s.writes.push_back(var(dst));
        s.code = dst + "$ = " + v + ";";
        return s;
    }

    void build() {
        long long cone_sum = 0;
        for (int o = 0; o < no; ++o) cone_sum += P.adj[o].fw_count;
        // outputs whose cones overlap share one point sweep (no output groups)
        shared_point = cone_sum > P.pt_count + P.pt_count / 8 + 16;
        if (shared_point) {
            Prog pp;
            for (int i = P.pt_begin; i < P.pt_begin + P.pt_count; ++i) pp.st.push_back(value_stmt('p', ins[i]));
            for (int o = 0; o < no; ++o)
                pp.st.push_back(copy_stmt("fc" + S(o), 'p', (uint32_t)P.pt_out_kind[o], (uint32_t)P.pt_out_ref[o], -1, 0));
            progs.push_back(pp);
        }
        for (int o = 0; o < no; ++o) {
            Prog pr;
            pr.out = o;
            std::vector<Stmt>& q = pr.st;
            const AdjProgram& A = P.adj[o];
            if (!shared_point) {
                // the point sweep of this output's cone: its forward program on [c,c]
                for (int i = A.fw_begin; i < A.fw_begin + A.fw_count; ++i) {
                    Stmt t = value_stmt('q', ins[i]);
                    t.out = o;
                    t.phase = 0;
                    q.push_back(t);
                }
                q.push_back(copy_stmt("fc" + S(o), 'q', (uint32_t)A.out_kind_ref, (uint32_t)A.out_ref, o, 0));
            }
            for (int i = A.fw_begin; i < A.fw_begin + A.fw_count; ++i) {
                Stmt t = value_stmt('r', ins[i]);
                t.out = o;
                q.push_back(t);
            }
            q.push_back(copy_stmt("nie" + S(o), 'r', (uint32_t)A.out_kind_ref, (uint32_t)A.out_ref, o, 1));
            if (!nie_only) {
                Stmt t;
                t.out = o;
                t.phase = 2;
                for (int i = 0; i < n; ++i) {
                    t.writes.push_back(var("g" + S(i)));
                    t.code += "g" + S(i) + "$ = zero(); ";
                }
                if (A.out_wslot >= 0) {
                    t.writes.push_back(var("w" + S(A.out_wslot)));
                    t.code += "w" + S(A.out_wslot) + "$ = one();";
                }
                q.push_back(t);
                for (int i = A.rv_begin; i < A.rv_begin + A.rv_count; ++i) {
                    Stmt r = reverse_stmt(rins[i]);
                    r.out = o;
                    q.push_back(r);
                }
            }
            // Mean Value Form (Definition 5), left to right, and the form
            Stmt m;
            m.out = o;
            m.phase = 3;
            const std::string F = "F" + S(o);
            if (nie_only) {
                m.reads.push_back(var("nie" + S(o)));
                m.code = F + "$ = final_form(1, nie" + S(o) + "$, nie" + S(o) + "$);";
            } else {
                m.reads.push_back(var("fc" + S(o)));
                m.code = "{ auto mvf = fc" + S(o) + "$; ";
                for (int i = 0; i < n; ++i) {
                    m.reads.push_back(var("g" + S(i)));
                    m.reads.push_back(var("X" + S(i)));
                    m.reads.push_back(var("c" + S(i), V_DBL));
                    m.code += "mvf = mvf_term(mvf, g" + S(i) + "$, X" + S(i) + "$, c" + S(i) + "$); ";
                }
                m.reads.push_back(var("nie" + S(o)));
                m.code += F + "$ = final_form(" + S(form) + ", mvf, nie" + S(o) + "$); }";
                m.cost = 2.0 * n + 2.0;
            }
            m.writes.push_back(var(F));
            q.push_back(m);
            progs.push_back(pr);
        }
        for (Prog& pr : progs)
            for (const Stmt& t : pr.st) pr.cost += t.cost;
    }
};

struct Chunk {
    std::vector<Stmt> body;
};

struct Plan {
    std::vector<Chunk> chunks;                  // every program's chunks, program after program
    std::vector<std::map<int, int>> load_slot;  // per chunk: variable read before written -> slot
    std::vector<std::map<int, int>> store_slot; // per chunk: variable it hands on -> slot
    std::vector<int> prog_first, prog_count;    // chunks of each program
    int n_slots = 0;
    long long loads = 0, stores = 0, recomputed = 0;   // per subdomain (all programs)
};

// Cut the statement list into chunks of bounded estimated work and statement
// count, then insert the recomputation of each reverse chunk's own forward
// values according to the policy.
std::vector<Chunk> cut(const Builder& B, const std::vector<Stmt>& prog, double budget, int max_stmts, int policy,
                       long long* recomputed) {
    std::vector<Chunk> ch;
    Chunk cur;
    double cost = 0.0;
    for (const Stmt& s : prog) {
        if (!cur.body.empty() && (cost + s.cost > budget || (int)cur.body.size() >= max_stmts)) {
            ch.push_back(cur);
            cur = Chunk{};
            cost = 0.0;
        }
        cur.body.push_back(s);
        cost += s.cost;
    }
    if (!cur.body.empty()) ch.push_back(cur);
    *recomputed = 0;
    if (policy <= 0) return ch;
    // forward statement of each record, per output
    std::vector<std::map<int, const Stmt*>> fwd(B.no);
    for (const Stmt& s : prog)
        if (s.fk >= 0) fwd[s.out][s.fk] = &s;
    for (Chunk& c : ch) {
        std::vector<Stmt> out;
        std::set<int> written;   // variables written so far in this chunk
        size_t i = 0;
        while (i < c.body.size()) {
            if (c.body[i].phase != 2) {
                for (int w : c.body[i].writes) written.insert(w);
                out.push_back(c.body[i]);
                ++i;
                continue;
            }
            // a run of reverse statements of output o: the segment of records
            // [lo_rec, ...) it differentiates
            const int o = c.body[i].out;
            std::map<int, int> rec_of;   // variable -> record of this output
            for (auto& kv : fwd[o]) rec_of[kv.second->writes[0]] = kv.first;
            size_t j = i;
            int lo_rec = 1 << 30;
            std::set<int> need;
            while (j < c.body.size() && c.body[j].phase == 2 && c.body[j].out == o) {
                const Stmt& r = c.body[j];
                if (r.rk >= 0) lo_rec = std::min(lo_rec, r.rk);
                for (int v : r.reads) {
                    auto it = rec_of.find(v);
                    if (it != rec_of.end() && !written.count(v)) need.insert(it->second);
                }
                ++j;
            }
            // records recomputed from the segment's checkpoints: those of the
            // segment that are cheap (policy 1) or all of them (policy 2), with
            // their operands of the segment, recursively; the rest is loaded
            std::set<int> rec;
            std::vector<int> stack(need.begin(), need.end());
            while (!stack.empty()) {
                const int k = stack.back();
                stack.pop_back();
                if (rec.count(k) || k < lo_rec) continue;
                const Stmt* f = fwd[o].at(k);
                if (policy == 1 && !cheap_op(f->op)) continue;
                rec.insert(k);
                for (int v : f->reads) {
                    auto it = rec_of.find(v);
                    if (it != rec_of.end() && !written.count(v)) stack.push_back(it->second);
                }
            }
            for (int k : rec) {   // increasing record index = forward order
                Stmt f = *fwd[o].at(k);
                f.fk = -1;
                f.phase = 2;
                out.push_back(f);
                for (int w : f.writes) written.insert(w);
                *recomputed += 1;
            }
            for (size_t q = i; q < j; ++q) {
                for (int w : c.body[q].writes) written.insert(w);
                out.push_back(c.body[q]);
            }
            i = j;
        }
        c.body.swap(out);
    }
    return ch;
}

// Liveness over one program's chunks and state slots for the values that
// cross chunk boundaries. Variables with a fixed slot (X_i, c_i, f(c)_o, F_o)
// always live there; the others take working slots from `w0` on, released
// one chunk after their last read (inside a chunk a live-in may be loaded
// after another variable's store).
std::string plan_prog(const Builder& B, const std::vector<Chunk>& ch, const std::map<int, int>& fixed,
                      const std::set<int>& ends, int w0, Plan& pl) {
    const int C = (int)ch.size();
    std::vector<std::set<int>> use(C), def(C), live_out(C);
    for (int c = 0; c < C; ++c)
        for (const Stmt& t : ch[c].body) {
            for (int v : t.reads) if (!def[c].count(v)) use[c].insert(v);
            for (int v : t.writes) def[c].insert(v);
        }
    std::set<int> live = ends;
    for (int c = C - 1; c >= 0; --c) {
        live_out[c] = live;
        std::set<int> in = use[c];
        for (int v : live) if (!def[c].count(v)) in.insert(v);
        live = in;
    }
    for (int v : live)
        if (!fixed.count(v)) return "internal: " + B.vname[v] + " is read before any statement writes it";
    std::vector<int> free_slots, released;
    int next = w0;
    auto get = [&]() { if (!free_slots.empty()) { int q = free_slots.back(); free_slots.pop_back(); return q; } return next++; };
    std::map<int, int> cur;   // working variable -> slot, live at the current boundary
    for (int c = 0; c < C; ++c) {
        free_slots.insert(free_slots.end(), released.begin(), released.end());
        released.clear();
        std::map<int, int> ld, stv;
        for (int v : use[c]) {
            auto f = fixed.find(v);
            ld[v] = f != fixed.end() ? f->second : cur.at(v);
        }
        std::map<int, int> nxt;
        for (auto& kv : cur) {
            if (live_out[c].count(kv.first)) nxt[kv.first] = kv.second;
            else released.push_back(kv.second);
        }
        for (int v : live_out[c]) {
            if (!def[c].count(v)) continue;
            auto f = fixed.find(v);
            if (f != fixed.end()) { stv[v] = f->second; continue; }
            if (!nxt.count(v)) nxt[v] = get();
            stv[v] = nxt[v];
        }
        pl.loads += (long long)ld.size();
        pl.stores += (long long)stv.size();
        pl.load_slot.push_back(ld);
        pl.store_slot.push_back(stv);
        cur = nxt;
    }
    if (next > pl.n_slots) pl.n_slots = next;
    return "";
}

// out-of-line copies of the short interval operations (option seg_outline):
// a statement then compiles to a call instead of the operation's selects and
// directed multiplies, which shrinks the code every warp streams through
const char* kOutline =
    "namespace ivb {\n"
    "static __device__ __noinline__ iv o_add(iv a, iv b) { return iv_add(a, b); }\n"
    "static __device__ __noinline__ iv o_sub(iv a, iv b) { return iv_sub(a, b); }\n"
    "static __device__ __noinline__ iv o_mul(iv a, iv b) { return iv_mul(a, b); }\n"
    "static __device__ __noinline__ iv o_sqr(iv a) { return iv_sqr(a); }\n"
    "static __device__ __noinline__ iv o_fma(iv a, iv b, iv c) { return iv_fma(a, b, c); }\n"
    "}\n";

// the statement's code with the short operations called out of line: all of
// them (level 1) or the products only (level 2: x sqr and the fused
// accumulation; + and - stay inline)
std::string outline_code(const std::string& code, int level = 1) {
    std::string r = code;
    for (const char* f : {"iv_add(", "iv_sub(", "iv_mul(", "iv_sqr(", "iv_fma("}) {
        const bool sum = f[3] == 'a' || (f[3] == 's' && f[4] == 'u');   // iv_add, iv_sub
        if (level == 2 && sum) continue;
        const std::string from = f, to = std::string("o_") + (f + 3);
        size_t at = 0;
        while ((at = r.find(from, at)) != std::string::npos) {
            r.replace(at, from.size(), to);
            at += to.size();
        }
    }
    return r;
}

// a statement's code for copy k of K (variable names end in '$')
std::string copy_code(const std::string& code, int K, int k) {
    const std::string sfx = K > 1 ? "_" + S(k) : "";
    std::string r;
    r.reserve(code.size() + 16);
    for (char ch : code) {
        if (ch == '$') r += sfx;
        else r += ch;
    }
    return r;
}

// Paired form of two subdomains per thread, the dual-pipe arrangement
// (seg_ilp = 2 with the short operations out of line and an emulation
// policy): every value is a pair (iv2, d2) of the two subdomains' values, and
// every interval operation of a statement is one call that computes both
// copies. The short operations and the long ones (/ sqrt exp log and the
// reciprocals) are out-of-line functions whose bodies hold the two copies
// inlined side by side, so the compiler interleaves their independent
// dependency chains; copy a's endpoint operations run on the FP64 pipe and
// copy b's short ones under the emulation policy IVB_EMU_B on the integer
// pipes (bit-identical to the FP64 instructions). Constants stay scalar
// intervals and convert to pairs of equal copies where they meet a pair.
// Without an emulation policy the two copies' calls alternate instead (the
// interleaved form of chunk_fn), which measured faster.
const char* kPair =
    "namespace ivb {\n"
    "struct iv2 {\n"
    "  iv a, b;\n"
    "  __device__ __forceinline__ iv2() {}\n"
    "  __device__ __forceinline__ iv2(const iv& x) : a(x), b(x) {}\n"
    "  __device__ __forceinline__ iv2(const iv& x, const iv& y) : a(x), b(y) {}\n"
    "};\n"
    "struct d2 { double a, b; };\n"
    "__device__ __forceinline__ iv2 mk(d2 x, d2 y) { return iv2(mk(x.a, y.a), mk(x.b, y.b)); }\n"
    "__device__ __forceinline__ iv2 ld2(const double* st, int ss, int slot, int ns) {\n"
    "  return iv2(st_ld(st, ss, slot), st_ld(st, ss, slot + ns)); }\n"
    "__device__ __forceinline__ d2 ldd2(const double* st, int ss, int slot, int ns) {\n"
    "  d2 r; r.a = st_d(st, ss, slot); r.b = st_d(st, ss, slot + ns); return r; }\n"
    "__device__ __forceinline__ void st2(double* st, int ss, int slot, int ns, const iv2& v) {\n"
    "  st_st(st, ss, slot, v.a); st_st(st, ss, slot + ns, v.b); }\n"
    "__device__ __forceinline__ void std2(double* st, int ss, int slot, int ns, const d2& v) {\n"
    "  st_sd(st, ss, slot, v.a); st_sd(st, ss, slot + ns, v.b); }\n"
    "static __device__ __noinline__ iv2 o_add(iv2 x, iv2 y) {\n"
    "  return iv2(iv_add_t<0>(x.a, y.a), iv_add_t<IVB_EMU_B>(x.b, y.b)); }\n"
    "static __device__ __noinline__ iv2 o_sub(iv2 x, iv2 y) {\n"
    "  return iv2(iv_sub_t<0>(x.a, y.a), iv_sub_t<IVB_EMU_B>(x.b, y.b)); }\n"
    "static __device__ __noinline__ iv2 o_mul(iv2 x, iv2 y) {\n"
    "  return iv2(iv_mul_t<0>(x.a, y.a), iv_mul_t<IVB_EMU_B>(x.b, y.b)); }\n"
    "static __device__ __noinline__ iv2 o_sqr(iv2 x) { return iv2(iv_sqr_t<0>(x.a), iv_sqr_t<IVB_EMU_B>(x.b)); }\n"
    "static __device__ __noinline__ iv2 o_fma(iv2 x, iv2 y, iv2 z) {\n"
    "  return iv2(iv_fma(x.a, y.a, z.a), iv_fma(x.b, y.b, z.b)); }\n"
    "static __device__ __noinline__ iv2 iv_div(iv2 x, iv2 y) { return iv2(iv_div(x.a, y.a), iv_div(x.b, y.b)); }\n"
    "static __device__ __noinline__ iv2 iv_sqrt(iv2 x) { return iv2(iv_sqrt(x.a), iv_sqrt(x.b)); }\n"
    "static __device__ __noinline__ iv2 iv_exp(iv2 x) { return iv2(iv_exp(x.a), iv_exp(x.b)); }\n"
    "static __device__ __noinline__ iv2 iv_log(iv2 x) { return iv2(iv_log(x.a), iv_log(x.b)); }\n"
    "static __device__ __noinline__ iv2 iv_recip(iv2 x) { return iv2(iv_recip(x.a), iv_recip(x.b)); }\n"
    "static __device__ __noinline__ iv2 iv_recip_pos(iv2 x) { return iv2(iv_recip_pos(x.a), iv_recip_pos(x.b)); }\n"
    "__device__ __forceinline__ iv2 iv_neg(iv2 x) { return iv2(iv_neg(x.a), iv_neg(x.b)); }\n"
    "__device__ __forceinline__ iv2 iv_twice(iv2 x) { return iv2(iv_twice(x.a), iv_twice(x.b)); }\n"
    "__device__ __forceinline__ iv2 mvf_term(iv2 acc, iv2 g, iv2 x, d2 c) {\n"
    "  return iv2(mvf_term(acc.a, g.a, x.a, c.a), mvf_term(acc.b, g.b, x.b, c.b)); }\n"
    "__device__ __forceinline__ iv2 final_form(int f, iv2 m, iv2 v) {\n"
    "  return iv2(final_form(f, m.a, v.a), final_form(f, m.b, v.b)); }\n"
    "}\n";

// C++ of one chunk function in the paired form (see kPair)
std::string chunk_fn_pair(const Builder& B, const Plan& pl, int c, int ns) {
    const Chunk& ch = pl.chunks[c];
    const std::map<int, int>& ld = pl.load_slot[c];
    const std::map<int, int>& stv = pl.store_slot[c];
    const std::string NS = S(ns);
    std::string s = "extern \"C\" __device__ __noinline__ void ivb_ck" + S(c) +
                    "(double* __restrict__ st, const int ss) {\n  using namespace ivb;\n";
    std::set<int> touched;
    for (const Stmt& t : ch.body) {
        for (int v : t.reads) touched.insert(v);
        for (int v : t.writes) touched.insert(v);
    }
    {
        std::string dv, dd;
        for (int v : touched) {
            if (B.vtype[v] == V_DBL) dd += (dd.empty() ? "  d2 " : ", ") + B.vname[v];
            else dv += (dv.empty() ? "  iv2 " : ", ") + B.vname[v];
        }
        if (!dv.empty()) s += dv + ";\n";
        if (!dd.empty()) s += dd + ";\n";
    }
    std::map<int, size_t> last_write;
    for (size_t i = 0; i < ch.body.size(); ++i)
        for (int v : ch.body[i].writes) last_write[v] = i;
    std::set<int> loaded, written;
    for (size_t i = 0; i < ch.body.size(); ++i) {
        const Stmt& t = ch.body[i];
        for (int v : t.reads)
            if (!written.count(v) && !loaded.count(v)) {
                s += "  " + B.vname[v] + (B.vtype[v] == V_DBL ? " = ldd2(st, ss, " : " = ld2(st, ss, ") +
                     S(ld.at(v)) + ", " + NS + ");\n";
                loaded.insert(v);
            }
        s += "  " + copy_code(outline_code(t.code), 1, 0) + "\n";
        for (int v : t.writes) written.insert(v);
        for (int v : t.writes) {
            auto it = stv.find(v);
            if (last_write[v] == i && it != stv.end())
                s += std::string(B.vtype[v] == V_DBL ? "  std2(st, ss, " : "  st2(st, ss, ") + S(it->second) + ", " +
                     NS + ", " + B.vname[v] + ");\n";
        }
    }
    s += "}\n";
    return s;
}

// C++ of one chunk function. With K = 2 every statement runs twice, on two
// subdomains, interleaved: two independent dependency chains per thread.
// Copy k keeps its values in state slots offset by k * ns.
std::string chunk_fn(const Builder& B, const Plan& pl, int c, int K, int ns, int outline) {
    const Chunk& ch = pl.chunks[c];
    const std::map<int, int>& ld = pl.load_slot[c];
    const std::map<int, int>& stv = pl.store_slot[c];
    std::string s = "extern \"C\" __device__ __noinline__ void ivb_ck" + S(c) +
                    "(double* __restrict__ st, const int ss) {\n  using namespace ivb;\n";
    std::set<int> touched;
    for (const Stmt& t : ch.body) {
        for (int v : t.reads) touched.insert(v);
        for (int v : t.writes) touched.insert(v);
    }
    auto nm = [&](int v, int k) { return B.vname[v] + (K > 1 ? "_" + S(k) : ""); };
    {
        std::string dv, dd;
        for (int v : touched)
            for (int k = 0; k < K; ++k) {
                if (B.vtype[v] == V_DBL) dd += (dd.empty() ? "  double " : ", ") + nm(v, k);
                else dv += (dv.empty() ? "  iv " : ", ") + nm(v, k);
            }
        if (!dv.empty()) s += dv + ";\n";
        if (!dd.empty()) s += dd + ";\n";
    }
    std::map<int, size_t> last_write;
    for (size_t i = 0; i < ch.body.size(); ++i)
        for (int v : ch.body[i].writes) last_write[v] = i;
    std::set<int> loaded, written;
    for (size_t i = 0; i < ch.body.size(); ++i) {
        const Stmt& t = ch.body[i];
        // live-ins are loaded before their first read (the scheduler hoists them)
        for (int v : t.reads)
            if (!written.count(v) && !loaded.count(v)) {
                for (int k = 0; k < K; ++k) {
                    const int slot = ld.at(v) + k * ns;
                    s += "  " + nm(v, k) + (B.vtype[v] == V_DBL ? " = st_d(st, ss, " : " = st_ld(st, ss, ") + S(slot) +
                         ");\n";
                }
                loaded.insert(v);
            }
        for (int k = 0; k < K; ++k) s += "  " + copy_code(outline ? outline_code(t.code, outline) : t.code, K, k) + "\n";
        for (int v : t.writes) written.insert(v);
        for (int v : t.writes) {
            auto it = stv.find(v);
            if (last_write[v] == i && it != stv.end())
                for (int k = 0; k < K; ++k)
                    s += std::string(B.vtype[v] == V_DBL ? "  st_sd(st, ss, " : "  st_st(st, ss, ") +
                         S(it->second + k * ns) + ", " + nm(v, k) + ");\n";
        }
    }
    s += "}\n";
    return s;
}

const char* kPrelude =
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n";

const char* kStateHelpers =
    "namespace ivb {\n"
    "__device__ __forceinline__ iv st_ld(const double* st, int ss, int slot) {\n"
    "  return mk(st[(size_t)(2 * slot) * ss], st[(size_t)(2 * slot + 1) * ss]); }\n"
    "__device__ __forceinline__ double st_d(const double* st, int ss, int slot) { return st[(size_t)(2 * slot) * ss]; }\n"
    "__device__ __forceinline__ void st_st(double* st, int ss, int slot, iv v) {\n"
    "  st[(size_t)(2 * slot) * ss] = v.lo; st[(size_t)(2 * slot + 1) * ss] = v.hi; }\n"
    "__device__ __forceinline__ void st_sd(double* st, int ss, int slot, double v) { st[(size_t)(2 * slot) * ss] = v; }\n"
    "}\n";

std::string unit_head(int emulate, bool kernel_unit, bool paired = false) {
    // paired units: copy a on the FP64 instructions, copy b under the policy;
    // the long primitives inline into the out-of-line pair functions
    std::string s = paired ? "#define IVB_EMU 0\n#define IVB_EMU_B " + S(emulate) + "\n#define IVB_HEAVY __forceinline__\n"
                           : "#define IVB_EMU " + S(emulate) + "\n#define IVB_HEAVY static __noinline__\n";
    if (!kernel_unit) s += "#define IVB_JIT_EXTERN_TABLES\n";
    s += kPrelude;
    s += "#include \"ivb_bound_common.cuh\"\n";
    s += kStateHelpers;
    return s;
}

// fixed state slots: X_i at i, c_i at n + i, F_o at 2n + 2o, f(c)_o at 2n + 2o + 1
int slot_X(int n, int i) { return i; }
int slot_c(int n, int i) { return n + i; }
int slot_F(int n, int o) { return 2 * n + 2 * o; }
int slot_fc(int n, int o) { return 2 * n + 2 * o + 1; }

// One kernel per number T of threads sharing a subdomain: a block's threads
// form T groups of blockDim/T (whole warps); group g runs the programs of its
// outputs on the same blockDim/T subdomains as the other groups. The tests
// that need every output of a subdomain (a constraint proving it infeasible
// for the filtered objective; the certified-feasible centre of the upper
// bound) are combined through shared memory by the objective's group; each
// group reduces its own outputs' hulls. T = 1 is the plain kernel.
std::string kernel_fn(const Builder& B, const Plan& pl, const std::vector<std::vector<int>>& groups, int T,
                      bool sync, int K, int ns, const std::string& name, int block_max, int min_blocks) {
    const int n = B.n, no = B.no, obj = B.P.obj;
    int gobj = 0;
    for (int g = 0; g < T; ++g)
        for (int o : groups[g]) if (o == obj) gobj = g;
    auto sub = [&](int k) { return "s" + S(k); };
    std::string s = "extern \"C\" __global__ void __launch_bounds__(" + S(block_max) + ", " + S(min_blocks) + ") " +
                    name + "(const ivb::KParams P) {\n";
    s += "  using namespace ivb;\n";
    s += "  double* const st = P.gframe + (size_t)blockIdx.x * P.frame_units * blockDim.x + threadIdx.x;\n";
    s += "  const int ss = blockDim.x;\n";
    s += "  const int per = blockDim.x / " + S(T) + ";\n";
    s += "  const int grp = threadIdx.x / per;\n";
    if (T > 1) s += "  __shared__ unsigned char s_fl[" + S(K) + "][" + S(block_max) + "];\n";
    if (K == 1) s += "  tile_loop_per(P, per, [&](const Sub& s0) {\n";
    else s += "  tile_loop_per2(P, per, [&](const Sub& s0, const Sub& s1) {\n";
    for (int k = 0; k < K; ++k) {
        std::string f = "    iv ";
        for (int o = 0; o < no; ++o) f += (o ? ", F" : "F") + S(o) + "_" + S(k) + " = zero()";
        s += f + ";\n";
        s += "    unsigned int fl_" + S(k) + " = 0u;\n";
        s += "    double obj_lo_" + S(k) + " = from_bits(0x7FF0000000000000LL), fco_" + S(k) +
             " = from_bits(0x7FF0000000000000LL);\n";
    }
    s += "    // fl bit 1: an output proves the subdomain infeasible; bit 2: its centre is not certified feasible\n";
    s += "    if (s0.valid) {\n";
    for (int k = 0; k < K; ++k) {
        // a second copy without a subdomain of its own repeats the first (its results are not reduced)
        const std::string sk = k == 0 ? "s0" : "(s1.valid ? s1 : s0)";
        s += "      { const Sub& d = " + sk + "; unsigned int kk = d.k;\n";
        for (int i = 0; i < n; ++i)
            s += "        { iv X; double c; decode_dim(d.rec, " + S(n) + ", " + S(i) + ", kk, X, c); st_st(st, ss, " +
                 S(slot_X(n, i) + k * ns) + ", X); st_sd(st, ss, " + S(slot_c(n, i) + k * ns) + ", c); }\n";
        s += "      }\n";
    }
    // with `sync`, the threads of a group wait for each other after every
    // chunk (named barrier 1 + group of blockDim / T threads), so the warps of a
    // group run the same chunk's code together and share the instruction
    // cache; a lane without a subdomain skips the chunk but not the barrier
    auto calls = [&](int prog, int g, const std::string& ind) {
        std::string r;
        for (int c = pl.prog_first[prog]; c < pl.prog_first[prog] + pl.prog_count[prog]; ++c) {
            if (sync)
                r += ind + "if (s0.valid) ivb_ck" + S(c) + "(st, ss);\n" + ind + "asm volatile(\"bar.sync " + S(1 + g) +
                     ", %0;\" :: \"r\"(per) : \"memory\");\n";
            else r += ind + "ivb_ck" + S(c) + "(st, ss);\n";
        }
        return r;
    };
    const int p0 = B.shared_point ? 1 : 0;   // program index of output 0
    if (sync) s += "    }\n";                  // the calls run outside the valid branch
    const std::string ind = sync ? "    " : "      ";
    if (B.shared_point) s += calls(0, 0, ind);
    for (int g = 0; g < T; ++g) {
        s += ind + (g ? "else if" : "if") + " (grp == " + S(g) + ") {\n";
        for (int o : groups[g]) {
            s += calls(p0 + o, g, ind + "  ");
            s += ind + "  " + (sync ? "if (s0.valid) " : "") + "{\n";
            for (int k = 0; k < K; ++k) {
                const std::string Fk = "F" + S(o) + "_" + S(k), fl = "fl_" + S(k);
                s += ind + "    " + Fk + " = st_ld(st, ss, " + S(slot_F(n, o) + k * ns) + ");\n";
                s += ind + "    if (excludes_feasible(" + S(B.P.out_kind[o]) + "u, " + Fk + ")) " + fl + " |= 1u;\n";
                if (B.P.out_kind[o] == OUT_INEQ)
                    s += ind + "    if (!le0(st_ld(st, ss, " + S(slot_fc(n, o) + k * ns) + ").hi)) " + fl + " |= 2u;\n";
                if (o == obj) {
                    s += ind + "    obj_lo_" + S(k) + " = " + Fk + ".lo;\n";
                    s += ind + "    fco_" + S(k) + " = st_ld(st, ss, " + S(slot_fc(n, o) + k * ns) + ").hi;\n";
                }
            }
            s += ind + "  }\n";
        }
        s += ind + "}\n";
    }
    if (!sync) s += "    }\n";
    if (T > 1) {
        for (int k = 0; k < K; ++k) s += "    s_fl[" + S(k) + "][threadIdx.x] = (unsigned char)fl_" + S(k) + ";\n";
        s += "    __syncthreads();\n";
        s += "    if (grp == " + S(gobj) + ") for (int h = 0; h < " + S(T) + "; ++h) {\n";
        for (int k = 0; k < K; ++k) s += "      fl_" + S(k) + " |= s_fl[" + S(k) + "][h * per + threadIdx.x % per];\n";
        s += "    }\n    __syncthreads();\n";
    }
    for (int k = 0; k < K; ++k) {
        const std::string kk = S(k);
        s += "    double ub_" + kk + " = from_bits(0x7FF0000000000000LL);\n";
        s += "    if (" + sub(k) + ".valid && grp == " + S(gobj) + ") {\n";
        s += std::string("      if (") + (B.P.has_eq ? "false" : "!(fl_" + kk + " & 2u)") + ") ub_" + kk + " = fco_" + kk +
             ";\n";
        s += "      if (fl_" + kk + " & 1u) obj_lo_" + kk + " = from_bits(0x7FF0000000000000LL);\n";
        s += "    }\n";
    }
    for (int g = 0; g < T; ++g) {
        s += std::string("    ") + (g ? "else if" : "if") + " (grp == " + S(g) + ") {\n";
        for (int k = 0; k < K; ++k) {
            for (int o : groups[g])
                s += "      reduce_output(P, " + sub(k) + ", " + S(no) + ", " + S(o) + ", F" + S(o) + "_" + S(k) + ");\n";
            if (g == gobj)
                s += "      reduce_extras(P, " + sub(k) + ", " + S(no) + ", ub_" + S(k) + ", obj_lo_" + S(k) + ");\n";
        }
        s += "    }\n";
    }
    s += "  });\n}\n";
    return s;
}

// output groups for T threads per subdomain: largest estimated work first to
// the least loaded group, each group's outputs in index order
std::vector<std::vector<int>> group_outputs(const Builder& B, int T) {
    const int p0 = B.shared_point ? 1 : 0;
    std::vector<int> order(B.no);
    for (int o = 0; o < B.no; ++o) order[o] = o;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return B.progs[p0 + a].cost > B.progs[p0 + b].cost; });
    std::vector<std::vector<int>> g(T);
    std::vector<double> load(T, 0.0);
    for (int o : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        g[k].push_back(o);
        load[k] += B.progs[p0 + o].cost;
    }
    for (auto& v : g) std::sort(v.begin(), v.end());
    return g;
}

// every "Used N registers" (max) and "N bytes spill stores" (sum) in a ptxas log
void ptxas_stats(const std::string& log, int* regs, int* spill) {
    size_t at = 0;
    while ((at = log.find("Used ", at)) != std::string::npos) {
        at += 5;
        const int r = std::atoi(log.c_str() + at);
        if (r > *regs) *regs = r;
    }
    at = 0;
    while ((at = log.find(" bytes spill stores", at)) != std::string::npos) {
        size_t b = at;
        while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
        *spill += std::atoi(log.substr(b, at - b).c_str());
        at += 5;
    }
}

struct UnitResult {
    std::vector<char> cubin;
    std::string err, tables;
    int regs = 0, spill = 0;
};

void compile_unit(const std::string& src, bool kernel, int max_regs, UnitResult& R) {
    nvrtcProgram prog;
    const int nh = (int)(sizeof(kJitHeaderNames) / sizeof(kJitHeaderNames[0]));
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), kernel ? "ivb_seg_kernel.cu" : "ivb_seg_unit.cu", nh,
                                       kJitHeaderSources, kJitHeaderNames);
    if (r != NVRTC_SUCCESS) { R.err = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r); return; }
    if (kernel) nvrtcAddNameExpression(prog, "&ivb::g_math");
    const std::string mr = "-maxrregcount=" + S(max_regs);
    const char* opts[] = {"-arch=sm_103a", "--fmad=false", "-std=c++17", "-rdc=true", "-lineinfo",
                          "--ptxas-options=-v", mr.c_str()};
    r = nvrtcCompileProgram(prog, 7, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS) {
        R.err = std::string("NVRTC compilation of a segmented kernel unit failed: ") + nvrtcGetErrorString(r) + "\n" +
                log.substr(0, 4000);
    } else {
        ptxas_stats(log, &R.regs, &R.spill);
        size_t cs = 0;
        nvrtcGetCUBINSize(prog, &cs);
        R.cubin.resize(cs);
        nvrtcGetCUBIN(prog, R.cubin.data());
        if (kernel) {
            const char* low = nullptr;
            nvrtcGetLoweredName(prog, "&ivb::g_math", &low);
            R.tables = low ? low : "";
            if (R.tables.empty()) R.err = "NVRTC: no lowered name for the math tables";
        }
    }
    nvrtcDestroyProgram(&prog);
}

}  // namespace

SegSource jit_seg_source(const HostProgram& P, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                         const std::vector<double>& consts, int block_max, int min_blocks, int emulate, int form,
                         const SegPolicy& pol) {
    Builder B{P, ins.data(), rins.data(), consts.data(), P.n_vars, P.n_out, form, form == 1};
    const int n = B.n, no = B.no;
    std::map<int, int> fixed;
    for (int i = 0; i < n; ++i) {
        fixed[B.var("X" + S(i))] = slot_X(n, i);
        fixed[B.var("c" + S(i), V_DBL)] = slot_c(n, i);
    }
    for (int o = 0; o < no; ++o) {
        fixed[B.var("F" + S(o))] = slot_F(n, o);
        fixed[B.var("fc" + S(o))] = slot_fc(n, o);
    }
    B.build();
    Plan pl;
    pl.n_slots = 2 * n + 2 * no;
    SegSource out;
    for (const Builder::Prog& pr : B.progs) {
        long long rec = 0;
        const int copies = pol.ilp == 2 ? 2 : 1;
        std::vector<Chunk> ch = cut(B, pr.st, pol.chunk_cost / copies, pol.chunk_stmts / copies,
                                    B.nie_only ? 0 : pol.recompute, &rec);
        std::set<int> ends;
        if (pr.out < 0) {
            for (int o = 0; o < no; ++o) ends.insert(B.vid.at("fc" + S(o)));
        } else {
            ends.insert(B.vid.at("F" + S(pr.out)));
            if (!B.shared_point) ends.insert(B.vid.at("fc" + S(pr.out)));
        }
        pl.prog_first.push_back((int)pl.chunks.size());
        pl.prog_count.push_back((int)ch.size());
        const std::string e = plan_prog(B, ch, fixed, ends, 2 * n + 2 * no, pl);
        if (!e.empty()) { out.error = e; return out; }
        pl.chunks.insert(pl.chunks.end(), ch.begin(), ch.end());
        pl.recomputed += rec;
    }
    const int K = pol.ilp == 2 ? 2 : 1;
    const int ns = std::max(pl.n_slots, 1);
    out.state_units = 2 * ns * K;
    out.ilp = K;
    out.chunks = (int)pl.chunks.size();
    out.loads = pl.loads;
    out.stores = pl.stores;
    out.recomputed = pl.recomputed;
    // kernels: T = 1, and T = 2, 4 threads per subdomain when the outputs have
    // programs of their own and there are at least T of them
    std::string k = unit_head(emulate, true);
    for (size_t c = 0; c < pl.chunks.size(); ++c)
        k += "extern \"C\" __device__ void ivb_ck" + S(c) + "(double* __restrict__ st, const int ss);\n";
    for (int T : {1, 2, 4}) {
        if (T > 1 && (B.shared_point || no < T || block_max < 32 * T)) continue;
        out.ts.push_back(T);
        const std::vector<std::vector<int>> groups = group_outputs(B, T);
        k += kernel_fn(B, pl, groups, T, false, K, ns, T == 1 ? "ivb_jit_bound" : "ivb_jit_bound_t" + S(T),
                       block_max, min_blocks);
        k += kernel_fn(B, pl, groups, T, true, K, ns, "ivb_jit_bound_t" + S(T) + "_sync", block_max, min_blocks);
    }
    out.kernel = k;
    // chunks spread over units of similar size, compiled in parallel
    const int C = (int)pl.chunks.size();
    const int U = std::max(1, std::min(C, pol.units));
    for (int u = 0; u < U; ++u) {
        const bool paired = K == 2 && pol.outline && emulate != 0;
        std::string src = unit_head(emulate, false, paired);
        if (pol.outline) src += kOutline;
        if (paired) src += kPair;
        const int b = (int)((long long)C * u / U), e = (int)((long long)C * (u + 1) / U);
        for (int c = b; c < e; ++c)
            src += paired ? chunk_fn_pair(B, pl, c, ns) : chunk_fn(B, pl, c, K, ns, pol.outline);
        out.units.push_back(src);
    }
    return out;
}

std::string jit_seg_compile(const SegSource& src, int max_regs, std::vector<char>& cubin, std::string& tables_name,
                            double* seconds, int* registers, int* spill_bytes) {
    if (!src.error.empty()) return src.error;
    const auto t0 = std::chrono::steady_clock::now();
    const int U = (int)src.units.size();
    std::vector<UnitResult> res(U + 1);
    std::atomic<int> next{0};
    auto work = [&]() {
        for (;;) {
            const int k = next.fetch_add(1);
            if (k > U) return;
            if (k == 0) compile_unit(src.kernel, true, max_regs, res[0]);
            else compile_unit(src.units[k - 1], false, max_regs, res[k]);
        }
    };
    int nt = (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt > 0 ? nt : 4, U + 1));
    std::vector<std::thread> pool;
    for (int i = 1; i < nt; ++i) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    std::string err;
    int regs = 0, spill = 0;
    for (const UnitResult& r : res) {
        if (err.empty() && !r.err.empty()) err = r.err;
        regs = std::max(regs, r.regs);
        spill += r.spill;
    }
    if (err.empty()) {
        tables_name = res[0].tables;
        nvJitLinkHandle h;
        const char* lopts[] = {"-arch=sm_103a"};
        nvJitLinkResult lr = nvJitLinkCreate(&h, 1, lopts);
        if (lr != NVJITLINK_SUCCESS) {
            err = "nvJitLinkCreate failed (" + S((int)lr) + ")";
        } else {
            for (int k = 0; k <= U && lr == NVJITLINK_SUCCESS; ++k) {
                const std::string nm = "unit" + S(k);
                lr = nvJitLinkAddData(h, NVJITLINK_INPUT_CUBIN, res[k].cubin.data(), res[k].cubin.size(), nm.c_str());
            }
            if (lr == NVJITLINK_SUCCESS) lr = nvJitLinkComplete(h);
            if (lr != NVJITLINK_SUCCESS) {
                size_t ls = 0;
                nvJitLinkGetErrorLogSize(h, &ls);
                std::string log(ls, '\0');
                if (ls) nvJitLinkGetErrorLog(h, &log[0]);
                err = "nvJitLink failed (" + S((int)lr) + "): " + log.substr(0, 2000);
            } else {
                size_t cs = 0;
                nvJitLinkGetLinkedCubinSize(h, &cs);
                cubin.resize(cs);
                nvJitLinkGetLinkedCubin(h, cubin.data());
            }
            nvJitLinkDestroy(&h);
        }
    }
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (registers) *registers = regs;
    if (spill_bytes) *spill_bytes = spill;
    return err;
}

}  // namespace ivb
