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
//  * a reverse chunk does not read the forward values of its own segment from
//    memory: it recomputes them from the segment's checkpoints (the values
//    that enter the segment from earlier statements) before running its
//    reverse statements -- tape recomputation instead of storing the whole
//    forward sweep. Policy 1 recomputes the cheap operations (+ - * sqr neg)
//    and keeps the values of the long ones (/ sqrt exp log) in the state area;
//    policy 2 recomputes every operation of the segment; policy 0 stores every
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
#include <mutex>
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
    std::vector<Stmt> st;

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
            return nm;
        }
        if (kind == K_VAR) {
            if (role == 'p') {
                reads.push_back(var("c" + S(idx), V_DBL));
                return "mk(c" + S(idx) + ", c" + S(idx) + ")";
            }
            reads.push_back(var("X" + S(idx)));
            return "X" + S(idx);
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
        s.code = D + " = " + eval(op, A, B) + ";";
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
        const std::string W = "w" + S(wslot);
        s.reads.push_back(var(W));
        if (op == OP_VAR) {
            const std::string g = "g" + S(R.w1);
            s.reads.push_back(var(g));
            s.writes.push_back(var(g));
            s.code = g + " = iv_add(" + g + ", " + W + ");";
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
        std::string body = "const iv W = " + W + "; ";
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
            body += "const iv Rb = iv_recip(" + rv(Bk, R.w2 >> 16) + "); ";
            cost += 4.0;
            ay = "Rb";
            if (!b_none) {
                body += "const iv nb = iv_neg(iv_mul(W, " + V() + ")); ";   // b gets -(W V) / B
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
        if (!a_none && a_prod) body += "const iv ya = " + ay + "; ";
        if (!b_none && b_prod) body += "const iv yb = " + by + "; ";
        std::string upd;
        if (!a_none) {
            const std::string u = "w" + S(R.w1 & 0xFFFFu);
            std::string v;
            if (a_prod) v = a_init ? "iv_mul(" + ax + ", ya)" : "iv_fma(" + ax + ", ya, " + u + ")";
            else if (a_init) v = sub_a ? "iv_neg(" + ax + ")" : ax;
            else v = sub_a ? "iv_sub(" + u + ", " + ax + ")" : "iv_add(" + u + ", " + ax + ")";
            if (!a_init) s.reads.push_back(var(u));
            upd += u + " = " + v + "; ";
            cost += (a_prod || !a_init) ? 2.0 : 0.0;
        }
        if (!b_none) {
            const std::string u = "w" + S(R.w1 >> 16);
            std::string v;
            if (b_prod) v = b_init ? "iv_mul(" + bx + ", yb)" : "iv_fma(" + bx + ", yb, " + u + ")";
            else if (b_init) v = sub_b ? "iv_neg(" + bx + ")" : bx;
            else v = sub_b ? "iv_sub(" + u + ", " + bx + ")" : "iv_add(" + u + ", " + bx + ")";
            if (!b_init) s.reads.push_back(var(u));
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

    // the whole per-subdomain program, in the order the compact kernel runs it
    void build() {
        // point sweep on [c,c] over every output's cone
        for (int i = P.pt_begin; i < P.pt_begin + P.pt_count; ++i) st.push_back(value_stmt('p', ins[i]));
        for (int o = 0; o < no; ++o) {
            Stmt s;
            const std::string ref = val('p', (uint32_t)P.pt_out_kind[o], (uint32_t)P.pt_out_ref[o], s.reads);
            s.writes.push_back(var("fc" + S(o)));
            s.code = "fc" + S(o) + " = " + ref + ";";
            st.push_back(s);
        }
        for (int o = 0; o < no; ++o) {
            const AdjProgram& A = P.adj[o];
            for (int i = A.fw_begin; i < A.fw_begin + A.fw_count; ++i) {
                Stmt s = value_stmt('r', ins[i]);
                s.out = o;
                st.push_back(s);
            }
            {
                Stmt s;
                s.out = o;
                s.phase = 1;
                const std::string ref = val('r', (uint32_t)A.out_kind_ref, (uint32_t)A.out_ref, s.reads);
                s.writes.push_back(var("nie" + S(o)));
                s.code = "nie" + S(o) + " = " + ref + ";";
                st.push_back(s);
            }
            if (!nie_only) {
                Stmt s;
                s.out = o;
                s.phase = 2;
                for (int i = 0; i < n; ++i) {
                    s.writes.push_back(var("g" + S(i)));
                    s.code += "g" + S(i) + " = zero(); ";
                }
                if (A.out_wslot >= 0) {
                    s.writes.push_back(var("w" + S(A.out_wslot)));
                    s.code += "w" + S(A.out_wslot) + " = one();";
                }
                st.push_back(s);
                for (int i = A.rv_begin; i < A.rv_begin + A.rv_count; ++i) {
                    Stmt r = reverse_stmt(rins[i]);
                    r.out = o;
                    st.push_back(r);
                }
            }
            // Mean Value Form (Definition 5), left to right, and the form
            Stmt m;
            m.out = o;
            m.phase = 3;
            const std::string F = "F" + S(o);
            if (nie_only) {
                m.reads.push_back(var("nie" + S(o)));
                m.code = F + " = final_form(1, nie" + S(o) + ", nie" + S(o) + ");";
            } else {
                m.reads.push_back(var("fc" + S(o)));
                m.code = "{ iv mvf = fc" + S(o) + "; ";
                for (int i = 0; i < n; ++i) {
                    m.reads.push_back(var("g" + S(i)));
                    m.reads.push_back(var("X" + S(i)));
                    m.reads.push_back(var("c" + S(i), V_DBL));
                    m.code += "mvf = mvf_term(mvf, g" + S(i) + ", X" + S(i) + ", c" + S(i) + "); ";
                }
                m.reads.push_back(var("nie" + S(o)));
                m.code += F + " = final_form(" + S(form) + ", mvf, nie" + S(o) + "); }";
                m.cost = 2.0 * n + 2.0;
            }
            m.writes.push_back(var(F));
            st.push_back(m);
        }
    }
};

struct Chunk {
    std::vector<Stmt> body;
};

struct Plan {
    std::vector<Chunk> chunks;
    std::vector<std::set<int>> live_in;    // per chunk: read before written
    std::vector<std::set<int>> live_out;   // per chunk: written or passed through and read later
    std::vector<std::map<int, int>> slot_after;   // per boundary (after chunk c): var -> state slot
    std::map<int, int> slot_pre;                  // after the prologue
    int n_slots = 0;
    long long loads = 0, stores = 0, recomputed = 0;   // per subdomain
};

// Cut the statement list into chunks of bounded estimated work and statement
// count, then insert the recomputation of each reverse chunk's own forward
// values according to the policy.
std::vector<Chunk> cut(const Builder& B, double budget, int max_stmts, int policy, long long* recomputed) {
    std::vector<Chunk> ch;
    Chunk cur;
    double cost = 0.0;
    for (const Stmt& s : B.st) {
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
    for (const Stmt& s : B.st)
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

// liveness over chunks and state slots for the values that cross boundaries
void plan_state(const Builder& B, Plan& pl, const std::vector<int>& pro_writes, const std::vector<int>& epi_reads) {
    const int C = (int)pl.chunks.size();
    std::vector<std::set<int>> use(C), def(C);
    for (int c = 0; c < C; ++c)
        for (const Stmt& s : pl.chunks[c].body) {
            for (int v : s.reads) if (!def[c].count(v)) use[c].insert(v);
            for (int v : s.writes) def[c].insert(v);
        }
    pl.live_in.assign(C, {});
    pl.live_out.assign(C, {});
    std::set<int> live(epi_reads.begin(), epi_reads.end());
    for (int c = C - 1; c >= 0; --c) {
        pl.live_out[c] = live;
        std::set<int> in = use[c];
        for (int v : live) if (!def[c].count(v)) in.insert(v);
        pl.live_in[c] = in;
        live = in;
    }
    // slots: the prologue writes pro_writes; those live into chunk 0 get slots.
    // A slot released in chunk c (its variable is last read there) is reused
    // from chunk c + 1 on: inside chunk c a live-in may be loaded after another
    // variable's store.
    std::vector<int> free_slots, released;
    int next = 0;
    auto get = [&]() { if (!free_slots.empty()) { int s = free_slots.back(); free_slots.pop_back(); return s; } return next++; };
    std::map<int, int> cur;
    for (int v : pro_writes) if (live.count(v)) cur[v] = get();
    pl.slot_pre = cur;
    pl.slot_after.assign(C, {});
    for (int c = 0; c < C; ++c) {
        free_slots.insert(free_slots.end(), released.begin(), released.end());
        released.clear();
        std::map<int, int> nxt;
        for (auto& kv : cur) {
            if (pl.live_out[c].count(kv.first)) {
                nxt[kv.first] = kv.second;     // passes through, or is redefined in place
                if (def[c].count(kv.first)) pl.stores += 1;
            } else {
                released.push_back(kv.second);
            }
        }
        for (int v : pl.live_out[c])
            if (!nxt.count(v)) {
                nxt[v] = get();
                pl.stores += 1;
            }
        pl.loads += (long long)use[c].size();
        cur = nxt;
        pl.slot_after[c] = cur;
    }
    pl.n_slots = next;
}

// C++ of one chunk function
std::string chunk_fn(const Builder& B, const Plan& pl, int c) {
    const Chunk& ch = pl.chunks[c];
    const std::map<int, int>& in_slots = c == 0 ? pl.slot_pre : pl.slot_after[c - 1];
    const std::map<int, int>& out_slots = pl.slot_after[c];
    std::string s = "extern \"C\" __device__ __noinline__ void ivb_ck" + S(c) +
                    "(double* __restrict__ st, const int ss) {\n  using namespace ivb;\n";
    // declarations of every variable the chunk touches
    std::set<int> touched;
    for (const Stmt& t : ch.body) {
        for (int v : t.reads) touched.insert(v);
        for (int v : t.writes) touched.insert(v);
    }
    {
        std::string dv, dd;
        for (int v : touched) {
            if (B.vtype[v] == V_DBL) dd += (dd.empty() ? "  double " : ", ") + B.vname[v];
            else dv += (dv.empty() ? "  iv " : ", ") + B.vname[v];
        }
        if (!dv.empty()) s += dv + ";\n";
        if (!dd.empty()) s += dd + ";\n";
    }
    // last write of each variable that leaves the chunk: store right after it
    std::map<int, size_t> last_write;
    for (size_t i = 0; i < ch.body.size(); ++i)
        for (int v : ch.body[i].writes) last_write[v] = i;
    std::set<int> loaded;
    auto load = [&](int v) -> std::string {
        const int slot = in_slots.at(v);
        if (B.vtype[v] == V_DBL) return "  " + B.vname[v] + " = st_d(st, ss, " + S(slot) + ");\n";
        return "  " + B.vname[v] + " = st_ld(st, ss, " + S(slot) + ");\n";
    };
    std::set<int> written;
    for (size_t i = 0; i < ch.body.size(); ++i) {
        const Stmt& t = ch.body[i];
        // live-ins are loaded before their first read (the scheduler hoists them)
        for (int v : t.reads)
            if (!written.count(v) && !loaded.count(v)) {
                s += load(v);
                loaded.insert(v);
            }
        s += "  " + t.code + "\n";
        for (int v : t.writes) written.insert(v);
        for (int v : t.writes)
            if (last_write[v] == i && out_slots.count(v) && pl.live_out[c].count(v)) {
                const int slot = out_slots.at(v);
                if (B.vtype[v] == V_DBL) s += "  st_sd(st, ss, " + S(slot) + ", " + B.vname[v] + ");\n";
                else s += "  st_st(st, ss, " + S(slot) + ", " + B.vname[v] + ");\n";
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

std::string unit_head(int emulate, bool kernel_unit) {
    std::string s = "#define IVB_EMU " + S(emulate) + "\n#define IVB_HEAVY static __noinline__\n";
    if (!kernel_unit) s += "#define IVB_JIT_EXTERN_TABLES\n";
    s += kPrelude;
    s += "#include \"ivb_bound_common.cuh\"\n";
    s += kStateHelpers;
    return s;
}

// the kernel unit: tile loop, Step 1, the chunk calls, tests and Step 3
std::string kernel_unit(const Builder& B, const Plan& pl, int block_max, int min_blocks, int emulate) {
    std::string s = unit_head(emulate, true);
    for (size_t c = 0; c < pl.chunks.size(); ++c)
        s += "extern \"C\" __device__ void ivb_ck" + S(c) + "(double* __restrict__ st, const int ss);\n";
    const int n = B.n, no = B.no;
    s += "extern \"C\" __global__ void __launch_bounds__(" + S(block_max) + ", " + S(min_blocks) +
         ") ivb_jit_bound(const ivb::KParams P) {\n";
    s += "  using namespace ivb;\n";
    s += "  double* const st = P.gframe + (size_t)blockIdx.x * P.frame_units * blockDim.x + threadIdx.x;\n";
    s += "  const int ss = blockDim.x;\n";
    s += "  tile_loop(P, [&](const Sub& s) {\n";
    {
        std::string f = "    iv ";
        for (int o = 0; o < no; ++o) f += (o ? ", F" : "F") + S(o) + " = zero()";
        s += f + ";\n";
    }
    s += "    bool cert = false;\n";
    s += "    double obj_lo = from_bits(0x7FF0000000000000LL);\n";
    s += "    double ub = from_bits(0x7FF0000000000000LL);\n";
    s += "    if (s.valid) {\n";
    s += "      unsigned int kk = s.k;\n";
    for (int i = 0; i < n; ++i) {
        s += "      { iv X; double c; decode_dim(s.rec, " + S(n) + ", " + S(i) + ", kk, X, c);";
        auto itX = B.vid.find("X" + S(i));
        auto itc = B.vid.find("c" + S(i));
        if (itX != B.vid.end() && pl.slot_pre.count(itX->second))
            s += " st_st(st, ss, " + S(pl.slot_pre.at(itX->second)) + ", X);";
        if (itc != B.vid.end() && pl.slot_pre.count(itc->second))
            s += " st_sd(st, ss, " + S(pl.slot_pre.at(itc->second)) + ", c);";
        s += " }\n";
    }
    for (size_t c = 0; c < pl.chunks.size(); ++c) s += "      ivb_ck" + S(c) + "(st, ss);\n";
    const std::map<int, int>& fin = pl.slot_after.empty() ? pl.slot_pre : pl.slot_after.back();
    s += std::string("      bool feas = ") + (B.P.has_eq ? "false" : "true") + ";\n";
    for (int o = 0; o < no; ++o) {
        s += "      F" + S(o) + " = st_ld(st, ss, " + S(fin.at(B.vid.at("F" + S(o)))) + ");\n";
        s += "      if (excludes_feasible(" + S(B.P.out_kind[o]) + "u, F" + S(o) + ")) cert = true;\n";
        if (o == B.P.obj) s += "      obj_lo = F" + S(o) + ".lo;\n";
        if (B.P.out_kind[o] == OUT_INEQ)
            s += "      if (!le0(st_ld(st, ss, " + S(fin.at(B.vid.at("fc" + S(o)))) + ").hi)) feas = false;\n";
    }
    s += "      if (feas) ub = st_ld(st, ss, " + S(fin.at(B.vid.at("fc" + S(B.P.obj)))) + ").hi;\n";
    s += "      if (cert) obj_lo = from_bits(0x7FF0000000000000LL);\n";
    s += "    }\n";
    for (int o = 0; o < no; ++o) s += "    reduce_output(P, s, " + S(no) + ", " + S(o) + ", F" + S(o) + ");\n";
    s += "    reduce_extras(P, s, " + S(no) + ", ub, obj_lo);\n";
    s += "  });\n}\n";
    return s;
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
    for (int i = 0; i < B.n; ++i) { B.var("X" + S(i)); B.var("c" + S(i), V_DBL); }
    B.build();
    Plan pl;
    pl.chunks = cut(B, pol.chunk_cost, pol.chunk_stmts, B.nie_only ? 0 : pol.recompute, &pl.recomputed);
    std::vector<int> pro, epi;
    for (int i = 0; i < B.n; ++i) { pro.push_back(B.vid.at("X" + S(i))); pro.push_back(B.vid.at("c" + S(i))); }
    for (int o = 0; o < B.no; ++o) {
        epi.push_back(B.vid.at("F" + S(o)));
        if (P.out_kind[o] == OUT_INEQ || o == P.obj) epi.push_back(B.vid.at("fc" + S(o)));
    }
    plan_state(B, pl, pro, epi);
    SegSource out;
    out.state_units = 2 * std::max(pl.n_slots, 1);
    out.chunks = (int)pl.chunks.size();
    out.loads = pl.loads;
    out.stores = pl.stores;
    out.recomputed = pl.recomputed;
    out.kernel = kernel_unit(B, pl, block_max, min_blocks, emulate);
    // chunks spread over units of similar size, compiled in parallel
    const int C = (int)pl.chunks.size();
    const int U = std::max(1, std::min(C, pol.units));
    for (int u = 0; u < U; ++u) {
        std::string src = unit_head(emulate, false);
        const int b = (int)((long long)C * u / U), e = (int)((long long)C * (u + 1) / U);
        for (int c = b; c < e; ++c) src += chunk_fn(B, pl, c);
        out.units.push_back(src);
    }
    return out;
}

std::string jit_seg_compile(const SegSource& src, int max_regs, std::vector<char>& cubin, std::string& tables_name,
                            double* seconds, int* registers, int* spill_bytes) {
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
