// ivb_compile.cpp -- host compiler: tape (Section 3.2, Fig. 5) -> device
// instruction streams with liveness-based slot allocation.
//
// Reordering is not needed for bit-exact results: every instruction computes
// the same function of the same operand values as the tape entry it comes
// from, so the per-thread evaluation order only decides storage, never values.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_compile.h"
#include "ivb_internal.h"

namespace ivb {

static bool is_binary(int op) { return op == OP_ADD || op == OP_SUB || op == OP_MUL || op == OP_DIV; }
static bool is_unary(int op) {
    return op == OP_SQR || op == OP_SQRT || op == OP_EXP || op == OP_LOG || op == OP_NEG;
}

std::string validate_tape(const ivb_tape* t) {
    if (!t) return "tape is NULL";
    if (t->n_vars < 1 || t->n_vars > IVB_MAX_VARS) return "n_vars must be in [1, 32]";
    if (t->n_ops < 1 || t->n_ops > IVB_MAX_OPS) return "n_ops must be in [1, 2^20]";
    if (t->n_outputs < 1 || t->n_outputs > IVB_MAX_OUTPUTS) return "n_outputs must be in [1, 64]";
    if (!t->ops || !t->out_idx || !t->out_kind) return "tape arrays must not be NULL";
    for (int32_t i = 0; i < t->n_ops; ++i) {
        const ivb_op& e = t->ops[i];
        const int op = e.op;
        if (op == OP_VAR) {
            if (e.a < 0 || e.a >= t->n_vars) return "entry " + std::to_string(i) + ": VAR index out of range";
        } else if (op == OP_CONST) {
            if (!std::isfinite(e.c)) return "entry " + std::to_string(i) + ": constant is not finite";
        } else if (is_binary(op)) {
            if (e.a < 0 || e.a >= i || e.b < 0 || e.b >= i)
                return "entry " + std::to_string(i) + ": operand does not refer to an earlier entry";
        } else if (is_unary(op)) {
            if (e.a < 0 || e.a >= i) return "entry " + std::to_string(i) + ": operand does not refer to an earlier entry";
        } else {
            return "entry " + std::to_string(i) + ": unknown opcode " + std::to_string(op);
        }
    }
    int n_obj = 0;
    for (int32_t o = 0; o < t->n_outputs; ++o) {
        if (t->out_idx[o] < 0 || t->out_idx[o] >= t->n_ops) return "output index out of range";
        if (t->out_kind[o] > OUT_EQ) return "unknown output kind";
        if (t->out_kind[o] == OUT_OBJ) ++n_obj;
    }
    if (n_obj != 1) return "exactly one objective output is required";
    return "";
}

namespace {

struct SlotAlloc {
    std::vector<int32_t> free_;  // free slot numbers, kept sorted descending (pop lowest)
    int32_t n = 0;
    int32_t get() {
        if (!free_.empty()) { int32_t s = free_.back(); free_.pop_back(); return s; }
        return n++;
    }
    void put(int32_t s) {
        // insert keeping descending order so that back() is the lowest slot
        auto it = free_.begin();
        while (it != free_.end() && *it > s) ++it;
        free_.insert(it, s);
    }
};

inline uint32_t pack_ins(uint32_t op, uint32_t ak, uint32_t bk, uint32_t dst) {
    return (op & 31u) | ((ak & 3u) << 5) | ((bk & 3u) << 7) | ((dst & 0xFFFFu) << 16);
}

}  // namespace

// Build the device program. Returns "" on success.
std::string compile_tape(const ivb_tape* t, HostProgram& P, std::vector<Ins>& ins, std::vector<RIns>& rins,
                         std::vector<double>& consts) {
    const int32_t T = t->n_ops, n = t->n_vars, no = t->n_outputs;
    P.n_vars = n;
    P.n_out = no;
    for (int o = 0; o < no; ++o) {
        P.out_kind[o] = t->out_kind[o];
        if (t->out_kind[o] == OUT_OBJ) P.obj = o;
        if (t->out_kind[o] == OUT_EQ) P.has_eq = true;
    }
    // constant table: one entry per CONST tape entry
    std::vector<int32_t> cidx(T, -1);
    for (int32_t i = 0; i < T; ++i)
        if (t->ops[i].op == OP_CONST) { cidx[i] = (int32_t)consts.size(); consts.push_back(t->ops[i].c); }

    // entries needed by some output
    std::vector<char> need(T, 0);
    for (int o = 0; o < no; ++o) need[t->out_idx[o]] = 1;
    for (int32_t i = T - 1; i >= 0; --i) {
        if (!need[i]) continue;
        const int op = t->ops[i].op;
        if (is_binary(op)) { need[t->ops[i].a] = 1; need[t->ops[i].b] = 1; }
        else if (is_unary(op)) need[t->ops[i].a] = 1;
    }
    for (int32_t i = 0; i < T; ++i) if (need[i]) P.op_hist[t->ops[i].op]++;

    // ---------------------------------------------------- point / tangent sweep
    {
        std::vector<int32_t> last(T, -1);
        for (int32_t i = 0; i < T; ++i) {
            if (!need[i]) continue;
            const int op = t->ops[i].op;
            if (is_binary(op)) { last[t->ops[i].a] = i; last[t->ops[i].b] = i; }
            else if (is_unary(op)) last[t->ops[i].a] = i;
        }
        for (int o = 0; o < no; ++o) last[t->out_idx[o]] = T;  // outputs live to the end
        std::vector<int32_t> slot(T, -1);
        SlotAlloc sa;
        P.pt_begin = (int32_t)ins.size();
        auto ref = [&](int32_t e, uint32_t& kind) -> uint32_t {
            const int op = t->ops[e].op;
            if (op == OP_VAR) { kind = K_VAR; return (uint32_t)t->ops[e].a; }
            if (op == OP_CONST) { kind = K_CONST; return (uint32_t)cidx[e]; }
            kind = K_SLOT;
            return (uint32_t)slot[e];
        };
        for (int32_t i = 0; i < T; ++i) {
            if (!need[i]) continue;
            const ivb_op& e = t->ops[i];
            if (e.op == OP_VAR || e.op == OP_CONST) continue;
            uint32_t ak = K_NONE, bk = K_NONE, av = 0, bv = 0;
            av = ref(e.a, ak);
            if (is_binary(e.op)) bv = ref(e.b, bk);
            int32_t d = sa.get();
            if (d >= 0xFFFF) return "too many live values (slot limit 65535)";
            slot[i] = d;
            Ins I;
            I.w0 = pack_ins(e.op, ak, bk, (uint32_t)d);
            I.w1 = (av & 0xFFFFu) | ((bv & 0xFFFFu) << 16);
            ins.push_back(I);
            // free operands whose last use is this entry (after allocating dst)
            if (ak == K_SLOT && last[e.a] == i) { sa.put(slot[e.a]); last[e.a] = -2; }
            if (bk == K_SLOT && e.b != e.a && last[e.b] == i) { sa.put(slot[e.b]); last[e.b] = -2; }
        }
        P.pt_count = (int32_t)ins.size() - P.pt_begin;
        P.pt_slots = sa.n;
        P.tan_begin = P.pt_begin;
        P.tan_count = P.pt_count;
        P.tan_slots = sa.n;
        for (int o = 0; o < no; ++o) {
            uint32_t k;
            uint32_t r = ref(t->out_idx[o], k);
            P.pt_out_ref[o] = (int32_t)r;
            P.pt_out_kind[o] = (int32_t)k;
            P.tan_out_ref[o] = (int32_t)r;
            P.tan_out_kind[o] = (int32_t)k;
        }
    }

    // ---------------------------------------------------- adjoint, per output
    int32_t adj_units_max = 0;
    for (int o = 0; o < no; ++o) {
        const int32_t out = t->out_idx[o];
        std::vector<char> cone(out + 1, 0);
        cone[out] = 1;
        for (int32_t i = out; i >= 0; --i) {
            if (!cone[i]) continue;
            const int op = t->ops[i].op;
            if (is_binary(op)) { cone[t->ops[i].a] = 1; cone[t->ops[i].b] = 1; }
            else if (is_unary(op)) cone[t->ops[i].a] = 1;
        }
        AdjProgram& A = P.adj[o];
        // forward: every interior cone entry gets its own tape record
        std::vector<int32_t> rec(out + 1, -1);
        int32_t n_rec = 0;
        A.fw_begin = (int32_t)ins.size();
        auto vref = [&](int32_t e, uint32_t& kind) -> uint32_t {
            const int op = t->ops[e].op;
            if (op == OP_VAR) { kind = K_VAR; return (uint32_t)t->ops[e].a; }
            if (op == OP_CONST) { kind = K_CONST; return (uint32_t)cidx[e]; }
            kind = K_SLOT;
            return (uint32_t)rec[e];
        };
        for (int32_t i = 0; i <= out; ++i) {
            if (!cone[i]) continue;
            const ivb_op& e = t->ops[i];
            if (e.op == OP_VAR || e.op == OP_CONST) continue;
            uint32_t ak = K_NONE, bk = K_NONE, av = 0, bv = 0;
            av = vref(e.a, ak);
            if (is_binary(e.op)) bv = vref(e.b, bk);
            if (n_rec >= 0xFFFF) return "cone too large (tape record limit 65535)";
            rec[i] = n_rec++;
            Ins I;
            I.w0 = pack_ins(e.op, ak, bk, (uint32_t)rec[i]);
            I.w1 = (av & 0xFFFFu) | ((bv & 0xFFFFu) << 16);
            ins.push_back(I);
        }
        A.fw_count = (int32_t)ins.size() - A.fw_begin;
        A.tape_records = n_rec;
        {
            uint32_t k;
            A.out_ref = (int32_t)vref(out, k);
            A.out_kind_ref = (int32_t)k;
        }
        // reverse: adjoint slots allocated at the first contribution (the
        // consumer with the largest index) and released after the entry
        std::vector<int32_t> aslot(out + 1, -1);
        SlotAlloc sa;
        A.rv_begin = (int32_t)rins.size();
        const int out_op = t->ops[out].op;
        A.out_wslot = -1;
        if (out_op != OP_CONST) { aslot[out] = sa.get(); A.out_wslot = aslot[out]; }
        for (int32_t i = out; i >= 0; --i) {
            if (!cone[i]) continue;
            const ivb_op& e = t->ops[i];
            if (e.op == OP_CONST) continue;
            RIns R{0, 0, 0, 0};
            const int32_t w = aslot[i];
            if (w < 0) return "internal: cone entry without adjoint";
            if (e.op == OP_VAR) {
                R.w0 = (uint32_t)OP_VAR | ((uint32_t)w << 16);
                R.w1 = (uint32_t)e.a;
                rins.push_back(R);
                sa.put(w);
                continue;
            }
            uint32_t a_init = 0, b_init = 0, a_none = 0, b_none = 0;
            uint32_t a_adj = kNoSlot, b_adj = kNoSlot;
            auto contrib = [&](int32_t x, uint32_t& init, uint32_t& none, uint32_t& adj) {
                if (t->ops[x].op == OP_CONST) { none = 1; adj = kNoSlot; return; }
                if (aslot[x] < 0) { aslot[x] = sa.get(); init = 1; }
                adj = (uint32_t)aslot[x];
            };
            contrib(e.a, a_init, a_none, a_adj);
            if (is_binary(e.op)) contrib(e.b, b_init, b_none, b_adj);
            else b_none = 1;
            if (sa.n >= 0xFFFF) return "too many live adjoints (slot limit 65535)";
            uint32_t Ak = K_NONE, Bk = K_NONE, Vk = K_SLOT;
            uint32_t Av = vref(e.a, Ak), Bv = 0;
            if (is_binary(e.op)) Bv = vref(e.b, Bk);
            uint32_t Vv = (uint32_t)rec[i];
            R.w0 = (uint32_t)e.op | (a_init << 5) | (b_init << 6) | (a_none << 7) | (b_none << 8) |
                   ((uint32_t)w << 16);
            R.w1 = (a_adj & 0xFFFFu) | ((b_adj & 0xFFFFu) << 16);
            R.w2 = (Av & 0xFFFFu) | ((Bv & 0xFFFFu) << 16);
            R.w3 = (Vv & 0xFFFFu) | ((Ak & 3u) << 16) | ((Bk & 3u) << 18) | ((Vk & 3u) << 20);
            rins.push_back(R);
            sa.put(w);
        }
        A.rv_count = (int32_t)rins.size() - A.rv_begin;
        A.adj_slots = sa.n;
        const int32_t units = 2 * n + 2 * A.adj_slots + 2 * A.tape_records;
        if (units > adj_units_max) adj_units_max = units;
    }

    // ---------------------------------------------------- operation counts
    // canonical endpoint operations per subdomain (categories of ivb.h)
    enum { ADD = 0, MUL = 1, DIV = 2, RCP = 3, SQRT = 4, EXP = 5, LOG = 6, RN = 7 };
    auto value_cost = [](int op, int64_t* c) {
        switch (op) {
        case OP_ADD: case OP_SUB: c[ADD] += 2; break;
        case OP_MUL: case OP_SQR: c[MUL] += 2; break;
        case OP_DIV: c[DIV] += 2; break;
        case OP_SQRT: c[SQRT] += 2; break;
        case OP_EXP: c[EXP] += 2; break;
        case OP_LOG: c[LOG] += 2; break;
        }
    };
    auto count_values = [&](int32_t begin, int32_t count, int64_t* c) {
        for (int32_t i = begin; i < begin + count; ++i) value_cost((int)(ins[i].w0 & 31u), c);
    };
    auto count_tangents = [&](int32_t begin, int32_t count, int64_t* c) {
        for (int32_t i = begin; i < begin + count; ++i) {
            const int op = (int)(ins[i].w0 & 31u);
            const uint32_t ak = (ins[i].w0 >> 5) & 3u, bk = (ins[i].w0 >> 7) & 3u;
            const bool az = ak == K_CONST, bz = bk == K_CONST || bk == K_NONE;
            value_cost(op, c);
            switch (op) {
            case OP_ADD: case OP_SUB: if (!az && !bz) c[ADD] += 2LL * n; break;
            case OP_MUL: c[MUL] += (az || bz) ? 2LL * n : 4LL * n; break;   // second product fused into the sum
            case OP_DIV:
                c[RCP] += 2;
                if (bz) c[MUL] += 2LL * n;
                else c[MUL] += 4LL * n;                              // V * db fused into the difference
                break;
            case OP_SQR: c[MUL] += 2 + 2LL * n; break;
            case OP_SQRT: c[MUL] += 2 + 2LL * n; c[RCP] += 2; break;
            case OP_EXP: c[MUL] += 2LL * n; break;
            case OP_LOG: c[RCP] += 2; c[MUL] += 2LL * n; break;
            }
        }
    };
    auto count_reverse = [&](int32_t begin, int32_t count, int64_t* c) {
        for (int32_t i = begin; i < begin + count; ++i) {
            const RIns& R = rins[i];
            const int op = (int)(R.w0 & 31u);
            const bool ai = (R.w0 >> 5) & 1u, bi = (R.w0 >> 6) & 1u, an = (R.w0 >> 7) & 1u, bn = (R.w0 >> 8) & 1u;
            const int acc = (an ? 0 : (ai ? 0 : 2)) + (bn ? 0 : (bi ? 0 : 2));
            switch (op) {
            case OP_VAR: c[ADD] += 2; break;
            case OP_ADD: case OP_SUB: case OP_NEG: c[ADD] += acc; break;
            // product contributions: the accumulating add is fused into the multiply
            case OP_MUL: c[MUL] += (an ? 0 : 2) + (bn ? 0 : 2); break;
            case OP_DIV: c[RCP] += 2; c[MUL] += (an ? 0 : 2) + (bn ? 0 : 4); break;
            case OP_SQR: c[MUL] += 4; break;
            case OP_SQRT: c[MUL] += 4; c[RCP] += 2; break;
            case OP_EXP: c[MUL] += 2; break;
            case OP_LOG: c[RCP] += 2; c[MUL] += 2; break;
            }
        }
    };
    for (int64_t* c : {P.cnt_fwd, P.cnt_adj}) {
        c[RN] += 6LL * n;                                   // decode: endpoints and centre
        count_values(P.pt_begin, P.pt_count, c);            // point sweep f(c)
        c[ADD] += 2LL * n;                                  // MVF: X - c once per dimension
        c[MUL] += 2LL * n * no;                             // each term fused into the sum
    }
    count_tangents(P.tan_begin, P.tan_count, P.cnt_fwd);
    for (int o = 0; o < no; ++o) {
        count_values(P.adj[o].fw_begin, P.adj[o].fw_count, P.cnt_adj);
        count_reverse(P.adj[o].rv_begin, P.adj[o].rv_count, P.cnt_adj);
    }
    // form 1: decode, point sweep (for the centre upper bound) and the value sweep over X
    for (int64_t* c : {P.cnt_nie_fwd, P.cnt_nie_adj}) {
        c[RN] += 6LL * n;
        count_values(P.pt_begin, P.pt_count, c);
    }
    count_values(P.tan_begin, P.tan_count, P.cnt_nie_fwd);
    for (int o = 0; o < no; ++o) count_values(P.adj[o].fw_begin, P.adj[o].fw_count, P.cnt_nie_adj);

    // ---------------------------------------------------- frame layout
    FrameLayout& L = P.L;
    L.n = n;
    L.n_out = no;
    L.x_base = 0;
    L.c_base = 2 * n;
    L.fc_base = 3 * n;
    L.phase_base = 3 * n + 2 * no;
    L.pt_units = 2 * P.pt_slots;
    L.tan_rec = 2 * (1 + n);
    L.tan_units = L.tan_rec * P.tan_slots;
    L.adj_units = adj_units_max;
    L.total_fwd = L.phase_base + (L.pt_units > L.tan_units ? L.pt_units : L.tan_units);
    L.total_adj = L.phase_base + (L.pt_units > L.adj_units ? L.pt_units : L.adj_units);
    return "";
}

}  // namespace ivb
