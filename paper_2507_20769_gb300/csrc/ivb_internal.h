// ivb_internal.h -- device program format shared by the host tape compiler
// (ivb_compile.cpp) and the CUDA kernels (ivb_kernels.cu).
//
// The tape (Section 3.2, Fig. 5) is compiled into straight-line instruction
// streams that every thread interprets for its own subdomain:
//   point sweep    : interval values on the degenerate box [c,c] (f(c) of
//                    Definition 5), liveness-reused value slots
//   tangent sweep  : interval values plus n tangent intervals per slot
//                    (forward mode, Section 3.2)
//   adjoint, per output o: a forward sweep over the cone of o writing every
//                    value to its own tape record, then the reverse sweep over
//                    the same cone with liveness-reused adjoint slots
// Operands name a slot (per-thread frame record), a variable of the box or
// an entry of the constant table, so VAR and CONST entries cost no storage.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ivb {

enum OpCode : uint32_t {
    OP_VAR = 0, OP_CONST = 1, OP_ADD = 2, OP_SUB = 3, OP_MUL = 4, OP_DIV = 5,
    OP_SQR = 6, OP_SQRT = 7, OP_EXP = 8, OP_LOG = 9, OP_NEG = 10
};
enum OperandKind : uint32_t { K_SLOT = 0, K_VAR = 1, K_CONST = 2, K_NONE = 3 };
enum OutKind : uint8_t { OUT_OBJ = 0, OUT_INEQ = 1, OUT_EQ = 2 };

// forward instruction: 8 bytes
//   w0 = op[0:5) | akind[5:7) | bkind[7:9) | dst[16:32)
//   w1 = a[0:16) | b[16:32)
struct Ins {
    uint32_t w0, w1;
};

// reverse (adjoint) instruction: 16 bytes
//   w0 = op[0:5) | a_init[5] | b_init[6] | a_none[7] | b_none[8] | wslot[16:32)
//   w1 = a_adj[0:16) | b_adj[16:32)             adjoint slots of the operands
//        (for op VAR: a_adj = variable index)
//   w2 = A[0:16) | B[16:32)                     value refs of the operands
//   w3 = V[0:16) | Akind[16:18) | Bkind[18:20) | Vkind[20:22)
// value refs name a tape record (K_SLOT), a variable or a constant
struct RIns {
    uint32_t w0, w1, w2, w3;
};

constexpr uint32_t kNoSlot = 0xFFFFu;

// one output's adjoint program inside the flat instruction arrays
struct AdjProgram {
    int32_t fw_begin, fw_count;   // forward instructions (Ins) of the cone
    int32_t rv_begin, rv_count;   // reverse instructions (RIns)
    int32_t tape_records;         // records written by the forward sweep
    int32_t adj_slots;            // adjoint slot file size
    int32_t out_ref;              // value ref of the output (tape record)
    int32_t out_kind_ref;         // K_SLOT / K_VAR / K_CONST of out_ref
    int32_t out_wslot;            // adjoint slot of the output entry
    int32_t pad;
};

// Per-thread frame layout, in doubles ("units"), common to all phases:
//   [0, 2n)                 X_i (lo, hi)
//   [2n, 3n)                c_i
//   [3n, 3n + 2 n_out)      f(c) of every output (point sweep results)
//   [phase_base, ...)       phase region (reused by each phase)
// Element u of thread t sits at frame[u * stride + t].
struct FrameLayout {
    int32_t n, n_out;
    int32_t x_base, c_base, fc_base, phase_base;
    int32_t pt_units;             // point sweep: 2 * pt_slots
    int32_t tan_rec;              // tangent record size = 2 (1 + n)
    int32_t tan_units;            // tangent sweep: tan_rec * tan_slots
    int32_t adj_units;            // adjoint phase: max over outputs
    int32_t total_fwd, total_adj; // frame units in forward / adjoint mode
};

struct HostProgram {
    int32_t n_vars = 0, n_out = 0, obj = -1;
    bool has_eq = false;
    // point sweep
    int32_t pt_begin = 0, pt_count = 0, pt_slots = 0;
    int32_t pt_out_ref[64], pt_out_kind[64];
    // tangent sweep (all outputs)
    int32_t tan_begin = 0, tan_count = 0, tan_slots = 0;
    int32_t tan_out_ref[64], tan_out_kind[64];
    // adjoint programs, one per output
    AdjProgram adj[64];
    uint8_t out_kind[64];
    // flat arrays
    Ins* ins = nullptr;   int32_t n_ins = 0;
    RIns* rins = nullptr; int32_t n_rins = 0;
    double* consts = nullptr; int32_t n_consts = 0;
    FrameLayout L{};
    // static op counts (per subdomain) for reporting
    int64_t op_hist[16] = {0};
    // directed endpoint operations per subdomain, per category (ivb.h IVB_CNT_*)
    int64_t cnt_fwd[8] = {0}, cnt_adj[8] = {0};
    // the same for the natural interval extension alone (form 1): no gradients
    int64_t cnt_nie_fwd[8] = {0}, cnt_nie_adj[8] = {0};
};

}  // namespace ivb
