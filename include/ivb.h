/*
 * ivb.h -- C ABI of the GB300 (sm_103a) interval Mean Value Form subdomain
 * bounding library.
 *
 * Method (Zhang et al., "Accelerating Deterministic Global Optimization via
 * GPU-parallel Interval Arithmetic"): each branch-and-bound node's box is
 * temporarily split into a uniform grid of subdomains (Section 2.2, splitting
 * technique; Section 3.1 Step 1); on every subdomain the objective and the
 * constraints are enclosed with the interval Mean Value Form
 * f(c) + <grad F(X), X - c> (Definition 5; Section 3.1 Step 2) in outward
 * rounded binary64; the enclosures are reduced to each node's refinement
 * (Section 3.1 Step 3): lower bound of the objective and an infeasibility
 * flag (Section 3.1, pruning by the feasibility check).
 *
 * Conventions for every entry point:
 *  - Pointers are plain host or device pointers; the library asks CUDA which
 *    kind each one is. The caller owns every array it passes in.
 *  - Calls are ordered on `cuda_stream` (NULL = the legacy default stream).
 *    A call that reads or writes any host array returns after the work is
 *    complete; a call on device arrays only returns after enqueueing.
 *  - Errors are reported by the return code, never by aborting; the text of
 *    the last error of a handle is available through ivb_last_error().
 *  - A handle is not re-entrant: use one handle per host thread.
 */
#ifndef IVB_H
#define IVB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IVB_ABI_VERSION 2
#define IVB_MAX_VARS 32        /* variables per problem */
#define IVB_MAX_OUTPUTS 64     /* objective + constraints per problem */
#define IVB_MAX_OPS 1048576    /* tape entries per problem */

typedef enum {
    IVB_OK = 0,
    IVB_EINVAL = 1,    /* an argument failed validation (message says which) */
    IVB_ENOMEM = 2,    /* device or pinned host allocation failed */
    IVB_ECUDA = 3,     /* a CUDA runtime call failed (message has its text) */
    IVB_ETAPE = 4,     /* the tape is malformed */
    IVB_ETIMEOUT = 5,  /* a bounded device wait ran out */
    IVB_ENOTSUP = 6    /* option combination not supported */
} ivb_status;

/* Tape alphabet: the intrinsic functions of a factorable function
 * (Definition 4), one DAG for objective and constraints (Section 3.2, Fig. 5). */
enum {
    IVB_OP_VAR = 0,    /* x_a                         (a = variable index)  */
    IVB_OP_CONST = 1,  /* the constant c                                    */
    IVB_OP_ADD = 2,    /* v_a + v_b                                         */
    IVB_OP_SUB = 3,    /* v_a - v_b                                         */
    IVB_OP_MUL = 4,    /* v_a * v_b                                         */
    IVB_OP_DIV = 5,    /* v_a / v_b                                         */
    IVB_OP_SQR = 6,    /* v_a^2                                             */
    IVB_OP_SQRT = 7,   /* sqrt(v_a)                                         */
    IVB_OP_EXP = 8,    /* exp(v_a)                                          */
    IVB_OP_LOG = 9,    /* log(v_a)                                          */
    IVB_OP_NEG = 10    /* -v_a                                              */
};

/* output kinds of the NLP in Section 3.1: min f s.t. g_i <= 0, h_j = 0 */
enum { IVB_OUT_OBJ = 0, IVB_OUT_INEQ = 1, IVB_OUT_EQ = 2 };

/* one tape entry, 24 bytes: operands a, b index EARLIER entries */
typedef struct {
    uint8_t op;
    uint8_t _pad[3];
    int32_t a, b;
    double c;
} ivb_op;

typedef struct {
    int32_t n_vars;            /* 1 .. IVB_MAX_VARS                         */
    int32_t n_ops;             /* 1 .. IVB_MAX_OPS                          */
    int32_t n_outputs;         /* 1 .. IVB_MAX_OUTPUTS                      */
    const ivb_op* ops;         /* host array [n_ops]                        */
    const int32_t* out_idx;    /* host array [n_outputs]: tape entry        */
    const uint8_t* out_kind;   /* host array [n_outputs]: IVB_OUT_*; exactly
                                  one IVB_OUT_OBJ                           */
} ivb_tape;

enum { IVB_GRAD_FORWARD = 0, IVB_GRAD_ADJOINT = 1 };
enum { IVB_FORM_MVF = 0, IVB_FORM_NIE = 1, IVB_FORM_MVF_NIE = 2 };
enum { IVB_SPLIT_UNIFORM = 0, IVB_SPLIT_LARGEST = 1, IVB_SPLIT_ADAPTIVE = 2 };

typedef struct {
    int32_t grad_mode;         /* IVB_GRAD_ADJOINT (default) or _FORWARD       */
    int32_t form;              /* IVB_FORM_MVF (default), _NIE, _MVF_NIE       */
    int32_t filter;            /* 1: objective minimum skips subdomains whose
                                  constraints are certainly violated (0)      */
    int32_t batched;           /* 1 (default): all nodes of a call in one
                                  persistent launch from a device node queue;
                                  0: one launch per node (plain path)         */
    int32_t use_graph;         /* 1 (default): replay the batched call as a
                                  CUDA graph                                  */
    int32_t autotune;          /* 1 (default): pick block size, blocks per SM
                                  and tile on first use                       */
    int32_t block_threads;     /* threads per block; 0 = tuned / default     */
    int32_t blocks_per_sm;     /* resident blocks per SM; 0 = tuned/default  */
    int32_t tile;              /* subdomains a block grabs at a time; 0: as
                                  many as it has threads (smallest tail)   */
    int32_t max_nodes;         /* capacity of one call (default 4096)       */
    int32_t frame_in_shared;   /* -1 auto (default), 0 global, 1 shared     */
    int32_t specialize;        /* 1: at creation, write the tape's programs
                                  out as straight-line CUDA, compile it with
                                  NVRTC for sm_103a and use it for
                                  ivb_bound_nodes / _ex (bit-identical bounds,
                                  values in registers instead of frame memory;
                                  creation fails with IVB_ENOTSUP if it cannot
                                  be compiled); the point sweep and each
                                  output's sweeps are functions of their own
                                  and the long primitives are called out of
                                  line, which halves the compile time at the
                                  same speed; 2: the same fully inlined;
                                  3: segmented -- the per-subdomain program
                                  cut into short chunk functions of bounded
                                  work and register use, values crossing
                                  chunks kept in a per-thread state area in
                                  device memory, the reverse sweep
                                  recomputing its segment's forward values
                                  from checkpoints (option recompute), chunks
                                  compiled in parallel and linked (adjoint
                                  mode only; for large tapes);
                                  0 (default): tape interpreter; -1: as 1 when
                                  the tape has at most 1024 interval
                                  operations per subdomain, else as 3 in
                                  adjoint mode and the interpreter in forward
                                  mode, and the autotuner keeps the
                                  interpreter instead when it times faster  */
    int32_t emulate;           /* tape-specialised kernel only: endpoint
                                  operations computed by an exact emulation
                                  on the integer pipes (bit-identical to the
                                  FP64 instructions), running beside the
                                  narrow FP64 pipe. Bitmask: 1 upper ends of
                                  products, 2 lower ends of products, 4 upper
                                  ends of sums and differences, 8 lower ends;
                                  -1 (default): the library's choice, now 0
                                  (no gain inside the bounding kernel)     */
    int32_t recompute;         /* segmented kernel: forward values of a
                                  reverse chunk's own segment that are
                                  recomputed from the segment's checkpoints
                                  instead of read back from the state area:
                                  0 none, 1 the cheap operations (+ - * sqr
                                  neg; the values of / sqrt exp log are
                                  stored), 2 all; -1 (default): the
                                  library's choice, now 0 (on this part the
                                  recomputed FP64 work costs more than the
                                  state traffic it saves)                  */
    int32_t seg_chunk;         /* segmented kernel: estimated FP64 issue
                                  slots per chunk (0 = default 320)         */
    int32_t seg_regs;          /* segmented kernel: register budget of every
                                  chunk function, 64..255 (0 = default 128) */
    int32_t threads_per_subdomain; /* segmented kernel with an own program
                                  per output: 1, 2 or 4 threads (in different
                                  warps of a block) share one subdomain, each
                                  running the programs of a group of its
                                  outputs; 0 (default): chosen by the
                                  autotuner among those compiled            */
    int32_t seg_sync;          /* segmented kernel: 1 the warps of a thread
                                  group wait for each other after every chunk
                                  function (they then run the same code and
                                  share the instruction cache), 0 they run
                                  freely; -1 (default): chosen by the
                                  autotuner                                  */
    int32_t seg_ilp;           /* segmented kernel: subdomains per thread,
                                  1 or 2 (two independent dependency chains
                                  per thread, every statement run on both,
                                  interleaved). With 2, the short operations
                                  out of line and an `emulate` policy, the
                                  two subdomains run in pairs instead: one
                                  call per operation computes both, the
                                  first on the FP64 pipe, the second's short
                                  operations under the policy on the integer
                                  pipes (dual-pipe). 0 (default): 1        */
    int32_t seg_outline;       /* segmented kernel: 1 calls + - * sqr and the
                                  fused accumulation out of line (a third of
                                  the code every warp streams through, a call
                                  per statement); 2 only * sqr and the fused
                                  accumulation (+ and - inline); 0 inlines
                                  them all; -1 (default): the library's
                                  choice, now 1                             */
} ivb_options;

typedef struct ivb_problem ivb_problem;

/* Fill `opt` with the defaults listed above. */
void ivb_options_default(ivb_options* opt);

/* Validate the tape, compile it into the device program and upload it.
 * Rejects (IVB_ETAPE): unknown opcodes, operands that do not refer to an
 * earlier entry, VAR indices outside [0, n_vars), non-finite constants,
 * outputs that are out of range, and anything other than exactly one
 * objective. `opt` may be NULL (defaults). On success *out owns device
 * memory until ivb_destroy(). */
ivb_status ivb_create_problem(const ivb_tape* tape, const ivb_options* opt, ivb_problem** out);

/* Steps 1-3 of Subdomain Lower Bounding (Section 3.1) for a batch of nodes.
 *   boxes          [n_nodes][n_vars][2] node boxes (lo, hi), finite, lo <= hi,
 *                  |endpoint| <= 2^1000
 *   splits_per_dim [n_nodes][n_vars], each >= 1, product <= 2^31 per node;
 *                  subdomain k of a node has j_i = (k / prod_{l<i} N_l) mod N_i
 *                  (dimension 0 fastest, as in Section 3.1.1)
 *   out_lb         [n_nodes] min over subdomains of lo(F_obj) (may be -inf)
 *   out_infeasible [n_nodes] 1 if some inequality's refinement lower end is
 *                  > 0 or some equality's refinement excludes 0
 * Host and device pointers may be mixed. 0 <= n_nodes <= max_nodes; an
 * empty batch returns IVB_OK without touching any array. */
ivb_status ivb_bound_nodes(ivb_problem* p, int32_t n_nodes, const double* boxes,
                           const int32_t* splits_per_dim, double* out_lb,
                           uint8_t* out_infeasible, void* cuda_stream);

/* As ivb_bound_nodes, with optional extra results (NULL to skip):
 *   out_ub     [n_nodes] smallest hi(f(c_k)) over subdomains whose centre
 *              c_k is certified feasible (every inequality has hi(g(c_k)) <= 0;
 *              none when equalities exist); +inf if none: a rigorous upper
 *              bound on the node's constrained minimum
 *   out_minlo  [n_nodes][n_outputs] refinement lower ends of every output
 *   out_maxhi  [n_nodes][n_outputs] refinement upper ends of every output */
ivb_status ivb_bound_nodes_ex(ivb_problem* p, int32_t n_nodes, const double* boxes,
                              const int32_t* splits_per_dim, double* out_lb,
                              uint8_t* out_infeasible, double* out_ub, double* out_minlo,
                              double* out_maxhi, void* cuda_stream);

/* Allocation-free variant of ivb_bound_nodes (the paper has no counterpart):
 * for callers that cannot allocate device memory while they run -- e.g. a
 * service whose GPU memory is reserved up front by another allocator, or a
 * loop that must not call cudaMalloc/cudaFree because they synchronize the
 * device and can fail under memory pressure. The call makes no allocation:
 * the node queue, reduction keys, work counter and an error word live in one
 * file-scope device array of 512 KiB, per-thread frames in shared memory.
 *   - boxes, splits_per_dim, out_lb, out_infeasible: DEVICE arrays of the
 *     device the problem was created on, with the layouts of ivb_bound_nodes;
 *     that device must be current (else IVB_EINVAL);
 *     1 <= n_nodes <= IVB_NOALLOC_MAX_NODES (larger or empty batches are
 *     rejected with IVB_EINVAL); problems whose per-thread frame does not fit
 *     in shared memory get IVB_ENOTSUP.
 *   - the first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (with that device current); make that first call
 *     before any stream capture.
 *   - every call on a device shares the one array and it keeps the last
 *     call's contents (each call resets what must start fixed: the counter,
 *     the keys and the error word); calls that overlap on the GPU race with
 *     each other, so order them (one stream, or events).
 *   - returns only after the work completes (it waits on cuda_stream):
 *     invalid boxes or splits, found on the device, are reported as
 *     IVB_EINVAL naming the first bad node; out_lb and out_infeasible are
 *     then unspecified for every node of the call.
 *   - the array stays allocated on every GPU that loads the library until
 *     the process exits. */
#define IVB_NOALLOC_MAX_NODES 256
ivb_status ivb_bound_nodes_noalloc(ivb_problem* p, int32_t n_nodes, const double* boxes,
                                   const int32_t* splits_per_dim, double* out_lb,
                                   uint8_t* out_infeasible, void* cuda_stream);

/* Per-subdomain enclosures (Step 2 without the reduction) for subdomains
 * first .. first+count-1 of ONE node:
 *   out_F  [count][n_outputs][2]          the enclosure of the chosen form
 *   out_Fc [count][n_outputs][2]          rigorous point value f(c_k) (or NULL)
 *   out_G  [count][n_outputs][n_vars][2]  gradient enclosure on X_k (or NULL)
 * count <= 2^24 per call. */
ivb_status ivb_enclose(ivb_problem* p, const double* box, const int32_t* splits_per_dim,
                       int64_t first, int64_t count, double* out_F, double* out_Fc,
                       double* out_G, void* cuda_stream);

/* Round-to-nearest point values and reverse-mode gradients of every output:
 *   x [n_points][n_vars] -> out_f [n_points][n_outputs],
 *   out_grad [n_points][n_outputs][n_vars] (or NULL). */
ivb_status ivb_point_grad(ivb_problem* p, int64_t n_points, const double* x, double* out_f,
                          double* out_grad, void* cuda_stream);

/* Split counts for one node (host arrays): uniform (Section 3.1.1: N per dim,
 * N = floor(target^(1/n))), largest (Section 3.1.1: widest dim only) or
 * adaptive (Section 3.1.2: uniform, then +1 on the dims of largest relative
 * width per subinterval while the product stays <= target). `ref_widths`
 * [n] scales widths for "relative" (NULL = absolute). */
ivb_status ivb_pick_splits(int32_t n, const double* box, const double* ref_widths,
                           int64_t target, int32_t strategy, int32_t* out_splits);

/* ---------------------------------------------------------------- B&B
 * Best-first spatial branch and bound (Section 3, Fig. 3) with this
 * library's Subdomain Lower Bounding as the lower-bounding solver; a
 * measurement harness for time-to-gap. Each iteration pops up to `batch`
 * open nodes of lowest lower bound, bisects each along the dimension of
 * largest width relative to the root box, optionally tightens each child by
 * constraint propagation (dropping children proven empty) and bounds the
 * children in one call of the bounding path. Upper bounds (in place of the
 * paper's local solver): the certified centre-point values of
 * ivb_bound_nodes_ex and, with corner_ub = 1, a descent-corner point per
 * iteration, evaluated rigorously on the host: for the child with the
 * smallest centre value, the corner of its box that the sign of the
 * objective's gradient enclosure over the box points to (centre where the
 * sign is unknown), else the midpoint between that corner and the centre,
 * used when certified feasible. All children of an iteration are bounded
 * and the incumbent updated before any is dropped; nodes are dropped when
 * infeasible or lb >= UB - max(eps_abs, eps_rel |UB|); the run stops when
 * UB - min(open lb) is within that tolerance or a limit is reached. */
typedef struct {
    int32_t batch;             /* nodes popped per iteration (>= 1)         */
    int32_t split_mode;        /* 0: fixed `splits`; 1 + IVB_SPLIT_*: picker */
    const int32_t* splits;     /* [n] fixed splits (split_mode 0), host     */
    int64_t target;            /* subdomains per node for the picker; 0: per
                                  iteration the smallest power of two >= 2^8
                                  (at most 2^20) with which the iteration's
                                  children cover four waves of the tuned
                                  bounding launch                            */
    double eps_abs, eps_rel;   /* optimality tolerance                      */
    int64_t max_nodes;         /* limit on bounded nodes (0 = none)         */
    double time_limit;         /* seconds (0 = none)                        */
    int32_t corner_ub;         /* 1: descent-corner upper bounds (default)  */
    int32_t propagate;         /* > 0: rounds of constraint propagation
                                  (forward-backward bound tightening against
                                  the constraints and f <= UB, on the host)
                                  applied to every box before it is bounded;
                                  boxes proven empty are dropped (0 default) */
    int32_t overlap;           /* 1: keep the GPU busy while the host works:
                                  the next batch is selected and enqueued
                                  before the results of the batch in flight
                                  are absorbed, so branching, propagation and
                                  upper bounding on the host overlap the
                                  bounding kernel (best-first order lags one
                                  batch); 0 (default): one batch at a time  */
} ivb_bnb_options;

typedef struct {
    double lb, ub;             /* final global bounds (lb <= min <= ub)     */
    int64_t iterations;        /* nodes branched                            */
    int64_t nodes_bounded;
    int64_t subdomains;        /* subdomains bounded in total               */
    double seconds;            /* wall clock of the whole solve             */
    int32_t converged;         /* 1 if the tolerance was met                */
    int64_t open_nodes;
    int64_t split_target;      /* subdomains per node the picker was given in
                                  the last iteration (0: fixed splits)       */
} ivb_bnb_result;

void ivb_bnb_options_default(ivb_bnb_options* o);

/* root: host array [n][2]; n must equal the problem's n_vars. */
ivb_status ivb_bnb_solve(ivb_problem* p, int32_t n, const double* root, const ivb_bnb_options* opt,
                         ivb_bnb_result* result, void* cuda_stream);

/* Constraint propagation on the host, no GPU needed: forward-backward bound
 * tightening (HC4-style projections through every operation) of n_boxes
 * boxes [n_boxes][n_vars][2] against the tape's inequalities (g <= 0),
 * equalities (h = 0) and f <= ub (ub = +inf: no objective cut), for at most
 * `passes` rounds (fewer when a round changes nothing). boxes_out receives
 * the tightened boxes (never wider than the input), infeasible[k] = 1 when
 * box k provably holds no such point. Outward-rounded on the CPU with the
 * kernels' interval rules. */
ivb_status ivb_propagate(const ivb_tape* tape, int32_t n_boxes, const double* boxes, double ub,
                         int32_t passes, double* boxes_out, uint8_t* infeasible);

/* Enclosure of the gradient of output `output` (index into the tape's
 * outputs) over one box [n_vars][2], on the host, no GPU needed: the kernels'
 * tangent (grad_mode IVB_GRAD_FORWARD) or reverse adjoint rules (Section 3.2),
 * fused accumulation included, outward-rounded on the CPU. G receives
 * [n_vars][2]. This is what the B&B's descent corner reads. IVB_EINVAL for a
 * bad output index or grad_mode, IVB_ETAPE for an invalid tape. */
ivb_status ivb_host_gradient(const ivb_tape* tape, const double* box, int32_t output, int32_t grad_mode,
                             double* G);

/* Tuning actually used by the batched path after autotuning (may be NULL):
 * block threads, blocks per SM, tile, frame in shared (0/1). */
ivb_status ivb_get_tuning(ivb_problem* p, int32_t* block_threads, int32_t* blocks_per_sm,
                          int32_t* tile, int32_t* frame_in_shared);

/* Launch configuration of the batched path after autotuning: the three
 * knobs of the bounding launch and what the tuner timed. */
typedef struct {
    int32_t block_threads;         /* threads per block                          */
    int32_t blocks_per_sm;         /* resident blocks per SM (grid = SMs x this) */
    int32_t tile;                  /* subdomains a block grabs from the work
                                      counter at a time (a multiple of the
                                      subdomains per pass)                      */
    int32_t frame_in_shared;       /* interpreter frames in shared memory (0/1)  */
    int32_t threads_per_subdomain; /* threads sharing one subdomain's outputs    */
    int32_t subdomains_per_pass;   /* block_threads / threads_per_subdomain x
                                      subdomains per thread                     */
    int32_t chunk_sync;            /* segmented kernel: groups kept on one chunk */
    int32_t kernel;                /* the reduce kernel the launches use: 0 the
                                      tape interpreter, 1 the tape-specialised
                                      kernel, 2 the segmented one (with
                                      specialize = -1 the autotuner times the
                                      interpreter beside the compiled kernel and
                                      keeps the faster)                          */
    int32_t candidates;            /* launch configurations timed (0: none)      */
    float best_ms, worst_ms;       /* their times on the tuning sample           */
} ivb_tuning;
ivb_status ivb_get_tuning_ex(ivb_problem* p, ivb_tuning* tuning);

/* The tape-specialised kernel of a problem (each may be NULL): active (0/1),
 * registers per thread, local memory bytes per thread, NVRTC compile time in
 * seconds, emulation policy compiled in. Not part of the paper's method:
 * reports how the bounds are computed, not what they are. */
ivb_status ivb_get_specialization(ivb_problem* p, int32_t* active, int32_t* registers,
                                  int32_t* local_bytes, double* compile_seconds, int32_t* emulate);

/* The segmented kernel of a problem (specialize = 3; each may be NULL):
 * doubles of per-thread state, chunk functions, state loads and stores per
 * subdomain (intervals and centre coordinates), forward operations recomputed
 * per subdomain by the reverse chunks, the recomputation policy compiled in,
 * and the subdomains each thread runs at once (seg_ilp). Zeros when the problem has no segmented kernel. Not part of the
 * paper's method: reports how the bounds are computed. */
ivb_status ivb_get_segmentation(ivb_problem* p, int32_t* state_units, int32_t* chunks, int64_t* state_loads,
                                int64_t* state_stores, int64_t* recomputed, int32_t* recompute, int32_t* ilp);

/* Generate and compile (NVRTC, sm_103a) the tape-specialised kernel of a
 * tape without loading it -- needs no GPU; compact = 1 as for specialize = 1,
 * 0 as for specialize = 2, 3 as for specialize = 3 (segmented, adjoint mode
 * only, default segmentation options), 4 as 3 with seg_ilp = 2 and emulate =
 * 15 (the paired dual-pipe form). Reports
 * ptxas' registers per thread (the largest over the functions compiled) and
 * spill-store bytes (summed), and the compile time (each may be NULL).
 * IVB_ETAPE for an invalid tape, IVB_ENOTSUP (message in ivb_last_error(NULL))
 * when the program does not compile. */
ivb_status ivb_specialize_compile(const ivb_tape* tape, int32_t grad_mode, int32_t compact, int32_t* registers,
                                  int32_t* spill_bytes, double* compile_seconds);

/* Static count of the outward-rounded endpoint operations one subdomain
 * needs under the problem's gradient mode and form (the canonical formulas:
 * value, tangent or adjoint rules, Mean Value Form, decode; with the natural
 * interval extension alone, IVB_FORM_NIE, the reduce kernels skip the
 * gradients: decode, point sweep and value sweep only), per category
 * IVB_CNT_*: the algorithmic work of the bounding kernel per subdomain.
 * Interval products count two directed multiplies (sign-case selection); a
 * product added to an accumulator (adjoint accumulation, tangent rules, the
 * Mean Value Form sum) is one fused multiply-add per end, counted as a
 * multiply with no separate add. */
enum {
    IVB_CNT_ADDSUB = 0, IVB_CNT_MUL = 1, IVB_CNT_DIV = 2, IVB_CNT_RCP = 3,
    IVB_CNT_SQRT = 4, IVB_CNT_EXP = 5, IVB_CNT_LOG = 6, IVB_CNT_RN = 7, IVB_CNT_N = 8
};
ivb_status ivb_op_counts(const ivb_problem* p, int64_t counts[IVB_CNT_N]);

/* Throughput of one FP64 primitive on the current GPU in lane operations
 * per second (a self-timed microbenchmark, 32 warps per SM, 8 independent
 * chains per thread): IVB_PROBE_DFMA is the FP64 pipe's peak; DADD..LOG are
 * CUDA's directed intrinsics and exp/log; OWN_* are the directed primitives
 * this library's kernels use (one directed end each, outward widening of
 * exp/log included) and give the cost of each category of ivb_op_counts in
 * DFMA issue slots. Both LOG probes include one round-to-nearest add and both
 * SQRT probes one round-to-nearest multiply. EMU_MUL / EMU_ADD run the
 * integer-pipe emulation of the directed multiply / add (option `emulate`);
 * MIXED_* run half the chains on the FP64 pipe and half emulated, side by
 * side. */
enum {
    IVB_PROBE_DADD = 0, IVB_PROBE_DMUL = 1, IVB_PROBE_DFMA = 2, IVB_PROBE_DDIV = 3,
    IVB_PROBE_DRCP = 4, IVB_PROBE_DSQRT = 5, IVB_PROBE_EXP = 6, IVB_PROBE_LOG = 7,
    IVB_PROBE_OWN_RCP = 8, IVB_PROBE_OWN_DIV = 9, IVB_PROBE_OWN_SQRT = 10,
    IVB_PROBE_OWN_EXP = 11, IVB_PROBE_OWN_LOG = 12, IVB_PROBE_EMU_MUL = 13,
    IVB_PROBE_MIXED_MUL = 14, IVB_PROBE_EMU_ADD = 15, IVB_PROBE_MIXED_ADD = 16
};
ivb_status ivb_fp64_probe(int32_t which, int32_t iters, double* lane_ops_per_s);

/* Test hook: one interval operation of the bounding kernels' own arithmetic
 * (the natural interval extension of an intrinsic, Section 2.2, with this
 * library's outward rounding) on n intervals: x, y, r are DEVICE arrays
 * [n][2]; opcode is a binary or unary tape opcode, IVB_EVAL_RECIP for the
 * interval reciprocal 1/x, IVB_EVAL_EMU_* for +, -, *, sqr with every
 * endpoint operation done by the integer-pipe emulation (option `emulate`),
 * or IVB_EVAL_FMA for r + x*y with one directed rounding per end (the fused
 * accumulation of the adjoint sweep, the tangent rules and the Mean Value
 * Form sum): r holds the addend on entry and the result on return.
 * Enqueued on cuda_stream. */
#define IVB_EVAL_RECIP 100
#define IVB_EVAL_EMU_ADD 101
#define IVB_EVAL_EMU_SUB 102
#define IVB_EVAL_EMU_MUL 103
#define IVB_EVAL_EMU_SQR 104
#define IVB_EVAL_FMA 105
ivb_status ivb_eval_op(int32_t opcode, int64_t n, const double* x, const double* y, double* r,
                       void* cuda_stream);

/* Number of kernel launches the library issued on this handle so far. */
int64_t ivb_launch_count(const ivb_problem* p);

/* Text of the last error on this handle ("" if none); p may be NULL for the
 * last error of ivb_create_problem on this thread. */
const char* ivb_last_error(const ivb_problem* p);

/* Release everything the handle owns; NULL is accepted. */
void ivb_destroy(ivb_problem* p);

#ifdef __cplusplus
}
#endif
#endif
