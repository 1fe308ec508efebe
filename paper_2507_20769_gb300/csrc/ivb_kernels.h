// ivb_kernels.h -- launch interface between the C ABI (ivb_api.cu) and the
// kernels (ivb_kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ivb_internal.h"
#include "ivb_kparams.h"

namespace ivb {

// program descriptor, resident in device memory for the life of a problem
struct ProgDesc {
    const Ins* ins;
    const RIns* rins;
    const double* consts;
    int32_t n, n_out, obj, has_eq;
    int32_t pt_begin, pt_count, tan_begin, tan_count;
    uint32_t pt_out_ref[64], pt_out_kind[64];
    uint32_t tan_out_ref[64], tan_out_kind[64];
    AdjProgram adj[64];
    uint8_t out_kind[64];
    FrameLayout L;
};

// node queue record size and buffer size (layout in ivb_kparams.h)
inline int queue_rec_bytes(int n) { return ((28 * n + 7) / 8) * 8; }
inline size_t queue_bytes(int n_nodes, int n) {
    return kQueueHeader + 8 * (size_t)(n_nodes + 1) + (size_t)n_nodes * queue_rec_bytes(n);
}

// node results from the keys
struct FinalizeParams {
    const unsigned long long* keys;
    const char* queue;     // n_nodes is read from the queue header
    int32_t max_nodes, n_out, obj, filter;
    const uint8_t* out_kind;
    double* lb;
    uint8_t* inf;
    double* ub;
    double* minlo;
    double* maxhi;
};

cudaError_t launch_bound(int mode, const KParams& P, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t set_bound_smem_limit(int mode, int bytes);
cudaError_t launch_init_keys(unsigned long long* keys, const char* queue, int max_nodes, int n_out, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeParams& F, cudaStream_t s);
cudaError_t launch_point_grad(const ProgDesc* prog, int n, int n_out, int frame_units, long long n_points,
                              const double* x, double* f, double* grad, double* gframe, int grid, int block,
                              cudaStream_t s);
int occupancy_blocks(int mode, int block, size_t smem);
// fill the exp/log tables of the current device (once per device)
cudaError_t init_math_tables();
// device address and size of this module's exp/log tables (for copies into
// run-time compiled modules)
cudaError_t math_tables_address(void** ptr, size_t* bytes);
// throughput run of one of this library's directed primitives (0 rcp, 1 div,
// 2 sqrt, 3 exp, 4 log) for ivb_fp64_probe
cudaError_t run_own_probe(int which, double* out, int grid, int block, int iters, float* ms);
// one interval operation of the kernels' arithmetic on arrays (test hook)
cudaError_t launch_eval_op(int opcode, long long n, const double* x, const double* y, double* r, cudaStream_t s);

}  // namespace ivb
