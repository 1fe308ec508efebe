// ivb_kernels.h -- launch interface between the C ABI (ivb_api.cu) and the
// kernels (ivb_kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ivb_internal.h"

namespace ivb {

// kernel modes: gradient method x (reduce to node keys | store per subdomain)
enum KernelMode { KM_FWD_REDUCE = 0, KM_ADJ_REDUCE = 1, KM_FWD_STORE = 2, KM_ADJ_STORE = 3 };

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

// Device node queue, one contiguous buffer written by a single host->device
// copy per call:
//   header   : int64 n_nodes, int64 g_end (end of the global index range)
//              padded to 64 bytes
//   off      : int64 [n_nodes + 1], exclusive prefix sums of subdomain counts
//   records  : n_nodes records of rec_bytes: double lo[n], hi[n], h[n] with
//              h = RN(RN(hi - lo) / N), then int32 N[n]
constexpr int kQueueHeader = 64;
inline int queue_rec_bytes(int n) { return ((28 * n + 7) / 8) * 8; }
inline size_t queue_bytes(int n_nodes, int n) {
    return kQueueHeader + 8 * (size_t)(n_nodes + 1) + (size_t)n_nodes * queue_rec_bytes(n);
}

struct KParams {
    const ProgDesc* prog;
    const char* queue;     // device node queue (layout above)
    int32_t rec_bytes;
    unsigned long long* counter;   // work counter: first global index to hand out
    int32_t tile;          // subdomains a block takes at a time (multiple of blockDim)
    // per-thread frames
    double* gframe;        // global frames: frame_units * blockDim per block
    int32_t frame_in_smem;
    int32_t frame_units;
    // results
    unsigned long long* keys;  // [n_nodes][2 n_out + 2]
    double* outF;          // store modes
    double* outFc;
    double* outG;
    long long store_first_g;
    int32_t form;          // 0 MVF, 1 NIE, 2 MVF meet NIE
};

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
// throughput run of one of this library's directed primitives (0 rcp, 1 div,
// 2 sqrt, 3 exp, 4 log) for ivb_fp64_probe
cudaError_t run_own_probe(int which, double* out, int grid, int block, int iters, float* ms);
// one interval operation of the kernels' arithmetic on arrays (test hook)
cudaError_t launch_eval_op(int opcode, long long n, const double* x, const double* y, double* r, cudaStream_t s);

}  // namespace ivb
