// ivb_problem.h -- the problem handle behind the opaque ivb_problem of the
// C ABI, shared by the translation units that implement entry points.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/ivb.h"
#include "ivb_host.h"
#include "ivb_internal.h"
#include "ivb_jit.h"
#include "ivb_kernels.h"

struct ivb_problem {
    ivb_options opt{};
    ivb::HostProgram P{};
    ivb::HostTape host;       // the tape for host-side evaluation (B&B)
    int n = 0, n_out = 0, obj = 0;
    int device = 0;           // the CUDA device current at creation (owns every buffer below)
    uint8_t out_kind[64]{};
    // program on the device
    ivb::ProgDesc* d_prog = nullptr;
    ivb::Ins* d_ins = nullptr;
    ivb::RIns* d_rins = nullptr;
    double* d_consts = nullptr;
    uint8_t* d_out_kind = nullptr;
    // per-call buffers (capacity max_nodes)
    int max_nodes = 0;
    int rec_bytes = 0;
    char* d_queue = nullptr;
    char* h_queue = nullptr;            // pinned staging of the queue
    cudaEvent_t queue_free = nullptr;   // the last copy out of h_queue has completed
    unsigned long long* d_keys = nullptr;
    unsigned long long* d_counter = nullptr;
    double *d_lb = nullptr, *d_ub = nullptr, *d_minlo = nullptr, *d_maxhi = nullptr;
    uint8_t* d_inf = nullptr;
    // frames
    double* d_frame = nullptr;
    size_t frame_bytes = 0;
    // tuning
    int sm_count = 0, smem_optin = 0;
    bool tuned = false;       // final configuration chosen
    bool cfg_ready = false;   // some configuration chosen (defaults while waiting for a batch worth tuning on)
    int block = 128, bps = 4, tile = 512, frame_smem = 0;
    int tpsub = 1;            // threads per subdomain (segmented kernel: 1, 2 or 4)
    bool chunk_sync = false;  // segmented kernel: a group's warps kept on the same chunk
    bool tuned_interp = false;  // the autotuner chose the interpreter over the specialised kernel
    int tune_candidates = 0;  // launch configurations the autotuner timed
    float tune_best_ms = 0.f, tune_worst_ms = 0.f;
    // graph of the batched call
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap_stream = nullptr;
    // point gradients
    double* d_pframe = nullptr;
    size_t pframe_bytes = 0;
    long long launches = 0;
    // tape-specialised reduce kernel (option specialize), unloaded by ivb_destroy
    ivb::JitKernel jit;
    std::string err;
};

// ivb_bound_nodes_ex without the final wait: results reach host buffers
// asynchronously (pinned buffers for true overlap); the caller orders on `s`
ivb_status bound_nodes_enqueue(ivb_problem* p, int32_t n_nodes, const double* boxes, const int32_t* splits,
                               double* out_lb, uint8_t* out_inf, double* out_ub, double* out_minlo,
                               double* out_maxhi, cudaStream_t s);
