// ivb_kparams.h -- launch parameters of the bounding kernels, shared by the
// host code, the tape interpreter and the tape-specialised kernels compiled at
// run time (which see this header without the CUDA runtime headers).
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace ivb {

// kernel modes: gradient method x (reduce to node keys | store per subdomain)
enum KernelMode { KM_FWD_REDUCE = 0, KM_ADJ_REDUCE = 1, KM_FWD_STORE = 2, KM_ADJ_STORE = 3 };

// Device node queue, one contiguous buffer written by a single host->device
// copy per call:
//   header   : int64 n_nodes, int64 g_end (end of the global index range)
//              padded to 64 bytes
//   off      : int64 [n_nodes + 1], exclusive prefix sums of subdomain counts
//   records  : n_nodes records of rec_bytes: double lo[n], hi[n], h[n] with
//              h = RN(RN(hi - lo) / N), then int32 N[n]
constexpr int kQueueHeader = 64;

struct ProgDesc;

struct KParams {
    const ProgDesc* prog;  // interpreter only
    const char* queue;     // device node queue (layout above)
    int32_t rec_bytes;
    unsigned long long* counter;   // work counter: first global index to hand out
    int32_t tile;          // subdomains a block takes at a time (multiple of its subdomains per pass)
    // per-thread frames (interpreter only)
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

}  // namespace ivb
