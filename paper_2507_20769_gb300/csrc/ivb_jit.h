// ivb_jit.h -- tape-specialised bounding kernels (generated CUDA C++,
// compiled with NVRTC at problem creation); see ivb_jit.cpp.
//
// Variants of the generated source: compact (the default, option specialize
// = 1) puts the point sweep and each output's adjoint sweeps in __noinline__
// functions and calls the long primitives out of line, which halves the
// compile time at the same speed; specialize = 2 inlines everything. With
// form 1 (the natural interval extension alone) the gradient sweeps are left
// out. Every variant is bit-identical to the interpreter.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ivb_internal.h"
#include "ivb_kparams.h"

namespace ivb {

// generated kernels: __launch_bounds__(kJitBlockMax, kJitMinBlocks), i.e. at
// most 128 registers per thread; specialize = -1 compiles tapes of at most
// kJitAutoMaxOps interval operations per subdomain (beyond that, compile time
// grows to tens of seconds and the interpreter was within 5 % on the
// configurations measured)
constexpr int kJitBlockMax = 256, kJitMinBlocks = 2, kJitAutoMaxOps = 1024;
// endpoint operations emulated on the integer pipes by default (ivb_iv.cuh
// policy bits): none -- on configuration 2 no policy beat the FP64 pipe alone
// by more than the noise (the kernel runs at its 128-register cap with 16
// warps per SM and long dependency chains, so the emulation's latency, not
// the FP64 pipe, ends up on the critical path)
constexpr int kJitDefaultEmulate = 0;

struct JitKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int mode = -1;             // KM_FWD_REDUCE or KM_ADJ_REDUCE
    int block_max = 0;         // __launch_bounds__ of the generated kernel
    int emulate = 0;           // emulation policy compiled in
    bool compact = false;      // long primitives called out of line
    int regs = 0, local_bytes = 0, max_threads = 0;
    double compile_seconds = 0.0;
    // segmented kernels (ivb_jit_seg.cpp): per-thread state area in doubles
    // (0 for the other variants), chunks, state loads and stores and
    // recomputed forward operations per subdomain, recomputation policy
    int state_units = 0, chunks = 0, recompute = -1, ilp = 1;
    long long state_loads = 0, state_stores = 0, recomputed = 0;
    // kernels of the segmented variant for 1, 2 and 4 threads per subdomain
    // (index 0, 1, 2; nullptr where not compiled), without and with the
    // warps of a thread group kept on the same chunk by a barrier
    cudaKernel_t kern_t[3] = {nullptr, nullptr, nullptr};
    cudaKernel_t kern_sync[3] = {nullptr, nullptr, nullptr};
};

// Segmented kernels for large tapes (ivb_jit_seg.cpp): the per-subdomain
// program cut into chunk functions of bounded estimated work, values that
// cross chunks in a per-thread state area, reverse chunks recomputing their
// segment's forward values (policy 0: none, stored; 1: the cheap operations
// + - * sqr neg; 2: all), chunks compiled in `units` parallel NVRTC programs
// and linked with nvJitLink.
struct SegPolicy {
    double chunk_cost = 320.0;   // estimated FP64 issue slots per chunk
    int chunk_stmts = 96;        // statements per chunk
    int recompute = 0;           // measured fastest: recomputation adds FP64 work, the state area streams with room to spare
    int units = 16;
    int max_regs = 128;          // register budget of every chunk function
    int ilp = 1;                 // subdomains per thread (1, or 2 interleaved)
    int outline = 1;             // short interval operations out of line: 0 none, 1 all, 2 products only
};
struct SegSource {
    std::string kernel;               // tile loop, Step 1, chunk calls, Step 3 (one kernel per T)
    std::vector<std::string> units;   // the chunk functions
    std::vector<int> ts;              // threads per subdomain with a kernel: ivb_jit_bound (1), _t2, _t4
    int state_units = 0, chunks = 0, ilp = 1;
    long long loads = 0, stores = 0, recomputed = 0;
    std::string error;                // "" unless the program could not be planned
};
SegSource jit_seg_source(const HostProgram& P, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                         const std::vector<double>& consts, int block_max, int min_blocks, int emulate, int form,
                         const SegPolicy& pol);
// compile the units in parallel and link them; "" on success
std::string jit_seg_compile(const SegSource& src, int max_regs, std::vector<char>& cubin, std::string& tables_name,
                            double* seconds, int* registers, int* spill_bytes);

// CUDA C++ of the reduce-mode bounding kernel for this program; form 1 (the
// natural interval extension alone) leaves out the gradient sweeps
std::string jit_source(const HostProgram& P, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                       const std::vector<double>& consts, int mode, int block_max, int min_blocks, int emulate,
                       bool compact, int form);
// NVRTC for sm_103a; "" on success, else the compiler's message. With
// `registers` / `spill_bytes` non-NULL, ptxas reports them (parsed from its log).
std::string jit_compile(const std::string& src, std::vector<char>& cubin, std::string& tables_name, double* seconds,
                        int* registers, int* spill_bytes);
cudaError_t jit_load(const std::vector<char>& cubin, const std::string& tables_name, JitKernel& K);
// launch / occupancy of the kernel for `tpsub` threads per subdomain (1 for
// every variant but the segmented one)
cudaError_t jit_launch(const JitKernel& K, const KParams& P, int grid, int block, cudaStream_t s, int tpsub = 1,
                       bool sync = false);
int jit_occupancy(const JitKernel& K, int block, int tpsub = 1, bool sync = false);
// index of a threads-per-subdomain value in JitKernel::kern_t (-1 if none)
inline int tpsub_index(int t) { return t == 1 ? 0 : t == 2 ? 1 : t == 4 ? 2 : -1; }
void jit_unload(JitKernel& K);

}  // namespace ivb
