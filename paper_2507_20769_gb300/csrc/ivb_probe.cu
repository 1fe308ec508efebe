// ivb_probe.cu -- throughput of the FP64 primitives the bounding kernels use,
// measured on the running GPU (lane operations per second). The DFMA rate is
// the FP64 pipe's peak; the others give each primitive's cost in DFMA issue
// slots for the roofline of the ALU-bound bounding kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ivb.h"
#include "ivb_kernels.h"

namespace {

constexpr int kChains = 8;

template <int W>
__device__ __forceinline__ double step(double x, double y) {
    if (W == IVB_PROBE_DADD) return __dadd_rd(x, y);
    if (W == IVB_PROBE_DMUL) return __dmul_rd(x, y);
    if (W == IVB_PROBE_DFMA) return __fma_rn(x, y, 1e-300);
    if (W == IVB_PROBE_DDIV) return __ddiv_rd(y, x);
    if (W == IVB_PROBE_DRCP) return __drcp_rd(x);
    if (W == IVB_PROBE_DSQRT) return __dsqrt_rd(x * 3.1);   // times one multiply (keeps x off powers of two)
    if (W == IVB_PROBE_EXP) return exp(-x);
    return __dadd_rn(log(x), 2.0);   // IVB_PROBE_LOG: log plus one add (fixed point near 3.15)
}

template <int W>
__global__ void k_probe(double* out, double seed, int iters) {
    double x[kChains];
    const double y = seed + threadIdx.x * 1e-12;
    for (int j = 0; j < kChains; ++j) x[j] = 1.5 + j * 1e-3 + threadIdx.x * 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = step<W>(x[j], y);
    }
    double s = 0.0;
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int W>
cudaError_t run(double* out, int grid, int block, int iters, float* ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_probe<W><<<grid, block>>>(out, 1.0000001, iters / 4 + 1);   // warm-up
    cudaEventRecord(a);
    k_probe<W><<<grid, block>>>(out, 1.0000001, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace

extern "C" ivb_status ivb_fp64_probe(int32_t which, int32_t iters, double* lane_ops_per_s) {
    if (!lane_ops_per_s || iters < 1 || which < 0 || which > IVB_PROBE_MIXED_ADD) return IVB_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IVB_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IVB_ECUDA;
    const int block = 128, grid = sms * 8;   // 32 warps per SM, 8 independent chains each
    double* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * block * sizeof(double)) != cudaSuccess) return IVB_ENOMEM;
    float ms = 0.f;
    cudaError_t e;
    switch (which) {
    case IVB_PROBE_OWN_RCP: case IVB_PROBE_OWN_DIV: case IVB_PROBE_OWN_SQRT: case IVB_PROBE_OWN_EXP:
    case IVB_PROBE_OWN_LOG: case IVB_PROBE_EMU_MUL: case IVB_PROBE_MIXED_MUL: case IVB_PROBE_EMU_ADD:
    case IVB_PROBE_MIXED_ADD:
        e = ivb::run_own_probe(which - IVB_PROBE_OWN_RCP, out, grid, block, iters, &ms);
        break;
    case IVB_PROBE_DADD: e = run<IVB_PROBE_DADD>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_DMUL: e = run<IVB_PROBE_DMUL>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_DFMA: e = run<IVB_PROBE_DFMA>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_DDIV: e = run<IVB_PROBE_DDIV>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_DRCP: e = run<IVB_PROBE_DRCP>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_DSQRT: e = run<IVB_PROBE_DSQRT>(out, grid, block, iters, &ms); break;
    case IVB_PROBE_EXP: e = run<IVB_PROBE_EXP>(out, grid, block, iters, &ms); break;
    default: e = run<IVB_PROBE_LOG>(out, grid, block, iters, &ms); break;
    }
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return IVB_ECUDA;
    *lane_ops_per_s = (double)grid * block * kChains * (double)iters / (ms * 1e-3);
    return IVB_OK;
}
