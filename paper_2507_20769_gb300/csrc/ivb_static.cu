// ivb_static.cu -- ivb_bound_nodes_noalloc: the batched bounding call for
// callers that cannot allocate device memory while they run (for example a
// service whose device memory is reserved up front by another allocator, or a
// loop that must not call cudaMalloc/cudaFree because those calls synchronize
// the device and can fail under memory pressure). The call allocates nothing:
// its working memory -- the node queue, the reduction keys, the work counter and
// an error word -- lives in one file-scope device array of fixed size, and the
// per-thread frames live in shared memory. The caller passes device inputs and
// outputs; the problem handle (created earlier with ivb_create_problem) supplies
// the compiled program.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/ivb.h"
#include "ivb_internal.h"
#include "ivb_kernels.h"
#include "ivb_problem.h"

using namespace ivb;

namespace {

// Fixed scratch, shared by every call on a device (see the header for the
// consequences): node queue for IVB_NOALLOC_MAX_NODES nodes of up to
// IVB_MAX_VARS variables, keys for IVB_MAX_OUTPUTS outputs, counter, error word.
constexpr size_t kQueueCap = kQueueHeader + 8 * (size_t)(IVB_NOALLOC_MAX_NODES + 1) +
                             (size_t)IVB_NOALLOC_MAX_NODES * 896;   // 896 = queue_rec_bytes(IVB_MAX_VARS)
constexpr size_t kKeysOff = (kQueueCap + 255) / 256 * 256;
constexpr size_t kKeysCap = (size_t)IVB_NOALLOC_MAX_NODES * (2 * IVB_MAX_OUTPUTS + 2) * 8;
constexpr size_t kCounterOff = (kKeysOff + kKeysCap + 255) / 256 * 256;
constexpr size_t kErrorOff = kCounterOff + 256;
constexpr size_t kScratchBytes = kErrorOff + 256;
static_assert(kScratchBytes <= 512 * 1024, "no-allocation scratch stays at 512 KiB");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// host-side addresses of g_noalloc_scratch, one per device (set up on the
// first call on that device, with the device current)
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Validate the device-resident boxes and splits and write the node queue
// (same layout as the regular path: header, prefix offsets, records with
// h = RN(RN(hi - lo) / N)). One block; error word = 1 + first bad node.
__global__ void k_prepare_queue(const double* __restrict__ boxes, const int32_t* __restrict__ splits, int n_nodes,
                                int n, int rec_bytes, char* queue, unsigned long long* err) {
    __shared__ long long cnt[IVB_NOALLOC_MAX_NODES];
    char* recs = queue + kQueueHeader + 8 * (size_t)(n_nodes + 1);
    const double lim = 0x1p1000;
    for (int nd = threadIdx.x; nd < n_nodes; nd += blockDim.x) {
        double* lo = reinterpret_cast<double*>(recs + (size_t)nd * rec_bytes);
        double* hi = lo + n;
        double* h = hi + n;
        int32_t* N = reinterpret_cast<int32_t*>(h + n);
        long long c = 1;
        bool bad = false;
        for (int i = 0; i < n; ++i) {
            const double a = boxes[((size_t)nd * n + i) * 2], b = boxes[((size_t)nd * n + i) * 2 + 1];
            const int32_t k = splits[(size_t)nd * n + i];
            if (!(a <= b) || !(fabs(a) <= lim) || !(fabs(b) <= lim) || k < 1) bad = true;
            if (!bad) {
                c *= k;
                if (c > (1LL << 31)) bad = true;
            }
            lo[i] = a;
            hi[i] = b;
            h[i] = bad ? 0.0 : __ddiv_rn(__dsub_rn(b, a), (double)k);
            N[i] = bad ? 1 : k;
        }
        if (bad) {
            // a rejected node becomes the one-subdomain box [0,0]^n, so the
            // kernels that still run on it read finite values only
            for (int i = 0; i < n; ++i) { lo[i] = 0.0; hi[i] = 0.0; h[i] = 0.0; N[i] = 1; }
            atomicMin(err, (unsigned long long)nd + 1);
            c = 1;
        }
        cnt[nd] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long* hdr = reinterpret_cast<long long*>(queue);
        long long* off = reinterpret_cast<long long*>(queue + kQueueHeader);
        long long acc = 0;
        for (int nd = 0; nd < n_nodes; ++nd) { off[nd] = acc; acc += cnt[nd]; }
        off[n_nodes] = acc;
        hdr[0] = n_nodes;
        hdr[1] = acc;
    }
}

ivb_status fail(ivb_problem* p, ivb_status st, const std::string& msg) {
    p->err = msg;
    return st;
}

ivb_status cuda_fail(ivb_problem* p, cudaError_t e, const char* where) {
    return fail(p, IVB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CKN(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, #call);    \
    } while (0)

// device memory of device `dev` (the problem's)
bool on_device(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" ivb_status ivb_bound_nodes_noalloc(ivb_problem* p, int32_t n_nodes, const double* boxes,
                                              const int32_t* splits_per_dim, double* out_lb,
                                              uint8_t* out_infeasible, void* cuda_stream) {
    if (!p) return IVB_EINVAL;
    p->err.clear();
    if (n_nodes < 1 || n_nodes > IVB_NOALLOC_MAX_NODES)
        return fail(p, IVB_EINVAL, "ivb_bound_nodes_noalloc: n_nodes must be in [1, " +
                                       std::to_string(IVB_NOALLOC_MAX_NODES) + "] (fixed scratch capacity)");
    if (!boxes || !splits_per_dim || !out_lb || !out_infeasible)
        return fail(p, IVB_EINVAL, "ivb_bound_nodes_noalloc: all four arrays are required");
    // the problem's program and kernel attributes belong to the device it was created on
    int cur = -1;
    CKN(cudaGetDevice(&cur));
    if (cur != p->device)
        return fail(p, IVB_EINVAL, "ivb_bound_nodes_noalloc: the current device (" + std::to_string(cur) +
                                       ") is not the device the problem was created on (" +
                                       std::to_string(p->device) + ")");
    if (!on_device(boxes, cur) || !on_device(splits_per_dim, cur) || !on_device(out_lb, cur) ||
        !on_device(out_infeasible, cur))
        return fail(p, IVB_EINVAL, "ivb_bound_nodes_noalloc: every array must be device memory of the problem's device");
    const int mode = p->opt.grad_mode == IVB_GRAD_ADJOINT ? KM_ADJ_REDUCE : KM_FWD_REDUCE;
    const int fu = p->opt.grad_mode == IVB_GRAD_ADJOINT ? p->P.L.total_adj : p->P.L.total_fwd;
    // per-thread frames in shared memory: the largest block of 128, 64 or 32 threads that fits
    int block = 0;
    for (int b : {128, 64, 32})
        if ((size_t)b * fu * sizeof(double) + 1024 <= (size_t)p->smem_optin) { block = b; break; }
    if (!block)
        return fail(p, IVB_ENOTSUP, "ivb_bound_nodes_noalloc: the problem's per-thread frame (" +
                                        std::to_string(fu * 8) + " bytes) does not fit in shared memory");
    const size_t smem = (size_t)block * fu * sizeof(double);
    const int bps = occupancy_blocks(mode, block, smem);
    if (bps < 1) return fail(p, IVB_ENOTSUP, "ivb_bound_nodes_noalloc: launch does not fit on an SM");

    // one-time set-up on this device: the device address of the scratch array
    const int dev = cur;
    if (dev < 0 || dev >= kMaxDevices) return fail(p, IVB_ENOTSUP, "ivb_bound_nodes_noalloc: device index too large");
    if (!g_scratch_addr[dev]) {
        void* addr = nullptr;
        CKN(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
        g_scratch_addr[dev] = addr;
    }
    char* base = static_cast<char*>(g_scratch_addr[dev]);
    char* queue = base;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(base + kKeysOff);
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(base + kCounterOff);
    unsigned long long* errw = reinterpret_cast<unsigned long long*>(base + kErrorOff);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // what must start at a fixed value: work counter 0, error word "no error"
    CKN(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    CKN(cudaMemsetAsync(errw, 0xFF, sizeof(unsigned long long), s));
    const int rec = queue_rec_bytes(p->n);
    k_prepare_queue<<<1, 256, 0, s>>>(boxes, splits_per_dim, n_nodes, p->n, rec, queue, errw);
    CKN(cudaGetLastError());
    CKN(launch_init_keys(keys, queue, n_nodes, p->n_out, s));
    KParams K{};
    K.prog = p->d_prog;
    K.queue = queue;
    K.rec_bytes = rec;
    K.counter = counter;
    K.tile = block;   // one subdomain per thread per grab (the smallest tail)
    K.gframe = nullptr;
    K.frame_in_smem = 1;
    K.frame_units = fu;
    K.keys = keys;
    K.form = p->opt.form;
    CKN(launch_bound(mode, K, p->sm_count * bps, block, smem, s));
    FinalizeParams F{};
    F.keys = keys;
    F.queue = queue;
    F.max_nodes = n_nodes;
    F.n_out = p->n_out;
    F.obj = p->obj;
    F.filter = p->opt.filter;
    F.out_kind = p->d_out_kind;
    F.lb = out_lb;
    F.inf = out_infeasible;
    CKN(launch_finalize(F, s));
    p->launches += 4;
    // report invalid nodes: read the error word (a copy into a local, no allocation)
    unsigned long long e = 0;
    CKN(cudaMemcpyAsync(&e, errw, sizeof(e), cudaMemcpyDeviceToHost, s));
    CKN(cudaStreamSynchronize(s));
    if (e != ~0ULL)
        return fail(p, IVB_EINVAL, "ivb_bound_nodes_noalloc: node " + std::to_string(e - 1) +
                                       ": box must be finite with lo <= hi and |endpoint| <= 2^1000, splits >= 1 "
                                       "with product <= 2^31");
    return IVB_OK;
}
