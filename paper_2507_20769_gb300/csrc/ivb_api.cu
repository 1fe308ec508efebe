// ivb_api.cu -- the C ABI declared in include/ivb.h: problem handles, input
// validation, the device node queue, the batched persistent launch replayed as
// a CUDA graph, the plain one-node-per-launch path, the autotuner, per-subdomain
// enclosures and point gradients.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_compile.h"
#include "ivb_internal.h"
#include "ivb_kernels.h"
#include "ivb_problem.h"


using namespace ivb;


namespace {

thread_local std::string g_create_error;

ivb_status fail(ivb_problem* p, ivb_status st, const std::string& msg) {
    if (p) p->err = msg;
    else g_create_error = msg;
    return st;
}

ivb_status cuda_fail(ivb_problem* p, cudaError_t e, const char* where) {
    return fail(p, e == cudaErrorMemoryAllocation ? IVB_ENOMEM : IVB_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(p, e_, #call);    \
    } while (0)

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int kernel_mode(const ivb_problem* p, bool store) {
    const bool adj = p->opt.grad_mode == IVB_GRAD_ADJOINT;
    return store ? (adj ? KM_ADJ_STORE : KM_FWD_STORE) : (adj ? KM_ADJ_REDUCE : KM_FWD_REDUCE);
}

// per-thread frame of the tape interpreter (store modes, and the reduce mode
// when no tape-specialised kernel is loaded)
int frame_units(const ivb_problem* p) {
    return p->opt.grad_mode == IVB_GRAD_ADJOINT ? p->P.L.total_adj : p->P.L.total_fwd;
}

bool use_jit(const ivb_problem* p) { return p->jit.kern != nullptr; }

// the reduce launches run the tape-specialised kernel (loaded, and not
// outtimed by the interpreter in the autotuner)
bool reduce_jit(const ivb_problem* p) { return use_jit(p) && !p->tuned_interp; }

// per-thread units of device memory the reduce kernel needs: the interpreter's
// frame, a segmented kernel's state area, nothing for the other specialised
// kernels (registers only)
int reduce_units(const ivb_problem* p) {
    if (!reduce_jit(p)) return frame_units(p);
    return p->jit.state_units;
}

// Read host or device input arrays into host vectors (device arrays are
// copied synchronously on the stream: validation needs the values).
template <class T>
ivb_status fetch(ivb_problem* p, const T* src, size_t count, std::vector<T>& dst, cudaStream_t s) {
    dst.resize(count);
    if (is_device_ptr(src)) {
        CK(cudaMemcpyAsync(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst.data(), src, count * sizeof(T));
    }
    return IVB_OK;
}

// Validate boxes and splits, write the node queue into the pinned staging
// buffer; returns the queue size in bytes through *bytes.
ivb_status stage_queue(ivb_problem* p, int n_nodes, const double* boxes, const int32_t* splits, long long g_begin,
                       long long g_count, bool enclose, size_t* bytes, long long* total_out, cudaStream_t s) {
    const int n = p->n;
    std::vector<double> B;
    std::vector<int32_t> S;
    ivb_status st = fetch(p, boxes, (size_t)n_nodes * n * 2, B, s);
    if (st) return st;
    st = fetch(p, splits, (size_t)n_nodes * n, S, s);
    if (st) return st;
    // the previous call's copy out of the staging buffer must have finished
    CK(cudaEventSynchronize(p->queue_free));
    char* q = p->h_queue;
    long long* hdr = reinterpret_cast<long long*>(q);
    long long* off = reinterpret_cast<long long*>(q + kQueueHeader);
    char* recs = q + kQueueHeader + 8 * (size_t)(n_nodes + 1);
    long long acc = 0;
    const double lim = std::ldexp(1.0, 1000);
    for (int nd = 0; nd < n_nodes; ++nd) {
        double* lo = reinterpret_cast<double*>(recs + (size_t)nd * p->rec_bytes);
        double* hi = lo + n;
        double* h = hi + n;
        int32_t* N = reinterpret_cast<int32_t*>(h + n);
        long long cnt = 1;
        for (int i = 0; i < n; ++i) {
            const double a = B[((size_t)nd * n + i) * 2], b = B[((size_t)nd * n + i) * 2 + 1];
            const int32_t k = S[(size_t)nd * n + i];
            if (!std::isfinite(a) || !std::isfinite(b) || !(a <= b))
                return fail(p, IVB_EINVAL, "node " + std::to_string(nd) + ": box bounds must be finite with lo <= hi");
            if (std::fabs(a) > lim || std::fabs(b) > lim)
                return fail(p, IVB_EINVAL, "node " + std::to_string(nd) + ": |box endpoint| exceeds 2^1000");
            if (k < 1) return fail(p, IVB_EINVAL, "node " + std::to_string(nd) + ": splits must be >= 1");
            cnt *= k;
            if (cnt > (1LL << 31))
                return fail(p, IVB_EINVAL, "node " + std::to_string(nd) + ": product of splits exceeds 2^31");
            lo[i] = a;
            hi[i] = b;
            h[i] = (b - a) / (double)k;   // RN(RN(hi - lo) / N), as in the subdomain endpoint formula
            N[i] = k;
        }
        off[nd] = acc;
        acc += cnt;
    }
    off[n_nodes] = acc;
    long long g_end = acc;
    if (enclose) {
        if (g_begin < 0 || g_count < 0 || g_begin + g_count > acc)
            return fail(p, IVB_EINVAL, "subdomain range outside the node");
        g_end = g_begin + g_count;
    }
    hdr[0] = n_nodes;
    hdr[1] = g_end;
    *bytes = queue_bytes(n_nodes, n);
    *total_out = g_end;
    return IVB_OK;
}

ivb_status ensure_frame(ivb_problem* p, int grid, int block, int units) {
    const size_t need = (size_t)grid * block * units * sizeof(double);
    if (need <= p->frame_bytes) return IVB_OK;
    if (p->d_frame) cudaFree(p->d_frame);
    p->d_frame = nullptr;
    p->frame_bytes = 0;
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    CK(cudaMalloc(&p->d_frame, need));
    p->frame_bytes = need;
    return IVB_OK;
}

KParams make_params(ivb_problem* p, int frame_smem) {
    KParams K{};
    K.prog = p->d_prog;
    K.queue = p->d_queue;
    K.rec_bytes = p->rec_bytes;
    K.counter = p->d_counter;
    K.tile = p->tile;
    K.gframe = p->d_frame;
    K.frame_in_smem = frame_smem;
    K.frame_units = reduce_units(p);
    K.keys = p->d_keys;
    K.form = p->opt.form;
    return K;
}

size_t smem_bytes(const ivb_problem* p, int block, int frame_smem) {
    return frame_smem ? (size_t)block * frame_units(p) * sizeof(double) : 0;
}

// the reduce-mode bounding kernel: tape-specialised when compiled, else the interpreter
cudaError_t launch_reduce(ivb_problem* p, const KParams& K, int grid, int block, int frame_smem, cudaStream_t s,
                          int tpsub, bool sync) {
    if (reduce_jit(p)) return jit_launch(p->jit, K, grid, block, s, tpsub, sync);
    return launch_bound(kernel_mode(p, false), K, grid, block, smem_bytes(p, block, frame_smem), s);
}

// resident blocks per SM of the reduce kernel
int reduce_occupancy(ivb_problem* p, int block, int frame_smem, int tpsub = 1, bool sync = false) {
    if (reduce_jit(p)) return block <= p->jit.max_threads ? jit_occupancy(p->jit, block, tpsub, sync) : 0;
    return occupancy_blocks(kernel_mode(p, false), block, smem_bytes(p, block, frame_smem));
}

// enqueue: keys, counter, bound kernel, finalize (the batched graph body)
ivb_status enqueue_bound(ivb_problem* p, int grid, int block, int tile, int frame_smem, int max_nodes, cudaStream_t s,
                         int tpsub, bool sync) {
    CK(launch_init_keys(p->d_keys, p->d_queue, max_nodes, p->n_out, s));
    CK(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), s));
    KParams K = make_params(p, frame_smem);
    K.tile = tile;
    CK(launch_reduce(p, K, grid, block, frame_smem, s, tpsub, sync));
    FinalizeParams F{};
    F.keys = p->d_keys;
    F.queue = p->d_queue;
    F.max_nodes = max_nodes;
    F.n_out = p->n_out;
    F.obj = p->obj;
    F.filter = p->opt.filter;
    F.out_kind = p->d_out_kind;
    F.lb = p->d_lb;
    F.inf = p->d_inf;
    F.ub = p->d_ub;
    F.minlo = p->d_minlo;
    F.maxhi = p->d_maxhi;
    CK(launch_finalize(F, s));
    p->launches += 3;
    return IVB_OK;
}

struct TuneCand {
    int block, bps, smem, tpsub, tile_mult;
    bool sync, interp;
};

// subdomains a block covers per pass of its tile loop
int pass_size(const ivb_problem* p, int block, int tpsub) {
    const int ilp = reduce_jit(p) && p->jit.state_units > 0 ? p->jit.ilp : 1;
    return block / std::max(1, tpsub) * ilp;
}

// threads-per-subdomain values the loaded kernel offers (1 unless segmented)
std::vector<int> tpsub_choices(const ivb_problem* p) {
    std::vector<int> v{1};
    if (reduce_jit(p))
        for (int t : {2, 4})
            if (p->jit.kern_t[tpsub_index(t)] && (p->opt.threads_per_subdomain == 0 || p->opt.threads_per_subdomain == t))
                v.push_back(t);
    if (p->opt.threads_per_subdomain > 1 && v.size() > 1) v.erase(v.begin());   // a fixed T > 1 excludes 1
    return v;
}

// chunk synchronisation choices: the segmented kernels come with and without
std::vector<bool> sync_choices(const ivb_problem* p) {
    if (!reduce_jit(p) || !p->jit.kern_sync[0]) return {false};
    if (p->opt.seg_sync == 0) return {false};
    if (p->opt.seg_sync == 1) return {true};
    return {false, true};
}

// Pick block size, blocks per SM, frame placement, threads per subdomain and
// subdomains per grab (tile) by timing the bound kernel on the first
// subdomains of the staged batch (results do not depend on the choice). The
// timed index range is capped at two waves of the widest candidate grid, and a
// candidate whose warm-up is already far slower than the best is not timed
// again, so that tuning stays a small fraction of a few calls. Stage 1 times every
// (threads per subdomain, block, blocks per SM, frame placement); stage 2
// times larger grabs (4 and 16 passes per grab) for the best of stage 1.
ivb_status autotune(ivb_problem* p, long long total, cudaStream_t s) {
    std::vector<TuneCand> cands;
    const int blocks[] = {64, 128, 256};
    const int bpss[] = {1, 2, 3, 4, 6, 8};
    int max_threads = 0;
    // with the library's choice of kernel, the interpreter competes with the
    // tape-specialised kernel; candidates are generated (and timed) with the
    // problem switched to the kernel they use
    std::vector<bool> kernels{false};
    if (use_jit(p) && p->opt.specialize == -1) kernels.push_back(true);
    for (bool ip : kernels) {
    p->tuned_interp = ip;
    for (bool sy : sync_choices(p))
    for (int t : tpsub_choices(p))
        for (int b : blocks)
            for (int k : bpss) {
                const int warps = b * k / 32;
                if (warps < 4 || warps > 32 || b < 32 * t) continue;
                for (int sm = 0; sm < 2; ++sm) {
                    const size_t bytes = smem_bytes(p, b, sm);
                    if (sm && (reduce_jit(p) || bytes + 1024 > (size_t)p->smem_optin || bytes * k > 220 * 1024)) continue;
                    if (p->opt.frame_in_shared == 0 && sm) continue;
                    if (p->opt.frame_in_shared == 1 && !sm && !reduce_jit(p)) continue;
                    if (reduce_occupancy(p, b, sm, t, sy) < k) continue;
                    cands.push_back({b, k, sm, t, 1, sy, ip});
                    max_threads = std::max(max_threads, b * k * p->sm_count);
                }
            }
    }
    p->tuned_interp = false;
    if (cands.empty()) cands.push_back({64, 1, 0, 1, 1, false, false});
    // time only [0, cap) of the global index range: two waves of the widest candidate grid
    const long long cap = std::min<long long>(total, std::max<long long>(2LL * max_threads, 1LL << 18));
    long long* hdr = reinterpret_cast<long long*>(p->h_queue);
    const long long g_end = hdr[1];
    CK(cudaEventSynchronize(p->queue_free));
    hdr[1] = cap;
    CK(cudaMemcpyAsync(p->d_queue, p->h_queue, 16, cudaMemcpyHostToDevice, s));
    cudaEvent_t ew, e0, e1;
    CK(cudaEventCreate(&ew));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f, worst = 0.f;
    TuneCand bc = cands[0];
    ivb_status st = IVB_OK;
    int timed = 0;
    auto time_one = [&](const TuneCand& c) -> ivb_status {
        const int grid = p->sm_count * c.bps;
        p->tuned_interp = c.interp;
        ivb_status r = IVB_OK;
        if (reduce_units(p) > 0) r = ensure_frame(p, grid, c.block, reduce_units(p));
        if (r) return r;
        const int tile = c.tile_mult * pass_size(p, c.block, c.tpsub);
        // warm-up run, timed too: a candidate whose warm-up already takes 1.5x the
        // best time so far is not run again (its warm-up time stands)
        CK(cudaEventRecord(ew, s));
        r = enqueue_bound(p, grid, c.block, tile, c.smem, p->max_nodes, s, c.tpsub, c.sync);
        if (r) return r;
        CK(cudaEventRecord(e0, s));
        CK(cudaEventSynchronize(e0));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ew, e0));
        if (!(best < 1e29f && ms > 1.5f * best)) {
            r = enqueue_bound(p, grid, c.block, tile, c.smem, p->max_nodes, s, c.tpsub, c.sync);
            if (r) return r;
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
        }
        ++timed;
        worst = std::max(worst, ms);
        if (ms < best) { best = ms; bc = c; }
        return IVB_OK;
    };
    for (const TuneCand& c : cands) {
        st = time_one(c);
        if (st) break;
    }
    if (!st && p->opt.tile <= 0) {
        const TuneCand base = bc;
        for (int mult : {4, 16}) {
            TuneCand c = base;
            c.tile_mult = mult;
            st = time_one(c);
            if (st) break;
        }
    }
    p->tuned_interp = false;
    cudaEventDestroy(ew);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the batch's index range
    hdr[1] = g_end;
    CK(cudaMemcpyAsync(p->d_queue, p->h_queue, 16, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    if (st) return st;
    p->block = bc.block;
    p->bps = bc.bps;
    p->frame_smem = bc.smem;
    p->tpsub = bc.tpsub;
    p->chunk_sync = bc.sync;
    p->tuned_interp = bc.interp;
    p->tile = bc.tile_mult * pass_size(p, bc.block, bc.tpsub);
    p->tune_candidates = timed;
    p->tune_best_ms = best;
    p->tune_worst_ms = worst;
    p->tuned = true;
    p->cfg_ready = true;
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    return IVB_OK;
}

ivb_status default_tuning(ivb_problem* p) {
    p->block = p->opt.block_threads > 0 ? p->opt.block_threads : 128;
    p->bps = p->opt.blocks_per_sm > 0 ? p->opt.blocks_per_sm : 4;
    const size_t bytes = smem_bytes(p, p->block, 1);
    if (reduce_jit(p)) p->frame_smem = 0;   // frames serve only the interpreter's store mode
    else if (p->opt.frame_in_shared == 1) p->frame_smem = 1;
    else if (p->opt.frame_in_shared == 0) p->frame_smem = 0;
    else p->frame_smem = (bytes + 1024 <= (size_t)p->smem_optin && bytes * p->bps <= 220 * 1024) ? 1 : 0;
    p->tpsub = tpsub_choices(p).front();
    if (p->block < 32 * p->tpsub) p->tpsub = 1;
    p->chunk_sync = sync_choices(p).front();
    const int occ = reduce_occupancy(p, p->block, p->frame_smem, p->tpsub, p->chunk_sync);
    if (occ < 1) return fail(p, IVB_ENOTSUP, "launch configuration does not fit on an SM");
    if (p->bps > occ) p->bps = occ;
    const int per = pass_size(p, p->block, p->tpsub);
    p->tile = p->opt.tile > 0 ? ((p->opt.tile + per - 1) / per) * per : per;
    p->cfg_ready = true;
    const bool explicit_cfg = p->opt.block_threads > 0 || p->opt.blocks_per_sm > 0;
    if (!p->opt.autotune || explicit_cfg) p->tuned = true;
    return IVB_OK;
}

// copy node results to the caller (device -> device or device -> host)
ivb_status deliver(ivb_problem* p, int n_nodes, double* out_lb, uint8_t* out_inf, double* out_ub, double* out_minlo,
                   double* out_maxhi, cudaStream_t s, bool* host_out) {
    struct Item { void* dst; const void* src; size_t bytes; };
    const Item items[] = {
        {out_lb, p->d_lb, (size_t)n_nodes * sizeof(double)},
        {out_inf, p->d_inf, (size_t)n_nodes},
        {out_ub, p->d_ub, (size_t)n_nodes * sizeof(double)},
        {out_minlo, p->d_minlo, (size_t)n_nodes * p->n_out * sizeof(double)},
        {out_maxhi, p->d_maxhi, (size_t)n_nodes * p->n_out * sizeof(double)},
    };
    for (const Item& it : items) {
        if (!it.dst) continue;
        const bool dev = is_device_ptr(it.dst);
        if (!dev) *host_out = true;
        CK(cudaMemcpyAsync(it.dst, it.src, it.bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    return IVB_OK;
}

}  // namespace

// ======================================================================= ABI

// generate, compile and load the tape-specialised reduce kernel
// segmentation options of a problem
SegPolicy seg_policy(const ivb_options& o) {
    SegPolicy pol;
    if (o.recompute >= 0) pol.recompute = o.recompute;
    if (o.seg_chunk > 0) pol.chunk_cost = o.seg_chunk;
    if (o.seg_ilp > 0) pol.ilp = o.seg_ilp;
    pol.outline = o.seg_outline < 0 ? 1 : o.seg_outline;   // -1: the library's choice, all out of line
    if (o.seg_regs > 0) pol.max_regs = o.seg_regs;
    const unsigned hc = std::thread::hardware_concurrency();
    pol.units = std::max(1, std::min(64, hc ? (int)hc : 8));
    return pol;
}

// blocks of kJitBlockMax threads per SM that a register budget allows
int seg_min_blocks(int max_regs) { return std::max(1, std::min(8, 65536 / (kJitBlockMax * max_regs))); }

cudaError_t specialize_seg(ivb_problem* p, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                           const std::vector<double>& consts, std::string* msg) {
    const int emu = p->opt.emulate >= 0 ? p->opt.emulate : kJitDefaultEmulate;
    const SegPolicy pol = seg_policy(p->opt);
    const SegSource src = jit_seg_source(p->P, ins, rins, consts, kJitBlockMax, seg_min_blocks(pol.max_regs), emu,
                                         p->opt.form, pol);
    std::vector<char> cubin;
    std::string tables;
    double secs = 0.0;
    *msg = jit_seg_compile(src, pol.max_regs, cubin, tables, &secs, nullptr, nullptr);
    if (!msg->empty()) return cudaSuccess;
    cudaError_t ce = jit_load(cubin, tables, p->jit);
    if (ce != cudaSuccess) return ce;
    p->jit.kern_t[0] = p->jit.kern;
    for (int t : src.ts) {
        const std::string name = "ivb_jit_bound_t" + std::to_string(t);
        if (t > 1) {
            ce = cudaLibraryGetKernel(&p->jit.kern_t[tpsub_index(t)], p->jit.lib, name.c_str());
            if (ce != cudaSuccess) return ce;
        }
        ce = cudaLibraryGetKernel(&p->jit.kern_sync[tpsub_index(t)], p->jit.lib, (name + "_sync").c_str());
        if (ce != cudaSuccess) return ce;
    }
    p->jit.mode = KM_ADJ_REDUCE;
    p->jit.emulate = emu;
    p->jit.compact = true;
    p->jit.block_max = kJitBlockMax;
    p->jit.compile_seconds = secs;
    p->jit.state_units = src.state_units;
    p->jit.chunks = src.chunks;
    p->jit.state_loads = src.loads;
    p->jit.state_stores = src.stores;
    p->jit.recomputed = src.recomputed;
    p->jit.recompute = pol.recompute;
    p->jit.ilp = src.ilp;
    return cudaSuccess;
}

cudaError_t specialize(ivb_problem* p, const std::vector<Ins>& ins, const std::vector<RIns>& rins,
                       const std::vector<double>& consts, int mode, std::string* msg) {
    const int emu = p->opt.emulate >= 0 ? p->opt.emulate : kJitDefaultEmulate;
    const bool compact = p->opt.specialize != 2;
    const std::string src =
        jit_source(p->P, ins, rins, consts, mode, kJitBlockMax, kJitMinBlocks, emu, compact, p->opt.form);
    std::vector<char> cubin;
    std::string tables;
    double secs = 0.0;
    *msg = jit_compile(src, cubin, tables, &secs, nullptr, nullptr);
    if (!msg->empty()) return cudaSuccess;
    const cudaError_t ce = jit_load(cubin, tables, p->jit);
    if (ce != cudaSuccess) return ce;
    p->jit.mode = mode;
    p->jit.emulate = emu;
    p->jit.compact = compact;
    p->jit.block_max = kJitBlockMax;
    p->jit.compile_seconds = secs;
    return cudaSuccess;
}

extern "C" void ivb_options_default(ivb_options* o) {
    if (!o) return;
    o->grad_mode = IVB_GRAD_ADJOINT;
    o->form = IVB_FORM_MVF;
    o->filter = 0;
    o->batched = 1;
    o->use_graph = 1;
    o->autotune = 1;
    o->block_threads = 0;
    o->blocks_per_sm = 0;
    o->tile = 0;
    o->max_nodes = 4096;
    o->frame_in_shared = -1;
    o->specialize = 0;
    o->emulate = -1;
    o->recompute = -1;
    o->seg_chunk = 0;
    o->seg_regs = 0;
    o->threads_per_subdomain = 0;
    o->seg_sync = -1;
    o->seg_ilp = 0;
    o->seg_outline = -1;
}

extern "C" ivb_status ivb_create_problem(const ivb_tape* tape, const ivb_options* opt, ivb_problem** out) {
    if (!out) return fail(nullptr, IVB_EINVAL, "out is NULL");
    *out = nullptr;
    std::string e = validate_tape(tape);
    if (!e.empty()) return fail(nullptr, IVB_ETAPE, e);
    ivb_options o;
    ivb_options_default(&o);
    if (opt) o = *opt;
    if (o.grad_mode != IVB_GRAD_FORWARD && o.grad_mode != IVB_GRAD_ADJOINT)
        return fail(nullptr, IVB_EINVAL, "grad_mode must be IVB_GRAD_FORWARD or IVB_GRAD_ADJOINT");
    if (o.form < 0 || o.form > 2) return fail(nullptr, IVB_EINVAL, "form must be 0, 1 or 2");
    if (o.max_nodes < 1 || o.max_nodes > (1 << 20)) return fail(nullptr, IVB_EINVAL, "max_nodes must be in [1, 2^20]");
    if (o.block_threads < 0 || o.block_threads > 512 || (o.block_threads % 32))
        return fail(nullptr, IVB_EINVAL, "block_threads must be a multiple of 32 up to 512 (0 = auto)");
    if (o.specialize < -1 || o.specialize > 3) return fail(nullptr, IVB_EINVAL, "specialize must be -1, 0, 1, 2 or 3");
    if (o.specialize == 3 && o.grad_mode != IVB_GRAD_ADJOINT)
        return fail(nullptr, IVB_EINVAL, "specialize = 3 (segmented) needs grad_mode IVB_GRAD_ADJOINT");
    if (o.recompute < -1 || o.recompute > 2) return fail(nullptr, IVB_EINVAL, "recompute must be -1, 0, 1 or 2");
    if (o.seg_chunk < 0 || o.seg_chunk > 100000) return fail(nullptr, IVB_EINVAL, "seg_chunk must be in [0, 100000]");
    if (o.threads_per_subdomain != 0 && o.threads_per_subdomain != 1 && o.threads_per_subdomain != 2 &&
        o.threads_per_subdomain != 4)
        return fail(nullptr, IVB_EINVAL, "threads_per_subdomain must be 0 (tuned), 1, 2 or 4");
    if (o.seg_sync < -1 || o.seg_sync > 1) return fail(nullptr, IVB_EINVAL, "seg_sync must be -1, 0 or 1");
    if (o.seg_ilp < 0 || o.seg_ilp > 2) return fail(nullptr, IVB_EINVAL, "seg_ilp must be 0, 1 or 2");
    if (o.seg_outline < -1 || o.seg_outline > 2) return fail(nullptr, IVB_EINVAL, "seg_outline must be -1, 0, 1 or 2");
    if (o.seg_regs != 0 && (o.seg_regs < 64 || o.seg_regs > 255))
        return fail(nullptr, IVB_EINVAL, "seg_regs must be 0 or in [64, 255]");
    if (o.emulate < -1 || o.emulate > 15) return fail(nullptr, IVB_EINVAL, "emulate must be -1 or a bitmask in [0, 15]");
    if (o.specialize && o.block_threads > kJitBlockMax)
        return fail(nullptr, IVB_EINVAL, "block_threads above 256 with a tape-specialised kernel");
    ivb_problem* p = new ivb_problem();
    p->opt = o;
    std::vector<Ins> ins;
    std::vector<RIns> rins;
    std::vector<double> consts;
    e = compile_tape(tape, p->P, ins, rins, consts);
    if (!e.empty()) { delete p; return fail(nullptr, IVB_ENOTSUP, e); }
    p->n = tape->n_vars;
    p->n_out = tape->n_outputs;
    p->obj = p->P.obj;
    for (int i = 0; i < p->n_out; ++i) p->out_kind[i] = tape->out_kind[i];
    p->max_nodes = o.max_nodes;
    p->rec_bytes = queue_rec_bytes(p->n);
    host_tape(tape, p->host);

    auto bail = [&](cudaError_t ce, const char* where) {
        std::string m = std::string(where) + ": " + cudaGetErrorString(ce);
        ivb_destroy(p);
        return fail(nullptr, ce == cudaErrorMemoryAllocation ? IVB_ENOMEM : IVB_ECUDA, m);
    };
#define CKC(call)                                   \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return bail(e_, #call); \
    } while (0)
    int dev = 0;
    CKC(cudaGetDevice(&dev));
    p->device = dev;
    CKC(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev));
    CKC(cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (int m = 0; m < 4; ++m) CKC(set_bound_smem_limit(m, p->smem_optin - 1024));
    CKC(init_math_tables());

    CKC(cudaMalloc(&p->d_ins, std::max<size_t>(1, ins.size()) * sizeof(Ins)));
    CKC(cudaMalloc(&p->d_rins, std::max<size_t>(1, rins.size()) * sizeof(RIns)));
    CKC(cudaMalloc(&p->d_consts, std::max<size_t>(1, consts.size()) * sizeof(double)));
    if (!ins.empty()) CKC(cudaMemcpy(p->d_ins, ins.data(), ins.size() * sizeof(Ins), cudaMemcpyHostToDevice));
    if (!rins.empty()) CKC(cudaMemcpy(p->d_rins, rins.data(), rins.size() * sizeof(RIns), cudaMemcpyHostToDevice));
    if (!consts.empty())
        CKC(cudaMemcpy(p->d_consts, consts.data(), consts.size() * sizeof(double), cudaMemcpyHostToDevice));
    ProgDesc D{};
    D.ins = p->d_ins;
    D.rins = p->d_rins;
    D.consts = p->d_consts;
    D.n = p->n;
    D.n_out = p->n_out;
    D.obj = p->obj;
    D.has_eq = p->P.has_eq;
    D.pt_begin = p->P.pt_begin;
    D.pt_count = p->P.pt_count;
    D.tan_begin = p->P.tan_begin;
    D.tan_count = p->P.tan_count;
    for (int i = 0; i < p->n_out; ++i) {
        D.pt_out_ref[i] = (uint32_t)p->P.pt_out_ref[i];
        D.pt_out_kind[i] = (uint32_t)p->P.pt_out_kind[i];
        D.tan_out_ref[i] = (uint32_t)p->P.tan_out_ref[i];
        D.tan_out_kind[i] = (uint32_t)p->P.tan_out_kind[i];
        D.adj[i] = p->P.adj[i];
        D.out_kind[i] = p->out_kind[i];
    }
    D.L = p->P.L;
    CKC(cudaMalloc(&p->d_prog, sizeof(ProgDesc)));
    CKC(cudaMemcpy(p->d_prog, &D, sizeof(ProgDesc), cudaMemcpyHostToDevice));
    CKC(cudaMalloc(&p->d_out_kind, 64));
    CKC(cudaMemcpy(p->d_out_kind, p->out_kind, 64, cudaMemcpyHostToDevice));

    const size_t qb = queue_bytes(p->max_nodes, p->n);
    CKC(cudaMalloc(&p->d_queue, qb));
    CKC(cudaMallocHost(&p->h_queue, qb));
    CKC(cudaEventCreateWithFlags(&p->queue_free, cudaEventDisableTiming));
    CKC(cudaEventRecord(p->queue_free, 0));
    CKC(cudaMalloc(&p->d_keys, (size_t)p->max_nodes * (2 * p->n_out + 2) * sizeof(unsigned long long)));
    CKC(cudaMalloc(&p->d_counter, sizeof(unsigned long long)));
    CKC(cudaMalloc(&p->d_lb, (size_t)p->max_nodes * sizeof(double)));
    CKC(cudaMalloc(&p->d_ub, (size_t)p->max_nodes * sizeof(double)));
    CKC(cudaMalloc(&p->d_inf, (size_t)p->max_nodes));
    CKC(cudaMalloc(&p->d_minlo, (size_t)p->max_nodes * p->n_out * sizeof(double)));
    CKC(cudaMalloc(&p->d_maxhi, (size_t)p->max_nodes * p->n_out * sizeof(double)));
    CKC(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    if (o.specialize) {
        const int64_t* cnt = o.grad_mode == IVB_GRAD_ADJOINT ? p->P.cnt_adj : p->P.cnt_fwd;
        long long ops = 0;
        for (int k = 0; k < IVB_CNT_N; ++k) ops += cnt[k];
        const bool small = ops / 2 <= kJitAutoMaxOps;
        const bool seg = o.specialize == 3 || (o.specialize == -1 && !small && o.grad_mode == IVB_GRAD_ADJOINT);
        if (o.specialize >= 1 || small || seg) {
            const int mode = o.grad_mode == IVB_GRAD_ADJOINT ? KM_ADJ_REDUCE : KM_FWD_REDUCE;
            std::string msg;
            const cudaError_t ce = seg ? specialize_seg(p, ins, rins, consts, &msg)
                                       : specialize(p, ins, rins, consts, mode, &msg);
            if (ce != cudaSuccess || !msg.empty()) {
                jit_unload(p->jit);
                if (o.specialize >= 1) {
                    ivb_destroy(p);
                    if (ce != cudaSuccess)
                        return fail(nullptr, ce == cudaErrorMemoryAllocation ? IVB_ENOMEM : IVB_ECUDA,
                                    std::string("loading the tape-specialised kernel: ") + cudaGetErrorString(ce));
                    return fail(nullptr, IVB_ENOTSUP, msg);
                }
                cudaGetLastError();
            }
        }
    }
#undef CKC
    *out = p;
    return IVB_OK;
}

namespace {
ivb_status bound_nodes_impl(ivb_problem* p, int32_t n_nodes, const double* boxes, const int32_t* splits_per_dim,
                            double* out_lb, uint8_t* out_infeasible, double* out_ub, double* out_minlo,
                            double* out_maxhi, cudaStream_t s, bool wait_host);
}  // namespace

extern "C" ivb_status ivb_bound_nodes_ex(ivb_problem* p, int32_t n_nodes, const double* boxes,
                                         const int32_t* splits_per_dim, double* out_lb, uint8_t* out_infeasible,
                                         double* out_ub, double* out_minlo, double* out_maxhi, void* cuda_stream) {
    return bound_nodes_impl(p, n_nodes, boxes, splits_per_dim, out_lb, out_infeasible, out_ub, out_minlo, out_maxhi,
                            (cudaStream_t)cuda_stream, true);
}

ivb_status bound_nodes_enqueue(ivb_problem* p, int32_t n_nodes, const double* boxes, const int32_t* splits,
                               double* out_lb, uint8_t* out_inf, double* out_ub, double* out_minlo,
                               double* out_maxhi, cudaStream_t s) {
    return bound_nodes_impl(p, n_nodes, boxes, splits, out_lb, out_inf, out_ub, out_minlo, out_maxhi, s, false);
}

namespace {
ivb_status bound_nodes_impl(ivb_problem* p, int32_t n_nodes, const double* boxes, const int32_t* splits_per_dim,
                            double* out_lb, uint8_t* out_infeasible, double* out_ub, double* out_minlo,
                            double* out_maxhi, cudaStream_t s, bool wait_host) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    p->err.clear();
    if (n_nodes == 0) return IVB_OK;   // empty batch: nothing to bound
    if (n_nodes < 0 || n_nodes > p->max_nodes)
        return fail(p, IVB_EINVAL, "n_nodes must be in [0, max_nodes]");
    if (!boxes || !splits_per_dim) return fail(p, IVB_EINVAL, "boxes and splits_per_dim must not be NULL");
    size_t qbytes = 0;
    long long total = 0;
    ivb_status st = stage_queue(p, n_nodes, boxes, splits_per_dim, 0, 0, false, &qbytes, &total, s);
    if (st) return st;
    bool host_out = false;

    if (!p->opt.batched) {
        // plain path: one node per launch, node queue of one record each
        if (!p->cfg_ready) { st = default_tuning(p); if (st) return st; }
        const int n = p->n;
        std::vector<char> one(queue_bytes(1, n));
        const char* q = p->h_queue;
        const long long* off = reinterpret_cast<const long long*>(q + kQueueHeader);
        const char* recs = q + kQueueHeader + 8 * (size_t)(n_nodes + 1);
        for (int nd = 0; nd < n_nodes; ++nd) {
            // build a one-node queue in place at the front of the device buffer
            long long hdr[2] = {1, off[nd + 1] - off[nd]};
            long long o2[2] = {0, off[nd + 1] - off[nd]};
            std::memset(one.data(), 0, kQueueHeader);
            std::memcpy(one.data(), hdr, sizeof(hdr));
            std::memcpy(one.data() + kQueueHeader, o2, sizeof(o2));
            std::memcpy(one.data() + kQueueHeader + 16, recs + (size_t)nd * p->rec_bytes, p->rec_bytes);
            CK(cudaMemcpyAsync(p->d_queue, one.data(), one.size(), cudaMemcpyHostToDevice, s));
            const long long S = o2[1];
            const long long tiles = (S + p->block - 1) / p->block;
            const int grid = (int)std::min<long long>(tiles, (long long)p->sm_count * p->bps);
            if (reduce_units(p) > 0) st = ensure_frame(p, grid, p->block, reduce_units(p));
            if (st) return st;
            CK(launch_init_keys(p->d_keys, p->d_queue, 1, p->n_out, s));
            CK(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), s));
            KParams K = make_params(p, p->frame_smem);
            K.tile = pass_size(p, p->block, p->tpsub);
            CK(launch_reduce(p, K, grid, p->block, p->frame_smem, s, p->tpsub, p->chunk_sync));
            FinalizeParams F{};
            F.keys = p->d_keys; F.queue = p->d_queue; F.max_nodes = 1; F.n_out = p->n_out; F.obj = p->obj;
            F.filter = p->opt.filter; F.out_kind = p->d_out_kind;
            F.lb = p->d_lb + nd; F.inf = p->d_inf + nd; F.ub = p->d_ub + nd;
            F.minlo = p->d_minlo + (size_t)nd * p->n_out; F.maxhi = p->d_maxhi + (size_t)nd * p->n_out;
            CK(launch_finalize(F, s));
            p->launches += 3;
            // the host buffer `one` is reused: wait for this node's copy
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaEventRecord(p->queue_free, s));
    } else {
        CK(cudaMemcpyAsync(p->d_queue, p->h_queue, qbytes, cudaMemcpyHostToDevice, s));
        CK(cudaEventRecord(p->queue_free, s));
        if (!p->tuned) {
            // tune on the first batch with enough work to time; defaults until then
            const bool explicit_cfg = p->opt.block_threads > 0 || p->opt.blocks_per_sm > 0;
            if (p->opt.autotune && !explicit_cfg && total >= (1LL << 18)) st = autotune(p, total, s);
            else if (!p->cfg_ready) st = default_tuning(p);
            if (st) return st;
        }
        const int grid = p->sm_count * p->bps;
        if (reduce_units(p) > 0) st = ensure_frame(p, grid, p->block, reduce_units(p));
        if (st) return st;
        if (p->opt.use_graph) {
            if (!p->gexec) {
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
                st = enqueue_bound(p, grid, p->block, p->tile, p->frame_smem, p->max_nodes, p->cap_stream, p->tpsub,
                                   p->chunk_sync);
                cudaGraph_t gg = nullptr;
                cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &gg);
                if (st) { if (gg) cudaGraphDestroy(gg); return st; }
                if (ce != cudaSuccess) return cuda_fail(p, ce, "cudaStreamEndCapture");
                g = gg;
                ce = cudaGraphInstantiate(&p->gexec, g, 0);
                cudaGraphDestroy(g);
                if (ce != cudaSuccess) { p->gexec = nullptr; return cuda_fail(p, ce, "cudaGraphInstantiate"); }
                p->launches -= 3;   // captured, not launched
            }
            CK(cudaGraphLaunch(p->gexec, s));
            p->launches += 3;
        } else {
            st = enqueue_bound(p, grid, p->block, p->tile, p->frame_smem, p->max_nodes, s, p->tpsub, p->chunk_sync);
            if (st) return st;
        }
    }
    st = deliver(p, n_nodes, out_lb, out_infeasible, out_ub, out_minlo, out_maxhi, s, &host_out);
    if (st) return st;
    if (host_out && wait_host) CK(cudaStreamSynchronize(s));
    return IVB_OK;
}
}  // namespace

extern "C" ivb_status ivb_bound_nodes(ivb_problem* p, int32_t n_nodes, const double* boxes,
                                      const int32_t* splits_per_dim, double* out_lb, uint8_t* out_infeasible,
                                      void* cuda_stream) {
    return ivb_bound_nodes_ex(p, n_nodes, boxes, splits_per_dim, out_lb, out_infeasible, nullptr, nullptr, nullptr,
                              cuda_stream);
}

extern "C" ivb_status ivb_enclose(ivb_problem* p, const double* box, const int32_t* splits_per_dim, int64_t first,
                                  int64_t count, double* out_F, double* out_Fc, double* out_G, void* cuda_stream) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    p->err.clear();
    if (!box || !splits_per_dim || !out_F) return fail(p, IVB_EINVAL, "box, splits and out_F must not be NULL");
    if (count < 1 || count > (1LL << 24)) return fail(p, IVB_EINVAL, "count must be in [1, 2^24]");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    size_t qbytes = 0;
    long long total = 0;
    ivb_status st = stage_queue(p, 1, box, splits_per_dim, first, count, true, &qbytes, &total, s);
    if (st) return st;
    if (!p->cfg_ready) { st = default_tuning(p); if (st) return st; }
    CK(cudaMemcpyAsync(p->d_queue, p->h_queue, qbytes, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(p->queue_free, s));
    const int n_out = p->n_out, n = p->n;
    const size_t fb = (size_t)count * n_out * 2 * sizeof(double), gb = fb * n;
    // outputs: written directly when device pointers, else through device temporaries
    const bool dF = is_device_ptr(out_F), dFc = out_Fc && is_device_ptr(out_Fc), dG = out_G && is_device_ptr(out_G);
    double *tF = nullptr, *tFc = nullptr, *tG = nullptr;
    if (!dF) CK(cudaMallocAsync(&tF, fb, s));
    if (out_Fc && !dFc) CK(cudaMallocAsync(&tFc, fb, s));
    if (out_G && !dG) CK(cudaMallocAsync(&tG, gb, s));
    const unsigned long long first_u = (unsigned long long)first;
    CK(cudaMemcpyAsync(p->d_counter, &first_u, sizeof(first_u), cudaMemcpyHostToDevice, s));
    const long long tiles = (count + p->block - 1) / p->block;
    const int grid = (int)std::min<long long>(tiles, (long long)p->sm_count * p->bps);
    st = ensure_frame(p, grid, p->block, frame_units(p));
    if (st) return st;
    KParams K = make_params(p, p->frame_smem);
    K.frame_units = frame_units(p);
    K.tile = p->block;
    K.outF = dF ? out_F : tF;
    K.outFc = out_Fc ? (dFc ? out_Fc : tFc) : nullptr;
    K.outG = out_G ? (dG ? out_G : tG) : nullptr;
    K.store_first_g = first;
    CK(launch_bound(kernel_mode(p, true), K, grid, p->block, smem_bytes(p, p->block, p->frame_smem), s));
    p->launches += 1;
    if (!dF) CK(cudaMemcpyAsync(out_F, tF, fb, cudaMemcpyDeviceToHost, s));
    if (out_Fc && !dFc) CK(cudaMemcpyAsync(out_Fc, tFc, fb, cudaMemcpyDeviceToHost, s));
    if (out_G && !dG) CK(cudaMemcpyAsync(out_G, tG, gb, cudaMemcpyDeviceToHost, s));
    if (tF) CK(cudaFreeAsync(tF, s));
    if (tFc) CK(cudaFreeAsync(tFc, s));
    if (tG) CK(cudaFreeAsync(tG, s));
    // the counter copy reads the stack variable first_u: wait before returning
    CK(cudaStreamSynchronize(s));
    return IVB_OK;
}

extern "C" ivb_status ivb_point_grad(ivb_problem* p, int64_t n_points, const double* x, double* out_f,
                                     double* out_grad, void* cuda_stream) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    p->err.clear();
    if (n_points < 1 || !x || !out_f) return fail(p, IVB_EINVAL, "n_points >= 1, x and out_f are required");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int n = p->n, n_out = p->n_out;
    const bool dx = is_device_ptr(x), df = is_device_ptr(out_f), dg = out_grad && is_device_ptr(out_grad);
    const size_t xb = (size_t)n_points * n * sizeof(double), fb = (size_t)n_points * n_out * sizeof(double),
                 gb = fb * n;
    double *tx = nullptr, *tf = nullptr, *tg = nullptr;
    if (!dx) { CK(cudaMallocAsync(&tx, xb, s)); CK(cudaMemcpyAsync(tx, x, xb, cudaMemcpyHostToDevice, s)); }
    if (!df) CK(cudaMallocAsync(&tf, fb, s));
    if (out_grad && !dg) CK(cudaMallocAsync(&tg, gb, s));
    int units = 0;
    for (int o = 0; o < n_out; ++o)
        units = std::max(units, n + p->P.adj[o].adj_slots + p->P.adj[o].tape_records);
    const int block = 128;
    const int grid = (int)std::min<long long>((n_points + block - 1) / block, (long long)p->sm_count * 8);
    const size_t need = (size_t)grid * block * std::max(units, 1) * sizeof(double);
    if (need > p->pframe_bytes) {
        if (p->d_pframe) CK(cudaFree(p->d_pframe));
        p->d_pframe = nullptr;
        p->pframe_bytes = 0;
        CK(cudaMalloc(&p->d_pframe, need));
        p->pframe_bytes = need;
    }
    CK(launch_point_grad(p->d_prog, n, n_out, std::max(units, 1), n_points, dx ? x : tx, df ? out_f : tf,
                         out_grad ? (dg ? out_grad : tg) : nullptr, p->d_pframe, grid, block, s));
    p->launches += 1;
    if (!df) CK(cudaMemcpyAsync(out_f, tf, fb, cudaMemcpyDeviceToHost, s));
    if (out_grad && !dg) CK(cudaMemcpyAsync(out_grad, tg, gb, cudaMemcpyDeviceToHost, s));
    if (tx) CK(cudaFreeAsync(tx, s));
    if (tf) CK(cudaFreeAsync(tf, s));
    if (tg) CK(cudaFreeAsync(tg, s));
    if (!dx || !df || (out_grad && !dg)) CK(cudaStreamSynchronize(s));
    return IVB_OK;
}

extern "C" ivb_status ivb_pick_splits(int32_t n, const double* box, const double* ref_widths, int64_t target,
                                      int32_t strategy, int32_t* out) {
    if (n < 1 || n > IVB_MAX_VARS || !box || !out || target < 1)
        return fail(nullptr, IVB_EINVAL, "pick_splits: n in [1,32], box, out and target >= 1 required");
    if (strategy < 0 || strategy > 2) return fail(nullptr, IVB_EINVAL, "pick_splits: unknown strategy");
    double w[IVB_MAX_VARS];
    for (int i = 0; i < n; ++i) {
        const double wi = box[2 * i + 1] - box[2 * i];
        w[i] = ref_widths ? (ref_widths[i] > 0 ? wi / ref_widths[i] : 0.0) : wi;
    }
    if (strategy == IVB_SPLIT_LARGEST) {
        int wi = 0;
        for (int i = 1; i < n; ++i) if (w[i] > w[wi]) wi = i;
        for (int i = 0; i < n; ++i) out[i] = 1;
        out[wi] = (int32_t)std::min<int64_t>(target, 2147483647);
        return IVB_OK;
    }
    // largest N with N^n <= target
    int64_t N = 1;
    for (;;) {
        const int64_t M = N + 1;
        int64_t prod = 1;
        bool over = false;
        for (int i = 0; i < n && !over; ++i) {
            if (prod > target / M) over = true;
            else prod *= M;
        }
        if (over || prod > target) break;
        N = M;
    }
    for (int i = 0; i < n; ++i) out[i] = (int32_t)N;
    if (strategy == IVB_SPLIT_ADAPTIVE) {
        int64_t prod = 1;
        for (int i = 0; i < n; ++i) prod *= out[i];
        for (;;) {
            int best = -1;
            double bv = -1.0;
            for (int i = 0; i < n; ++i) {
                const int64_t rest = prod / out[i];
                if (rest > target / (out[i] + 1)) continue;
                if (rest * (out[i] + 1) > target) continue;
                const double v = w[i] / out[i];
                if (v > bv) { bv = v; best = i; }
            }
            if (best < 0) break;
            prod = (prod / out[best]) * (out[best] + 1);
            out[best] += 1;
        }
    }
    return IVB_OK;
}

extern "C" ivb_status ivb_get_tuning(ivb_problem* p, int32_t* block_threads, int32_t* blocks_per_sm, int32_t* tile,
                                     int32_t* frame_in_shared) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    if (block_threads) *block_threads = p->block;
    if (blocks_per_sm) *blocks_per_sm = p->bps;
    if (tile) *tile = p->tile;
    if (frame_in_shared) *frame_in_shared = p->frame_smem;
    return IVB_OK;
}

extern "C" ivb_status ivb_get_tuning_ex(ivb_problem* p, ivb_tuning* t) {
    if (!p || !t) return fail(p, IVB_EINVAL, "problem handle and result are required");
    t->block_threads = p->block;
    t->blocks_per_sm = p->bps;
    t->tile = p->tile;
    t->frame_in_shared = p->frame_smem;
    t->threads_per_subdomain = p->tpsub;
    t->chunk_sync = p->chunk_sync ? 1 : 0;
    t->kernel = reduce_jit(p) ? (p->jit.state_units > 0 ? 2 : 1) : 0;
    t->subdomains_per_pass = pass_size(p, p->block, p->tpsub);
    t->candidates = p->tune_candidates;
    t->best_ms = p->tune_best_ms;
    t->worst_ms = p->tune_worst_ms;
    return IVB_OK;
}

extern "C" ivb_status ivb_get_specialization(ivb_problem* p, int32_t* active, int32_t* registers,
                                             int32_t* local_bytes, double* compile_seconds, int32_t* emulate) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    if (active) *active = use_jit(p) ? 1 : 0;
    if (emulate) *emulate = use_jit(p) ? p->jit.emulate : 0;
    if (registers) *registers = p->jit.regs;
    if (local_bytes) *local_bytes = p->jit.local_bytes;
    if (compile_seconds) *compile_seconds = p->jit.compile_seconds;
    return IVB_OK;
}

extern "C" ivb_status ivb_get_segmentation(ivb_problem* p, int32_t* state_units, int32_t* chunks,
                                           int64_t* state_loads, int64_t* state_stores, int64_t* recomputed,
                                           int32_t* recompute, int32_t* ilp) {
    if (!p) return fail(nullptr, IVB_EINVAL, "problem handle is NULL");
    const bool seg = use_jit(p) && p->jit.state_units > 0;
    if (state_units) *state_units = seg ? p->jit.state_units : 0;
    if (chunks) *chunks = seg ? p->jit.chunks : 0;
    if (state_loads) *state_loads = seg ? p->jit.state_loads : 0;
    if (state_stores) *state_stores = seg ? p->jit.state_stores : 0;
    if (recomputed) *recomputed = seg ? p->jit.recomputed : 0;
    if (recompute) *recompute = seg ? p->jit.recompute : 0;
    if (ilp) *ilp = seg ? p->jit.ilp : 0;
    return IVB_OK;
}

extern "C" ivb_status ivb_specialize_compile(const ivb_tape* tape, int32_t grad_mode, int32_t compact,
                                             int32_t* registers, int32_t* spill_bytes, double* seconds) {
    std::string e = validate_tape(tape);
    if (!e.empty()) return fail(nullptr, IVB_ETAPE, e);
    if (grad_mode != IVB_GRAD_FORWARD && grad_mode != IVB_GRAD_ADJOINT)
        return fail(nullptr, IVB_EINVAL, "grad_mode must be IVB_GRAD_FORWARD or IVB_GRAD_ADJOINT");
    HostProgram P;
    std::vector<Ins> ins;
    std::vector<RIns> rins;
    std::vector<double> consts;
    e = compile_tape(tape, P, ins, rins, consts);
    if (!e.empty()) return fail(nullptr, IVB_ENOTSUP, e);
    const int mode = grad_mode == IVB_GRAD_ADJOINT ? KM_ADJ_REDUCE : KM_FWD_REDUCE;
    std::vector<char> cubin;
    std::string tables;
    int regs = 0, spill = 0;
    if (compact == 3 || compact == 4) {
        if (grad_mode != IVB_GRAD_ADJOINT)
            return fail(nullptr, IVB_EINVAL, "the segmented kernel needs grad_mode IVB_GRAD_ADJOINT");
        ivb_options o;
        ivb_options_default(&o);
        if (compact == 4) o.seg_ilp = 2;
        const SegPolicy pol = seg_policy(o);
        const SegSource src = jit_seg_source(P, ins, rins, consts, kJitBlockMax, seg_min_blocks(pol.max_regs),
                                             compact == 4 ? 15 : kJitDefaultEmulate, 0, pol);
        e = jit_seg_compile(src, pol.max_regs, cubin, tables, seconds, &regs, &spill);
    } else {
        const std::string src =
            jit_source(P, ins, rins, consts, mode, kJitBlockMax, kJitMinBlocks, kJitDefaultEmulate, compact != 0, 0);
        e = jit_compile(src, cubin, tables, seconds, &regs, &spill);
    }
    if (!e.empty()) return fail(nullptr, IVB_ENOTSUP, e);
    if (registers) *registers = regs;
    if (spill_bytes) *spill_bytes = spill;
    return IVB_OK;
}

extern "C" ivb_status ivb_eval_op(int32_t opcode, int64_t n, const double* x, const double* y, double* r,
                                  void* cuda_stream) {
    if (n < 0 || !x || !r) return fail(nullptr, IVB_EINVAL, "ivb_eval_op: x and r are required");
    const bool binary = opcode == IVB_OP_ADD || opcode == IVB_OP_SUB || opcode == IVB_OP_MUL || opcode == IVB_OP_DIV ||
                        opcode == IVB_EVAL_EMU_ADD || opcode == IVB_EVAL_EMU_SUB || opcode == IVB_EVAL_EMU_MUL ||
                        opcode == IVB_EVAL_FMA;
    const bool unary = opcode == IVB_OP_SQR || opcode == IVB_OP_SQRT || opcode == IVB_OP_EXP || opcode == IVB_OP_LOG ||
                       opcode == IVB_OP_NEG || opcode == IVB_EVAL_RECIP || opcode == IVB_EVAL_EMU_SQR;
    if (!binary && !unary) return fail(nullptr, IVB_EINVAL, "ivb_eval_op: unknown opcode");
    if (binary && !y) return fail(nullptr, IVB_EINVAL, "ivb_eval_op: binary operation needs y");
    if (n == 0) return IVB_OK;
    cudaError_t e = init_math_tables();
    if (e == cudaSuccess) e = launch_eval_op(opcode, n, x, binary ? y : nullptr, r, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(nullptr, IVB_ECUDA, std::string("ivb_eval_op: ") + cudaGetErrorString(e));
    return IVB_OK;
}

extern "C" ivb_status ivb_op_counts(const ivb_problem* p, int64_t counts[IVB_CNT_N]) {
    if (!p || !counts) return IVB_EINVAL;
    const bool adj = p->opt.grad_mode == IVB_GRAD_ADJOINT;
    const int64_t* c = p->opt.form == IVB_FORM_NIE ? (adj ? p->P.cnt_nie_adj : p->P.cnt_nie_fwd)
                                                   : (adj ? p->P.cnt_adj : p->P.cnt_fwd);
    for (int i = 0; i < IVB_CNT_N; ++i) counts[i] = c[i];
    return IVB_OK;
}

extern "C" int64_t ivb_launch_count(const ivb_problem* p) { return p ? p->launches : 0; }

extern "C" const char* ivb_last_error(const ivb_problem* p) {
    return p ? p->err.c_str() : g_create_error.c_str();
}

extern "C" void ivb_destroy(ivb_problem* p) {
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->queue_free) { cudaEventSynchronize(p->queue_free); cudaEventDestroy(p->queue_free); }
    cudaFree(p->d_prog);
    cudaFree(p->d_ins);
    cudaFree(p->d_rins);
    cudaFree(p->d_consts);
    cudaFree(p->d_out_kind);
    cudaFree(p->d_queue);
    if (p->h_queue) cudaFreeHost(p->h_queue);
    cudaFree(p->d_keys);
    cudaFree(p->d_counter);
    cudaFree(p->d_lb);
    cudaFree(p->d_ub);
    cudaFree(p->d_inf);
    cudaFree(p->d_minlo);
    cudaFree(p->d_maxhi);
    cudaFree(p->d_frame);
    cudaFree(p->d_pframe);
    jit_unload(p->jit);
    delete p;
}
