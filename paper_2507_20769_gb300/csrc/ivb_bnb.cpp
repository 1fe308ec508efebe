// ivb_bnb.cpp -- best-first spatial branch and bound (Section 3, Fig. 3)
// with GPU Subdomain Lower Bounding as the lower-bounding solver.
//
// Each iteration pops up to `batch` open nodes of lowest lower bound, bisects
// each along the dimension of largest width relative to the root box,
// optionally tightens every child by constraint propagation on the host
// (dropping children proven empty), and bounds all children in ONE call of
// the bounding path (one persistent launch when the problem is batched; one
// launch per child otherwise). The incumbent comes from the rigorous
// centre-point upper bounds of the children and from a descent-corner point
// evaluated on the host (the paper's local-solver upper bounding is replaced
// by these certified values). With `overlap`, the next batch is selected and
// enqueued before the batch in flight is absorbed, so host work runs while
// the GPU bounds.
// Children that are infeasible or have lb >= UB - max(eps_abs, eps_rel |UB|)
// are dropped. The run stops when UB - min(open lb) <= that tolerance, the
// heap empties, or a node / time limit is reached; the reported lower bound
// is min(open lb, lb of nodes dropped by the bound test).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_compile.h"
#include "ivb_host.h"
#include "ivb_problem.h"


namespace {

struct Node {
    double lb;
    std::vector<double> box;
};
struct Cmp {
    bool operator()(const Node* a, const Node* b) const { return a->lb > b->lb; }
};

// one batch of children on its way through the bounding kernel: boxes and
// splits staged on the host, results in pinned buffers, an event when done
struct Batch {
    std::vector<Node*> kids;
    std::vector<double> boxes;
    std::vector<int32_t> splits;
    double* lb = nullptr;
    double* ub = nullptr;
    uint8_t* inf = nullptr;
    cudaEvent_t done = nullptr;
    double parent_lb = INFINITY;   // smallest lower bound of the parents (open while in flight)
    bool in_flight = false;
};

}  // namespace

extern "C" void ivb_bnb_options_default(ivb_bnb_options* o) {
    if (!o) return;
    o->batch = 1;
    o->split_mode = 0;
    o->splits = nullptr;
    o->target = 0;
    o->eps_abs = 0.0;
    o->eps_rel = 1e-3;
    o->max_nodes = 0;
    o->time_limit = 0.0;
    o->corner_ub = 1;
    o->propagate = 0;
    o->overlap = 0;
}

extern "C" ivb_status ivb_propagate(const ivb_tape* tape, int32_t n_boxes, const double* boxes, double ub,
                                    int32_t passes, double* boxes_out, uint8_t* infeasible) {
    if (!boxes || !boxes_out || !infeasible || n_boxes < 0 || passes < 0) return IVB_EINVAL;
    if (!ivb::validate_tape(tape).empty()) return IVB_ETAPE;
    ivb::HostTape H;
    ivb::host_tape(tape, H);
    const int n = H.n;
    for (int k = 0; k < n_boxes; ++k) {
        double* b = boxes_out + (size_t)k * 2 * n;
        if (b != boxes + (size_t)k * 2 * n) std::memcpy(b, boxes + (size_t)k * 2 * n, 2 * n * sizeof(double));
        infeasible[k] = (uint8_t)ivb::host_propagate(H, b, ub, passes);
    }
    return IVB_OK;
}

extern "C" ivb_status ivb_host_gradient(const ivb_tape* tape, const double* box, int32_t output, int32_t grad_mode,
                                        double* G) {
    if (!tape || !box || !G) return IVB_EINVAL;
    if (!ivb::validate_tape(tape).empty()) return IVB_ETAPE;
    if (output < 0 || output >= tape->n_outputs || (grad_mode != IVB_GRAD_FORWARD && grad_mode != IVB_GRAD_ADJOINT))
        return IVB_EINVAL;
    ivb::HostTape H;
    ivb::host_tape(tape, H);
    std::vector<ivb::hiv> g(H.n);
    ivb::host_gradient(H, box, output, grad_mode, g.data());
    for (int i = 0; i < H.n; ++i) {
        G[2 * i] = g[i].lo;
        G[2 * i + 1] = g[i].hi;
    }
    return IVB_OK;
}

extern "C" ivb_status ivb_bnb_solve(ivb_problem* p, int32_t n, const double* root, const ivb_bnb_options* o,
                                    ivb_bnb_result* res, void* stream_) {
    if (!p) return IVB_EINVAL;
    p->err.clear();
    if (!root || !o || !res || n != p->n) {
        p->err = "ivb_bnb_solve: root, options and result are required and n must equal the problem's n_vars";
        return IVB_EINVAL;
    }
    if (o->batch < 1 || (o->split_mode == 0 && !o->splits) || (o->split_mode > 0 && o->target < 0) ||
        o->propagate < 0) {
        p->err = "ivb_bnb_solve: batch >= 1, splits (split_mode 0) or target >= 0, propagate >= 0";
        return IVB_EINVAL;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    const ivb::HostTape& H = p->host;
    const int grad_mode = p->opt.grad_mode;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<double> ref(n);
    for (int i = 0; i < n; ++i) ref[i] = root[2 * i + 1] - root[2 * i];
    std::priority_queue<Node*, std::vector<Node*>, Cmp> heap;
    double UB = INFINITY, lb_pruned = INFINITY;
    int64_t iters = 0, bounded = 0, subs = 0;
    const int cap = std::max(2 * o->batch, 1);
    if (cap > p->max_nodes) {
        p->err = "ivb_bnb_solve: 2 * batch exceeds the problem's max_nodes";
        return IVB_EINVAL;
    }

    Batch bat[2];
    ivb_status st = IVB_OK;
    for (Batch& b : bat) {
        b.boxes.resize((size_t)cap * n * 2);
        b.splits.resize((size_t)cap * n);
        if (cudaMallocHost(&b.lb, cap * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&b.ub, cap * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&b.inf, cap) != cudaSuccess ||
            cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
            st = IVB_ENOMEM;
    }
    auto release = [&]() {
        for (Batch& b : bat) {
            if (b.in_flight && b.done) cudaEventSynchronize(b.done);
            for (Node* k : b.kids) delete k;
            b.kids.clear();
            if (b.lb) cudaFreeHost(b.lb);
            if (b.ub) cudaFreeHost(b.ub);
            if (b.inf) cudaFreeHost(b.inf);
            if (b.done) cudaEventDestroy(b.done);
        }
        while (!heap.empty()) { delete heap.top(); heap.pop(); }
    };
    if (st) { release(); return st; }

    auto tol_of = [&](double ub) { return std::max(o->eps_abs, o->eps_rel * std::fabs(ub)); };
    // constraint propagation of a child against the incumbent; false: drop it
    auto keep = [&](Node* k) {
        return o->propagate == 0 || ivb::host_propagate(H, k->box.data(), UB, o->propagate) == 0;
    };
    // stage and enqueue a batch; its results arrive in the pinned buffers
    int64_t last_target = o->split_mode > 0 ? o->target : 0;
    auto launch = [&](Batch& b) -> ivb_status {
        const int cnt = (int)b.kids.size();
        // subdomains per child for the split picker: the given target, or with
        // target 0 the smallest power of two >= 2^8 (at most 2^20) with which
        // this iteration's children cover four waves of the bounding launch
        int64_t target = o->target;
        if (o->split_mode > 0 && target == 0) {
            const int ilp = p->jit.kern && p->jit.state_units > 0 ? p->jit.ilp : 1;
            const int64_t wave =
                (int64_t)p->sm_count * std::max(1, p->bps) * (std::max(1, p->block) / std::max(1, p->tpsub)) * ilp;
            const int64_t want = (4 * wave + cnt - 1) / std::max(1, cnt);
            target = 1 << 8;
            while (target < want && target < (1 << 20)) target <<= 1;
        }
        last_target = target;
        for (int k = 0; k < cnt; ++k) {
            std::memcpy(&b.boxes[(size_t)k * n * 2], b.kids[k]->box.data(), n * 2 * sizeof(double));
            int32_t* sp = &b.splits[(size_t)k * n];
            if (o->split_mode == 0) std::memcpy(sp, o->splits, n * sizeof(int32_t));
            else if (ivb_status e = ivb_pick_splits(n, b.kids[k]->box.data(), ref.data(), target,
                                                    o->split_mode - 1, sp))
                return e;
            int64_t s = 1;
            for (int i = 0; i < n; ++i) s *= sp[i];
            subs += s;
        }
        bounded += cnt;
        ivb_status e = bound_nodes_enqueue(p, cnt, b.boxes.data(), b.splits.data(), b.lb, b.inf, b.ub, nullptr,
                                           nullptr, stream);
        if (e) return e;
        if (cudaEventRecord(b.done, stream) != cudaSuccess) return IVB_ECUDA;
        b.in_flight = true;
        return IVB_OK;
    };
    // wait for a batch, update the incumbent, push or drop its children
    auto absorb = [&](Batch& b) -> ivb_status {
        if (cudaEventSynchronize(b.done) != cudaSuccess) return IVB_ECUDA;
        b.in_flight = false;
        const int cnt = (int)b.kids.size();
        int best = -1;
        for (int k = 0; k < cnt; ++k) {
            if (b.ub[k] < UB) UB = b.ub[k];
            if (best < 0 || b.ub[k] < b.ub[best]) best = k;
        }
        if (o->corner_ub && best >= 0) {
            const double v = ivb::host_corner_value(H, b.kids[best]->box.data(), grad_mode);
            if (v < UB) UB = v;
        }
        for (int k = 0; k < cnt; ++k) {
            const double tol = tol_of(UB);
            if (!b.inf[k] && !(b.lb[k] >= UB - tol)) {
                b.kids[k]->lb = b.lb[k];
                heap.push(b.kids[k]);
            } else {
                if (!b.inf[k] && b.lb[k] < lb_pruned) lb_pruned = b.lb[k];
                delete b.kids[k];
            }
        }
        b.kids.clear();
        return IVB_OK;
    };
    // pop up to `batch` parents of lowest lower bound and bisect each along
    // the dimension of largest width relative to the root box
    auto select = [&](Batch& b) {
        b.kids.clear();
        b.parent_lb = INFINITY;
        const double tol = tol_of(UB);
        int parents = 0;
        while (!heap.empty() && parents < o->batch) {
            Node* nd = heap.top();
            heap.pop();
            if (nd->lb >= UB - tol) {
                if (nd->lb < lb_pruned) lb_pruned = nd->lb;
                delete nd;
                continue;
            }
            ++iters;
            ++parents;
            b.parent_lb = std::min(b.parent_lb, nd->lb);
            int bi = 0;
            double bw = -1.0;
            for (int i = 0; i < n; ++i) {
                const double w = (nd->box[2 * i + 1] - nd->box[2 * i]) / ref[i];
                if (w > bw) { bw = w; bi = i; }
            }
            const double lo = nd->box[2 * bi], hi = nd->box[2 * bi + 1];
            const double mid = lo + (hi - lo) * 0.5;
            Node* l = new Node{0.0, nd->box};
            l->box[2 * bi + 1] = mid;
            nd->box[2 * bi] = mid;
            for (Node* k : {l, nd}) {
                if (keep(k)) b.kids.push_back(k);
                else delete k;
            }
        }
    };

    int converged = 0;
    {
        Node* r = new Node{0.0, std::vector<double>(root, root + 2 * n)};
        if (keep(r)) bat[0].kids.push_back(r);
        else delete r;
        if (!bat[0].kids.empty()) {
            st = launch(bat[0]);
            if (!st) st = absorb(bat[0]);
        }
    }
    int cur = 0;   // overlap: the batch in flight, if any
    while (!st) {
        const double tol = tol_of(UB);
        double open_lb = heap.empty() ? INFINITY : heap.top()->lb;
        if (bat[cur].in_flight) open_lb = std::min(open_lb, bat[cur].parent_lb);
        const bool idle = heap.empty() && !bat[cur].in_flight;
        if (idle || UB - open_lb <= tol) {
            converged = 1;
            if (bat[cur].in_flight) st = absorb(bat[cur]);
            break;
        }
        if ((o->max_nodes > 0 && bounded >= o->max_nodes) || (o->time_limit > 0 && elapsed() > o->time_limit)) {
            if (bat[cur].in_flight) st = absorb(bat[cur]);
            break;
        }
        if (!o->overlap) {
            select(bat[0]);
            if (bat[0].kids.empty()) continue;
            st = launch(bat[0]);
            if (!st) st = absorb(bat[0]);
            continue;
        }
        // overlap: enqueue the next batch behind the one in flight, then absorb that one
        Batch& next = bat[1 - cur];
        select(next);
        if (!next.kids.empty()) st = launch(next);
        if (!st && bat[cur].in_flight) st = absorb(bat[cur]);
        cur = 1 - cur;
    }
    double lbg = heap.empty() ? UB : heap.top()->lb;
    if (lb_pruned < lbg) lbg = lb_pruned;
    res->lb = lbg;
    res->ub = UB;
    res->iterations = iters;
    res->nodes_bounded = bounded;
    res->subdomains = subs;
    res->seconds = elapsed();
    res->converged = converged;
    res->open_nodes = (int64_t)heap.size();
    res->split_target = last_target;
    release();
    return st;
}
