// ivb_bnb.cpp -- best-first spatial branch and bound (Section 3, Fig. 3)
// with GPU Subdomain Lower Bounding as the lower-bounding solver.
//
// Each iteration pops up to `batch` open nodes of lowest lower bound, bisects
// each along the dimension of largest width relative to the root box, and
// bounds all children in ONE ivb_bound_nodes_ex call (one persistent launch
// when the problem is batched; one launch per child otherwise). The incumbent
// comes from the rigorous centre-point upper bounds of the children (the
// paper's local-solver upper bounding is replaced by these certified values).
// Children that are infeasible or have lb >= UB - max(eps_abs, eps_rel |UB|)
// are dropped. The run stops when UB - min(open lb) <= that tolerance, the
// heap empties, or a node / time limit is reached; the reported lower bound
// is min(open lb, lb of nodes dropped by the bound test).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "../../include/ivb.h"
#include "ivb_problem.h"

namespace {

struct Node {
    double lb;
    std::vector<double> box;
};
struct Cmp {
    bool operator()(const Node* a, const Node* b) const { return a->lb > b->lb; }
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
}

extern "C" ivb_status ivb_bnb_solve(ivb_problem* p, int32_t n, const double* root, const ivb_bnb_options* o,
                                    ivb_bnb_result* res, void* stream) {
    if (!p || !root || !o || !res || n < 1 || n > IVB_MAX_VARS) return IVB_EINVAL;
    if (o->batch < 1 || (o->split_mode == 0 && !o->splits) || (o->split_mode > 0 && o->target < 1))
        return IVB_EINVAL;
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<double> ref(n);
    for (int i = 0; i < n; ++i) ref[i] = root[2 * i + 1] - root[2 * i];
    std::priority_queue<Node*, std::vector<Node*>, Cmp> heap;
    double UB = INFINITY, lb_pruned = INFINITY;
    int64_t iters = 0, bounded = 0, subs = 0;
    const int cap = 2 * o->batch;
    std::vector<double> boxes((size_t)cap * n * 2), lb(cap), ub(cap);
    std::vector<int32_t> splits((size_t)cap * n);
    std::vector<uint8_t> inf(cap);
    std::vector<Node*> kids;

    auto set_splits = [&](const double* box, int32_t* sp) -> ivb_status {
        if (o->split_mode == 0) { std::memcpy(sp, o->splits, n * sizeof(int32_t)); return IVB_OK; }
        return ivb_pick_splits(n, box, ref.data(), o->target, o->split_mode - 1, sp);
    };
    auto bound = [&](int cnt) -> ivb_status {
        for (int k = 0; k < cnt; ++k) {
            std::memcpy(&boxes[(size_t)k * n * 2], kids[k]->box.data(), n * 2 * sizeof(double));
            ivb_status st = set_splits(kids[k]->box.data(), &splits[(size_t)k * n]);
            if (st) return st;
            int64_t s = 1;
            for (int i = 0; i < n; ++i) s *= splits[(size_t)k * n + i];
            subs += s;
        }
        bounded += cnt;
        return ivb_bound_nodes_ex(p, cnt, boxes.data(), splits.data(), lb.data(), inf.data(), ub.data(), nullptr,
                                  nullptr, stream);
    };
    // rigorous value of the objective at a point, +inf unless certified feasible
    const int n_out = p->n_out, obj = p->obj;
    std::vector<double> ptbox(2 * n), Fv(2 * n_out), Fcv(2 * n_out), Gv((size_t)2 * n_out * n);
    std::vector<int32_t> ones(n, 1);
    auto point_value = [&](const double* x) -> double {
        for (int i = 0; i < n; ++i) { ptbox[2 * i] = x[i]; ptbox[2 * i + 1] = x[i]; }
        if (ivb_enclose(p, ptbox.data(), ones.data(), 0, 1, Fv.data(), Fcv.data(), nullptr, stream) != IVB_OK)
            return INFINITY;
        if (p->P.has_eq) return INFINITY;
        for (int q = 0; q < n_out; ++q)
            if (p->out_kind[q] == IVB_OUT_INEQ && !(Fcv[2 * q + 1] <= 0.0)) return INFINITY;
        return Fcv[2 * obj + 1];
    };
    // descent corner of a box: the sign of the objective's gradient enclosure
    // over the box picks lo or hi per dimension, the centre where it is unknown
    std::vector<double> cpt(n), mpt(n);
    auto corner_value = [&](const double* box) -> double {
        if (ivb_enclose(p, box, ones.data(), 0, 1, Fv.data(), nullptr, Gv.data(), stream) != IVB_OK) return INFINITY;
        const double* G = Gv.data() + (size_t)obj * n * 2;
        for (int i = 0; i < n; ++i) {
            const double lo = box[2 * i], hi = box[2 * i + 1], c = (lo + hi) * 0.5;
            cpt[i] = G[2 * i] > 0.0 ? lo : (G[2 * i + 1] < 0.0 ? hi : c);
            mpt[i] = (cpt[i] + c) * 0.5;
        }
        const double v = point_value(cpt.data());
        if (v < INFINITY) return v;
        return point_value(mpt.data());
    };
    auto absorb = [&](int cnt) {
        int best = -1;
        for (int k = 0; k < cnt; ++k) {
            if (ub[k] < UB) UB = ub[k];
            if (best < 0 || ub[k] < ub[best]) best = k;
        }
        if (o->corner_ub && best >= 0) {
            const double v = corner_value(kids[best]->box.data());
            if (v < UB) UB = v;
        }
        for (int k = 0; k < cnt; ++k) {
            const double tol = std::max(o->eps_abs, o->eps_rel * std::fabs(UB));
            if (!inf[k] && !(lb[k] >= UB - tol)) {
                kids[k]->lb = lb[k];
                heap.push(kids[k]);
            } else {
                if (!inf[k] && lb[k] < lb_pruned) lb_pruned = lb[k];
                delete kids[k];
            }
        }
        kids.clear();
    };

    kids.push_back(new Node{0.0, std::vector<double>(root, root + 2 * n)});
    ivb_status st = bound(1);
    if (st) { for (Node* k : kids) delete k; return st; }
    absorb(1);
    int converged = 0;
    for (;;) {
        if (heap.empty()) { converged = 1; break; }
        const double tol = std::max(o->eps_abs, o->eps_rel * std::fabs(UB));
        if (UB - heap.top()->lb <= tol) { converged = 1; break; }
        if ((o->max_nodes > 0 && bounded >= o->max_nodes) || (o->time_limit > 0 && elapsed() > o->time_limit)) break;
        while (!heap.empty() && (int)kids.size() < cap) {
            Node* nd = heap.top();
            heap.pop();
            if (nd->lb >= UB - tol) {
                if (nd->lb < lb_pruned) lb_pruned = nd->lb;
                delete nd;
                continue;
            }
            ++iters;
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
            kids.push_back(l);
            kids.push_back(nd);
        }
        if (kids.empty()) continue;
        const int cnt = (int)kids.size();
        st = bound(cnt);
        if (st) { for (Node* k : kids) delete k; break; }
        absorb(cnt);
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
    while (!heap.empty()) { delete heap.top(); heap.pop(); }
    return st;
}
