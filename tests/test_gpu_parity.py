"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on seeded inputs.

Bar (from the method's arithmetic): tapes with only + - * / sqr sqrt are
bit-exact in both gradient modes (every directed operation is correctly
rounded on both sides and the formulas are the same). With exp/log, each GPU
exp/log end lies within 4 representable steps of the oracle's tight end (at
most 3 from the true value: error below one ulp plus the two-step widening;
the oracle's tight end is within one), and every other operation is the same
monotone outward-rounded function on both sides; by inclusion isotonicity
(Definition 2) every GPU enclosure, at any tape depth, lies between the
oracle's tight sweep and its sweep with each exp/log end moved 4 further steps
outward (oracle mode tight=5). The tests check that bracket element by element
and record the largest distance of a GPU end from the tight end."""
from __future__ import annotations

import functools
import math

import numpy as np
import pytest

import oracle
import problems as P
from paper_2507_20769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_20769_gb300 import build as B  # noqa: E402

B.build()
from paper_2507_20769_gb300 import ivb  # noqa: E402

DEV = torch.device("cuda:0")
INF = math.inf


def rational_problem(n=3, K=60, n_ineq=2, seed=777):
    return W.random_problem(n, K, n_ineq, W.OPS_RATIONAL, [[-3, 2]] * n, seed, "rational")


def ulps(a, b):
    """number of doubles between a and b (both finite, same sign handled)"""
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    ia = np.where(ia < 0, np.int64(-(2 ** 63)) - ia, ia)
    ib = np.where(ib < 0, np.int64(-(2 ** 63)) - ib, ib)
    return np.abs(ia - ib)


WIDE = 5   # oracle mode: tight ends moved 4 steps outward per exp/log operation


def assert_bracketed(gpu, tight, wide, what=""):
    """tight ⊆ gpu ⊆ wide, end by end; records the largest number of
    representable steps between a GPU end and the tight end"""
    import conftest
    gl, gh = gpu[..., 0], gpu[..., 1]
    assert np.all(gl <= tight[..., 0]), f"{what}: lower end does not contain the oracle's"
    assert np.all(gh >= tight[..., 1]), f"{what}: upper end does not contain the oracle's"
    assert np.all(gl >= wide[..., 0]), f"{what}: lower end beyond the 4-step bracket"
    assert np.all(gh <= wide[..., 1]), f"{what}: upper end beyond the 4-step bracket"
    fl, fh = np.isfinite(tight[..., 0]) & np.isfinite(gl), np.isfinite(tight[..., 1]) & np.isfinite(gh)
    d = max(int(ulps(gl[fl], tight[..., 0][fl]).max(initial=0)), int(ulps(gh[fh], tight[..., 1][fh]).max(initial=0)))
    if what:
        key = what.split(":")[0]
        conftest.ULP_LOG[key] = max(conftest.ULP_LOG.get(key, 0), d)
    return d


def assert_enclose_bracketed(t, F, box, splits, first=0, count=None, grad_mode="adjoint", what="", **kw):
    """per-subdomain enclosures against the oracle's tight and 4-step sweeps"""
    Fo, _, _ = oracle.enclose(t, box, splits, first=first, count=count, grad_mode=grad_mode, tight=True, **kw)
    Fw, _, _ = oracle.enclose(t, box, splits, first=first, count=count, grad_mode=grad_mode, tight=WIDE, **kw)
    return assert_bracketed(F, Fo, Fw, what)


def hull(r):
    return np.stack([r["minlo"], r["maxhi"]], -1)


# ------------------------------------------------------------ per subdomain

@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("form", ["mvf", "nie", "mvf_nie"])
def test_enclose_bit_exact_rational(grad_mode, form):
    """Steps 1-2 per subdomain: F, f(c) and G equal the oracle's bit for bit
    (140 subdomains: several 128-thread tiles and a ragged tail)."""
    t = rational_problem()
    box = np.array([[-2.5, 1.0], [-1.0, 1.75], [0.5, 2.0]])
    splits = np.array([5, 4, 7], np.int32)
    with ivb.Problem(t, grad_mode=grad_mode, form=form) as p:
        F, Fc, G = p.enclose(box, splits, want_fc=True, want_g=True)
    Fo, Fco, Go = oracle.enclose(t, box, splits, grad_mode=grad_mode, form=form, tight=True,
                                 want_fc=True, want_g=True)
    assert np.array_equal(Fc, Fco)
    assert np.array_equal(G, Go)
    assert np.array_equal(F, Fo)


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_enclose_exp_log_bracketed(grad_mode):
    """configuration 2 per subdomain: f(c), the gradient enclosure and the
    Mean Value Form between the oracle's tight and 4-step sweeps"""
    t = W.config_tape(2)
    box = W.bisection_frontier(t.root_box, 8, seed=5)[3]
    splits = np.array([3, 4, 3, 3], np.int32)
    with ivb.Problem(t, grad_mode=grad_mode) as p:
        F, Fc, G = p.enclose(box, splits, want_fc=True, want_g=True)
    Fo, Fco, Go = oracle.enclose(t, box, splits, grad_mode=grad_mode, tight=True, want_fc=True, want_g=True)
    Fw, Fcw, Gw = oracle.enclose(t, box, splits, grad_mode=grad_mode, tight=WIDE, want_fc=True, want_g=True)
    assert_bracketed(Fc, Fco, Fcw, f"config 2 f(c) {grad_mode}")
    assert_bracketed(G, Go, Gw, f"config 2 gradient {grad_mode}")
    assert_bracketed(F, Fo, Fw, f"config 2 MVF {grad_mode}")


@pytest.mark.parametrize("fn,lo,hi", [("exp", -30.0, 30.0), ("exp", -740.0, 700.0), ("log", 1e-300, 1e300),
                                      ("log", 0.25, 4.0)])
def test_transcendental_op_within_4_ulps(fn, lo, hi):
    """one exp / log operation on 4096 intervals: contains the oracle's tight
    enclosure, each end within 4 ulps of it"""
    Bd = P.Builder(1)
    x = Bd.x(0)
    Bd.output(Bd.exp(x) if fn == "exp" else Bd.log(x))
    t = Bd.tape([[lo, hi]])
    with ivb.Problem(t, form="nie", grad_mode="forward") as p:
        F, _, _ = p.enclose(t.root_box, np.array([4096], np.int32))
    Fo, _, _ = oracle.enclose(t, t.root_box, [4096], form="nie", tight=True)
    g, r = F[:, 0], Fo[:, 0]
    assert np.all(g[:, 0] <= r[:, 0]) and np.all(g[:, 1] >= r[:, 1])
    m = np.isfinite(r[:, 0]) & (r[:, 0] != 0)
    assert np.all(ulps(g[m, 0], r[m, 0]) <= 4)
    m = np.isfinite(r[:, 1])
    assert np.all(ulps(g[m, 1], r[m, 1]) <= 4)


def test_domain_violations_give_entire_like_the_oracle():
    """sqrt of a negative part, log of a non-positive part, division by an
    interval with zero: ENTIRE, identically on both sides"""
    Bd = P.Builder(2)
    x, y = Bd.x(0), Bd.x(1)
    a = Bd.sqrt(Bd.sub(x, Bd.const(0.5)))
    b = Bd.div(Bd.const(1.0), y)
    Bd.output(Bd.add(a, b))
    t = Bd.tape([[-1.0, 1.0], [-1.0, 1.0]])
    for gm in ("forward", "adjoint"):
        with ivb.Problem(t, grad_mode=gm) as p:
            F, Fc, G = p.enclose(t.root_box, np.array([4, 5], np.int32), want_fc=True, want_g=True)
        Fo, Fco, Go = oracle.enclose(t, t.root_box, [4, 5], grad_mode=gm, want_fc=True, want_g=True)
        assert np.array_equal(F, Fo) and np.array_equal(Fc, Fco) and np.array_equal(G, Go)
        assert np.any(np.isinf(F))


# ------------------------------------------------------------------ per node

def ragged_batch(t, n_nodes, seed, max_split=6):
    rng = np.random.default_rng(seed)
    boxes = W.bisection_frontier(t.root_box, n_nodes, seed=seed)
    splits = rng.integers(1, max_split + 1, (n_nodes, t.n_vars)).astype(np.int32)
    splits[0] = 1                          # S = 1
    boxes[1, 0, 1] = boxes[1, 0, 0]        # degenerate dimension
    return boxes, splits


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("path", ["graph", "nograph", "plain"])
def test_bound_nodes_bit_exact_rational(grad_mode, path):
    """Steps 1-3 for a ragged batch (S from 1 to 216 per node, tiles crossing
    nodes): lb, infeasibility, centre upper bound and every output's hull
    equal the oracle's bit for bit, on every launch path."""
    t = rational_problem()
    boxes, splits = ragged_batch(t, 37, seed=11)
    opts = dict(grad_mode=grad_mode, use_graph=int(path == "graph"), batched=int(path != "plain"))
    with ivb.Problem(t, **opts) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        r2 = p.bound_nodes_ex(boxes, splits, want_hull=True)      # second call replays the graph
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=True)
    for rr in (r, r2):
        assert np.array_equal(rr["lb"], ref["lb"])
        assert np.array_equal(rr["minlo"], ref["minlo"])
        assert np.array_equal(rr["maxhi"], ref["maxhi"])
        assert np.array_equal(rr["ub"], ref["ub"])
        assert np.array_equal(rr["infeasible"].astype(bool), ref["infeasible"])


def test_device_and_host_pointers_agree():
    t = rational_problem()
    boxes, splits = ragged_batch(t, 20, seed=3)
    with ivb.Problem(t) as p:
        rh = p.bound_nodes_ex(boxes, splits, want_hull=True)
        rd = p.bound_nodes_ex(torch.from_numpy(boxes).to(DEV), torch.from_numpy(splits).to(DEV), want_hull=True)
        torch.cuda.synchronize()
    for k in ("lb", "ub", "minlo", "maxhi", "infeasible"):
        assert np.array_equal(rh[k], rd[k].cpu().numpy()), k


@pytest.mark.parametrize("kind", ["feasible", "infeasible", "eq_out", "eq_in"])
@pytest.mark.parametrize("filt", [0, 1])
def test_feasibility_filter_and_ub_match_oracle(kind, filt):
    t = P.constrained_toy(kind)
    boxes = W.bisection_frontier(t.root_box, 9, seed=2)
    splits = np.array([[6, 5]] * 9, np.int32)
    with ivb.Problem(t, filter=filt) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, filter=bool(filt))
    assert np.array_equal(r["lb"], ref["lb"])
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])
    assert np.array_equal(r["ub"], ref["ub"])


@pytest.mark.parametrize("config", [1, 2, 3, 4])
@pytest.mark.parametrize("grad_mode", ["adjoint", "forward"])
def test_bound_nodes_exp_log_configs_bracketed(config, grad_mode):
    """paper-shaped tapes with exp/log: node hulls and lower bounds between
    the oracle's tight and 4-step sweeps"""
    t = W.config_tape(config)
    n_nodes = 6
    boxes = W.bisection_frontier(t.root_box, n_nodes, seed=config)
    splits = np.full((n_nodes, t.n_vars), 3 if t.n_vars <= 4 else (2 if t.n_vars <= 8 else 1), np.int32)
    with ivb.Problem(t, grad_mode=grad_mode) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=True)
    wide = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=WIDE)
    assert_bracketed(hull(r), hull(ref), hull(wide), f"config {config} node hulls {grad_mode}")
    assert np.all(r["lb"] <= ref["lb"]) and np.all(r["lb"] >= wide["lb"])


@functools.lru_cache(maxsize=None)
def _config2_full_size_oracle():
    wl = W.config_workload(2)
    t = wl.tape
    boxes = W.bisection_frontier(t.root_box, 16, seed=20)
    splits = np.tile(wl.splits, (16, 1))
    return (t, boxes, splits, oracle.bound_nodes(t, boxes, splits, tight=True),
            oracle.bound_nodes(t, boxes, splits, tight=WIDE))


@pytest.mark.parametrize("specialize", [0, 1])
def test_full_size_config2_every_node_hull(specialize):
    """configuration 2 at full size, in the launch configuration bench.py
    times for that workload (16 nodes x 16^4 = 65536 subdomains per node, one
    batched launch, autotuned, CUDA graph), with the interpreter (0) and the
    tape-specialised kernel ivb_jit_bound (1): every node's hull, lower bound
    and flag against the oracle over all 2^20 subdomains, bracketed between
    its tight and 4-step sweeps"""
    t, boxes, splits, ref, wide = _config2_full_size_oracle()
    with ivb.Problem(t, specialize=specialize) as p:
        assert p.get_specialization()["active"] == bool(specialize)
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    assert_bracketed(hull(r), hull(ref), hull(wide), f"config 2 full-size hulls spec{specialize}")
    assert np.all(r["lb"] <= ref["lb"]) and np.all(r["lb"] >= wide["lb"])
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])


def test_full_size_config2_sampled_subdomains():
    """256 sampled subdomains of two full-size configuration-2 nodes, one by
    one, bracketed"""
    wl = W.config_workload(2)
    t = wl.tape
    boxes = W.bisection_frontier(t.root_box, 16, seed=20)
    with ivb.Problem(t) as p:
        rng = np.random.default_rng(0)
        for nd in (5, 11):
            for k in np.sort(rng.choice(65536, 128, replace=False)):
                F, _, _ = p.enclose(boxes[nd], wl.splits, first=int(k), count=1)
                assert_enclose_bracketed(t, F, boxes[nd], wl.splits, first=int(k), count=1,
                                         what=f"config 2 sampled subdomains: node {nd} subdomain {k}")


# ------------------------------------------------------------- edge cases

def test_invalid_inputs_rejected():
    t = rational_problem()
    with ivb.Problem(t, max_nodes=4) as p:
        good_b = np.array([t.root_box] * 2)
        good_s = np.ones((2, t.n_vars), np.int32)
        bad = []
        b = good_b.copy(); b[0, 0] = [1.0, 0.0]; bad.append((b, good_s))
        b = good_b.copy(); b[1, 2, 1] = np.nan; bad.append((b, good_s))
        s = good_s.copy(); s[1, 1] = 0; bad.append((good_b, s))
        s = good_s.copy(); s[0] = [2048, 2048, 2048]; bad.append((good_b, s))
        bad.append((np.array([t.root_box] * 5), np.ones((5, t.n_vars), np.int32)))   # > max_nodes
        for bb, ss in bad:
            with pytest.raises(ivb.IvbError) as e:
                p.bound_nodes(bb, ss)
            assert e.value.status == ivb.IVB_EINVAL
        # the handle stays usable after errors; an empty batch is a no-op
        lb, inf = p.bound_nodes(good_b, good_s)
        assert np.all(np.isfinite(lb))
        lb0, _ = p.bound_nodes(np.zeros((0, t.n_vars, 2)), np.zeros((0, t.n_vars), np.int32))
        assert lb0.shape == (0,)


def test_single_subdomain_equals_unsplit_mvf():
    """N = 1 everywhere: the node bound is the MVF on the whole box"""
    t = rational_problem(seed=5)
    with ivb.Problem(t) as p:
        r = p.bound_nodes_ex(t.root_box[None], np.ones((1, t.n_vars), np.int32), want_hull=True)
        F, _, _ = p.enclose(t.root_box, np.ones(t.n_vars, np.int32))
    assert np.array_equal(r["minlo"][0], F[0, :, 0])
    assert np.array_equal(r["maxhi"][0], F[0, :, 1])


# ---------------------------------------------------------- point gradients

def test_point_grad_matches_oracle():
    t = rational_problem()
    x = W.sample_points(t.root_box, 300, seed=1)
    with ivb.Problem(t) as p:
        f, g = p.point_grad(x)
    for i in range(x.shape[0]):
        fo, go = oracle.point_grad(t, x[i])
        assert np.array_equal(f[i], fo) and np.array_equal(g[i], go)
    t = W.config_tape(4)
    x = W.sample_points(t.root_box, 64, seed=2)
    with ivb.Problem(t) as p:
        f, g = p.point_grad(torch.from_numpy(x).to(DEV))
        f, g = f.cpu().numpy(), g.cpu().numpy()
    for i in range(x.shape[0]):
        fo, go = oracle.point_grad(t, x[i])
        assert np.allclose(f[i], fo, rtol=1e-12, atol=1e-12)
        assert np.allclose(g[i], go, rtol=1e-10, atol=1e-12)
        h = 1e-6 * np.maximum(1.0, np.abs(x[i]))
        gfd = oracle.central_diff_q(t, x[i], h)
        assert np.all(np.abs(g[i] - gfd) <= 1e-6 * np.maximum(1.0, np.abs(g[i])))


def test_adjoint_contains_sampled_point_gradients_config4():
    """configuration 4 (n=16, K=400): on a 2^12 subsample of the 2^20
    subdomains, every interval adjoint contains 64 point gradients sampled in
    its subdomain (round-to-nearest point gradients, slack 1e-9 relative for
    their own rounding)."""
    wl = W.config_workload(4)
    t = wl.tape
    S = int(np.prod(wl.splits))
    rng = np.random.default_rng(4)
    ks = np.sort(rng.choice(S, 4096, replace=False))
    with ivb.Problem(t, grad_mode="adjoint") as p:
        Gs = []
        for k in ks:
            _, _, G = p.enclose(t.root_box, wl.splits, first=int(k), count=1, want_g=True)
            Gs.append(G[0, 0])
        pts = []
        for k in ks:
            X, _ = oracle.decode(t.root_box, wl.splits, int(k))
            pts.append(rng.uniform(X[:, 0], X[:, 1], (64, t.n_vars)))
        pts = np.concatenate(pts)
        _, g = p.point_grad(pts)
    g = g[:, 0, :].reshape(len(ks), 64, t.n_vars)
    Gs = np.stack(Gs)
    slack = 1e-9 * np.maximum(1.0, np.abs(g))
    assert np.all(g >= Gs[:, None, :, 0] - slack)
    assert np.all(g <= Gs[:, None, :, 1] + slack)


# --------------------------------------------------------------- B&B

def test_bnb_gpu_matches_oracle_tiny():
    wl = W.config_workload(1)
    t = wl.tape
    ref = oracle.bnb(t, splits=wl.splits, eps_abs=wl.gap_abs, eps_rel=0.0, grad_mode="forward", tight=True,
                     max_nodes=100000)
    for gm, batched, batch in (("forward", 0, 1), ("adjoint", 1, 8)):
        with ivb.Problem(t, grad_mode=gm, batched=batched) as p:
            r = p.bnb_solve(t.root_box, splits=wl.splits, batch=batch, eps_abs=wl.gap_abs, eps_rel=0.0,
                            max_nodes=100000)
        assert r["converged"] and ref["converged"]
        assert r["ub"] - r["lb"] <= wl.gap_abs
        # both bracket the same minimum
        assert r["lb"] <= ref["ub"] and ref["lb"] <= r["ub"]


def test_bnb_gpu_follows_oracle_trajectory_rational():
    """bit-exact bounds give the same B&B: one node per iteration, same
    bounded-node count and final bounds (node limit reached or converged)"""
    t = rational_problem(n=2, K=40, n_ineq=1, seed=99)
    sp = np.array([6, 6], np.int32)
    ref = oracle.bnb(t, splits=sp, eps_abs=0.0, eps_rel=1e-4, grad_mode="adjoint", tight=True, max_nodes=400)
    with ivb.Problem(t, grad_mode="adjoint", batched=0) as p:
        r = p.bnb_solve(t.root_box, splits=sp, batch=1, eps_abs=0.0, eps_rel=1e-4, max_nodes=400)
    assert (r["nodes"], r["lb"], r["ub"], r["converged"]) == (ref["nodes"], ref["lb"], ref["ub"], ref["converged"])


def test_bnb_shifted_squares_closed_form():
    t = P.shifted_squares(3, [0.3, -1.1, 0.7], [[-2, 2]] * 3)
    with ivb.Problem(t) as p:
        r = p.bnb_solve(t.root_box, splits=[8, 8, 8], batch=4, eps_abs=1e-6, eps_rel=0.0, max_nodes=100000)
    assert r["converged"] and r["lb"] <= 0.0 <= r["ub"] <= 1e-6


def test_launch_count_and_tuning_reported():
    t = rational_problem()
    boxes, splits = ragged_batch(t, 8, seed=1)
    with ivb.Problem(t) as p:
        c0 = p.launch_count()
        p.bound_nodes(boxes, splits)
        assert p.launch_count() == c0 + 3
        tun = p.get_tuning()
        assert tun["block_threads"] > 0 and tun["blocks_per_sm"] > 0


# ------------------------------------------------------- autograd Function

def test_autograd_point_grad_against_oracle_and_central_differences():
    """IvbPointGrad: torch gradients of sum(w * f(x)) equal the oracle's point
    gradients, and agree with binary128 central differences (h = 1e-6
    max(1,|x_i|), rel tol 1e-6)"""
    from paper_2507_20769_gb300.autograd import point_values
    t = W.config_tape(2)
    pts = W.sample_points(t.root_box, 16, seed=9)
    x = torch.tensor(pts, dtype=torch.float64, device=DEV, requires_grad=True)
    w = torch.linspace(0.5, 2.0, t.n_out, dtype=torch.float64, device=DEV)
    with ivb.Problem(t) as p:
        f = point_values(p, x)
        (f * w).sum().backward()
    gx = x.grad.cpu().numpy()
    wn = w.cpu().numpy()
    for i in range(pts.shape[0]):
        fo, go = oracle.point_grad(t, pts[i])
        assert np.allclose(f[i].detach().cpu().numpy(), fo, rtol=1e-12, atol=1e-12)
        assert np.allclose(gx[i], wn @ go, rtol=1e-10, atol=1e-12)
        h = 1e-6 * np.maximum(1.0, np.abs(pts[i]))
        gfd = wn @ oracle.central_diff_q(t, pts[i], h)
        assert np.all(np.abs(gx[i] - gfd) <= 1e-6 * np.maximum(1.0, np.abs(gx[i])))


# --------------------------------------------------- other workload configs

def test_config3_uneven_batch_full_size():
    """configuration 3: 256 nodes of uneven widths (10^U[-4,1] per dim) on the
    n=6 problem, per-node subdomain targets 2^U{10..20} split by the adaptive
    picker, one persistent launch. Nodes with <= 2^12 subdomains are checked
    whole against the oracle; 64 sampled subdomains of large nodes one by one."""
    t = W.config_tape(3)
    boxes, targets = W.uneven_nodes(t.n_vars, 256, t.root_box, seed=W.config_seed(3) + 5)
    ref_w = t.root_box[:, 1] - t.root_box[:, 0]
    splits = np.stack([ivb.ivb_pick_splits(b, int(tg), "adaptive", ref_w) for b, tg in zip(boxes, targets)])
    S = np.prod(splits.astype(np.int64), axis=1)
    with ivb.Problem(t) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        small = np.nonzero(S <= 4096)[0][:6]
        ref = oracle.bound_nodes(t, boxes[small], splits[small], tight=True)
        wide = oracle.bound_nodes(t, boxes[small], splits[small], tight=WIDE)
        h = np.stack([r["minlo"][small], r["maxhi"][small]], -1)
        assert_bracketed(h, hull(ref), hull(wide), "config 3 small nodes")
        big = np.argsort(-S)[:4]
        rng = np.random.default_rng(3)
        for nd in big:
            for k in rng.choice(int(S[nd]), 16, replace=False):
                F, _, _ = p.enclose(boxes[nd], splits[nd], first=int(k), count=1)
                assert_enclose_bracketed(t, F, boxes[nd], splits[nd], first=int(k), count=1,
                                         what=f"config 3 large nodes: node {nd} subdomain {k}")
                # the node hull contains every subdomain's enclosure
                assert np.all(r["minlo"][nd] <= F[0, :, 0]) and np.all(r["maxhi"][nd] >= F[0, :, 1])


def test_config5_full_scale_benched_kernel():
    """configuration 5 in the launch bench.py times: 64 frontier nodes x 2^18
    subdomains (2^24, 11 outputs of 1000-entry tapes), one batched launch
    with the library's kernel choice (the segmented tape-specialised kernel),
    autotuned, CUDA graph -- plus four 2^8-subdomain nodes in the same launch.
    The small nodes' hulls and lower bounds are bracketed by the oracle whole;
    on the full-size nodes, the hull contains the oracle's tight enclosure of
    sampled subdomains (it is a minimum / maximum over all of them) and every
    lower bound is finite."""
    t = W.config_tape(5)
    boxes = W.bisection_frontier(t.root_box, 64, seed=2026)
    splits = np.array([W.full_scale_splits(b, t.root_box) for b in boxes], np.int32)
    extra = W.bisection_frontier(t.root_box, 64, seed=55)[:4]
    boxes = np.concatenate([boxes, extra])
    splits = np.concatenate([splits, np.full((4, 8), 2, np.int32)])
    with ivb.Problem(t, specialize=-1, max_nodes=128) as p:
        assert p.get_segmentation()["chunks"] > 0
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, extra, splits[64:], tight=True)
    wide = oracle.bound_nodes(t, extra, splits[64:], tight=WIDE)
    h = np.stack([r["minlo"][64:], r["maxhi"][64:]], -1)
    assert_bracketed(h, hull(ref), hull(wide), "config 5 small nodes in the full-scale launch")
    assert np.all(r["lb"][64:] <= ref["lb"]) and np.all(r["lb"][64:] >= wide["lb"])
    rng = np.random.default_rng(5)
    for nd in rng.choice(64, 4, replace=False):
        ks = rng.choice(1 << 18, 4, replace=False)
        for k in ks:
            Fo, _, _ = oracle.enclose(t, boxes[nd], splits[nd], first=int(k), count=1, tight=True)
            assert np.all(r["minlo"][nd] <= Fo[0, :, 0]) and np.all(r["maxhi"][nd] >= Fo[0, :, 1])
    assert np.all(np.isfinite(r["lb"]))


def test_config5_sampled_subdomains_bracketed():
    """configuration 5 per subdomain (the interpreter's store mode, which the
    segmented kernel matches bit for bit): sampled subdomains of 4^8-split
    nodes between the oracle's tight and 4-step sweeps"""
    t = W.config_tape(5)
    boxes = W.bisection_frontier(t.root_box, 256, seed=55)
    splits = np.full((256, 8), 4, np.int32)
    with ivb.Problem(t, max_nodes=256) as p:
        rng = np.random.default_rng(5)
        for nd in rng.choice(256, 4, replace=False):
            for k in rng.choice(65536, 4, replace=False):
                F, _, _ = p.enclose(boxes[nd], splits[nd], first=int(k), count=1)
                assert_enclose_bracketed(t, F, boxes[nd], splits[nd], first=int(k), count=1,
                                         what=f"config 5 sampled: node {nd} subdomain {k}")
