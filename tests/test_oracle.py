"""Pins for the CPU oracle against what the paper and the mathematics fix
(worked examples, exact rational arithmetic, high-precision evaluation,
closed-form minima, Theorem 1 convergence orders). No GPU needed."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import problems as P
from paper_2507_20769_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = math.inf


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _next_up(x):
    return np.nextafter(x, INF)


def _next_dn(x):
    return np.nextafter(x, -INF)


# ----------------------------------------------------------- Step 1 pins

def test_partition_worked_example():
    """Section 3.1.1: [-3,1]x[0,2] into four subdomains, listed X1..X4."""
    rows = _golden("partition_worked_example.txt")
    box = np.array([float(v) for v in rows[0][1:]]).reshape(2, 2)
    splits = [int(v) for v in rows[1][1:]]
    for r in rows[2:]:
        k = int(r[0])
        X, c = oracle.decode(box, splits, k)
        assert X.ravel().tolist() == [float(v) for v in r[1:]]
        assert c.tolist() == [0.5 * (X[0, 0] + X[0, 1]), 0.5 * (X[1, 0] + X[1, 1])]


def test_adaptive_partition_worked_example():
    """Section 3.1.2: n=5 on 2560 cores -> uniform 4^5=1024, adaptive 5^4*4=2500."""
    g = {r[0]: r[1:] for r in _golden("adaptive_partition_example.txt")}
    n, target = int(g["n"][0]), int(g["target"][0])
    box = [[0.0, 1.0]] * n
    uni = oracle.pick_splits(box, target, "uniform")
    assert uni.tolist() == [int(v) for v in g["uniform"]]
    assert int(np.prod(uni)) == int(g["uniform_count"][0])
    ada = oracle.pick_splits(box, target, "adaptive")
    assert ada.tolist() == [int(v) for v in g["adaptive"]]
    assert int(np.prod(ada)) == int(g["adaptive_count"][0])


def test_largest_and_adaptive_follow_widths():
    """Largest: only the widest dimension is split; adaptive grows wide dims first."""
    box = [[0, 1], [0, 8], [0, 2]]
    assert oracle.pick_splits(box, 100, "largest").tolist() == [1, 100, 1]
    ada = oracle.pick_splits(box, 100, "adaptive")
    assert int(np.prod(ada)) <= 100 and ada[1] >= ada[2] >= ada[0]
    assert oracle.pick_splits(box, 1, "adaptive").tolist() == [1, 1, 1]


@pytest.mark.parametrize("seed", range(6))
def test_partition_covers_box(seed):
    """Section 2.2 splitting: union of X_k is X; neighbours share endpoints,
    the end subdomains reach lo and hi exactly, c lies in X_k."""
    rng = np.random.default_rng(seed)
    n = 3
    lo = rng.uniform(-10, 10, n)
    w = 10.0 ** rng.uniform(-12, 1, n)
    box = np.stack([lo, lo + w], 1)
    splits = rng.integers(1, 9, n).astype(np.int32)
    S = int(np.prod(splits))
    Xs = [oracle.decode(box, splits, k) for k in range(S)]
    for k, (X, c) in enumerate(Xs):
        assert np.all(X[:, 0] <= X[:, 1])
        assert np.all(box[:, 0] <= X[:, 0]) and np.all(X[:, 1] <= box[:, 1])
        assert np.all(X[:, 0] <= c) and np.all(c <= X[:, 1])
        j = k
        for i in range(n):
            ji = j % splits[i]
            j //= splits[i]
            if ji == 0:
                assert X[i, 0] == box[i, 0]
            if ji == splits[i] - 1:
                assert X[i, 1] == box[i, 1]
            else:  # neighbour along i shares the endpoint bit for bit
                stride = int(np.prod(splits[:i]))
                assert Xs[k + stride][0][i, 0] == X[i, 1]


# ------------------------------------------------ interval operation pins

def _rand_dyadic_intervals(rng, m, scale=8):
    a = rng.integers(-scale * 4, scale * 4, (m, 2)) / 4.0
    a.sort(axis=1)
    return a


def _special_intervals():
    v = [0.0, -0.0, 1.0, -1.0, 2.5, -3.25]
    out = [[x, y] for x in v for y in v if x <= y]
    out += [[-INF, INF], [0.0, INF], [-INF, 0.0], [1.0, INF], [-INF, -2.0]]
    return np.array(out)


def _hull(vals):
    return min(vals), max(vals)


def _check_tight(lo, hi, exact_lo: Fraction, exact_hi: Fraction):
    """lo = largest double <= exact_lo and hi = smallest double >= exact_hi"""
    assert Fraction(lo) <= exact_lo < Fraction(_next_up(lo)) or (Fraction(lo) == exact_lo)
    assert Fraction(_next_dn(hi)) < exact_hi <= Fraction(hi) or (Fraction(hi) == exact_hi)


@pytest.mark.parametrize("opcode", [W.OP_ADD, W.OP_SUB, W.OP_MUL, W.OP_DIV])
def test_binary_ops_exact_rational(opcode):
    """Natural interval extension of + - * / (Section 2.2) with outward rounding:
    on random operands the endpoints are the tightest doubles around the exact
    rational hull of the endpoint results (all sign cases, inexact quotients)."""
    rng = np.random.default_rng(100 + opcode)
    X = rng.uniform(-5, 5, (400, 2)); X.sort(1)
    Y = rng.uniform(-5, 5, (400, 2)); Y.sort(1)
    # sign cases: make a third of the operands one-signed
    X[::3] = np.abs(X[::3]); X[::3].sort(1)
    Y[1::3] = -np.abs(Y[1::3]); Y[1::3].sort(1)
    R = oracle.iv_op(opcode, X, Y)
    for (xl, xh), (yl, yh), (rl, rh) in zip(X, Y, R):
        fx = [Fraction(xl), Fraction(xh)]
        fy = [Fraction(yl), Fraction(yh)]
        if opcode == W.OP_ADD:
            ex = (fx[0] + fy[0], fx[1] + fy[1])
        elif opcode == W.OP_SUB:
            ex = (fx[0] - fy[1], fx[1] - fy[0])
        elif opcode == W.OP_MUL:
            ex = _hull([p * q for p in fx for q in fy])
        else:
            if yl <= 0 <= yh:
                assert (rl, rh) == (-INF, INF)
                continue
            ex = _hull([p / q for p in fx for q in fy])
        _check_tight(rl, rh, *ex)


def test_fused_accumulation_exact_rational():
    """acc + x*y with one directed rounding per end (the adjoint accumulation,
    tangent rules and Mean Value Form sum): on random operands of every sign
    case the ends are the tightest doubles around acc.lo + min and acc.hi + max
    of the exact endpoint products -- which a rounding after the product
    (unfused) misses on part of these operands"""
    rng = np.random.default_rng(105)
    X = rng.uniform(-5, 5, (600, 2)); X.sort(1)
    Y = rng.uniform(-5, 5, (600, 2)); Y.sort(1)
    Z = rng.uniform(-50, 50, (600, 2)); Z.sort(1)
    X[::3] = np.abs(X[::3]); X[::3].sort(1)
    Y[1::3] = -np.abs(Y[1::3]); Y[1::3].sort(1)
    X[2::7, 0] = 0.0                                   # zero endpoints
    R = oracle.iv_fma(X, Y, Z)
    unfused = oracle.iv_op(W.OP_ADD, Z, oracle.iv_op(W.OP_MUL, X, Y))
    differs = 0
    for (xl, xh), (yl, yh), (zl, zh), (rl, rh), u in zip(X, Y, Z, R, unfused):
        P = [Fraction(p) * Fraction(q) for p in (xl, xh) for q in (yl, yh)]
        _check_tight(rl, rh, Fraction(zl) + min(P), Fraction(zh) + max(P))
        differs += (rl, rh) != tuple(u)
    assert differs > 20


def test_fused_accumulation_special_cases():
    """zero factors add an exact zero (0 * inf = 0), -0 + 0 rounds up to +0,
    infinite products, and an addend of zero gives the directed product"""
    fma = lambda x, y, z: oracle.iv_fma([x], [y], [z])[0].tolist()
    assert fma([0.0, 0.0], [-INF, INF], [1.0, 2.0]) == [1.0, 2.0]
    r = fma([0.0, 0.0], [3.0, 4.0], [-0.0, -0.0])
    assert r == [0.0, 0.0] and np.signbit(r[0]) and not np.signbit(r[1])
    assert fma([1.0, INF], [1.0, 2.0], [0.0, 1.0]) == [1.0, INF]
    assert fma([-1.0, 1.0], [-INF, INF], [0.0, 0.0]) == [-INF, INF]
    third = oracle.iv_op(W.OP_DIV, [[1.0, 1.0]], [[3.0, 3.0]])[0].tolist()
    assert fma([1.0, 1.0], third, [0.0, 0.0]) == third
    p = oracle.iv_op(W.OP_MUL, [[0.1, 0.3]], [[-0.7, 0.9]])[0].tolist()
    assert fma([0.1, 0.3], [-0.7, 0.9], [0.0, 0.0]) == p


def test_textbook_values():
    """Exact textbook results on representable operands."""
    iv = lambda op, x, y=None: oracle.iv_op(op, [x], None if y is None else [y])[0].tolist()
    assert iv(W.OP_MUL, [1, 2], [-3, 4]) == [-6, 8]
    assert iv(W.OP_MUL, [-2, -1], [-3, 4]) == [-8, 6]
    assert iv(W.OP_MUL, [-2, 3], [-5, 4]) == [-15, 12]
    assert iv(W.OP_DIV, [1, 2], [4, 8]) == [0.125, 0.5]
    assert iv(W.OP_DIV, [-1, 2], [-4, -2]) == [-1, 0.5]
    assert iv(W.OP_SQR, [-3, 2]) == [0, 9]
    assert iv(W.OP_SQR, [-3, -2]) == [4, 9]
    assert iv(W.OP_SQRT, [4, 9]) == [2, 3]
    assert iv(W.OP_NEG, [-1, 3]) == [-3, 1]
    assert iv(W.OP_SUB, [1, 2], [1, 2]) == [-1, 1]          # dependency effect of NIE
    assert iv(W.OP_LOG, [1, 1]) == [0, 0]
    e = iv(W.OP_EXP, [0, 0])                                # enclosure of 1, one ulp each side
    assert e[0] <= 1.0 <= e[1] and e[0] >= np.nextafter(1.0, 0) and e[1] <= np.nextafter(1.0, 2)


def test_domain_rules_and_zero_times_inf():
    """Domain exits give ENTIRE; a zero factor times an unbounded one is zero."""
    iv = lambda op, x, y=None: oracle.iv_op(op, [x], None if y is None else [y])[0].tolist()
    assert iv(W.OP_SQRT, [-1, 4]) == [-INF, INF]
    assert iv(W.OP_LOG, [0, 4]) == [-INF, INF]
    assert iv(W.OP_LOG, [-3, -1]) == [-INF, INF]
    assert iv(W.OP_DIV, [1, 2], [-1, 1]) == [-INF, INF]
    assert iv(W.OP_DIV, [1, 2], [0, 1]) == [-INF, INF]
    assert iv(W.OP_MUL, [0, 0], [-INF, INF]) == [0, 0]
    assert iv(W.OP_MUL, [0, 1], [1, INF]) == [0, INF]
    assert iv(W.OP_SQRT, [0, 4]) == [0, 2]
    e = iv(W.OP_EXP, [-INF, 0])
    assert e[0] == 0.0 and 1.0 <= e[1] <= np.nextafter(1.0, 2)


def test_special_operand_sign_cases_match_brute_force():
    """Products over intervals with zero and infinite endpoints equal the hull
    of the endpoint products under 0 * inf = 0 (set semantics)."""
    S = _special_intervals()
    X = np.repeat(S, len(S), axis=0)
    Y = np.tile(S, (len(S), 1))
    R = oracle.iv_op(W.OP_MUL, X, Y)

    def p(u, v):
        return 0.0 if (u == 0 or v == 0) else u * v
    for x, y, r in zip(X, Y, R):
        prods = [p(u, v) for u in x for v in y]
        assert r[0] == min(prods) and r[1] == max(prods), (x, y, r)


def test_sqrt_tight():
    rng = np.random.default_rng(7)
    X = rng.uniform(0, 100, (300, 2)); X.sort(1)
    R = oracle.iv_op(W.OP_SQRT, X)
    for (xl, xh), (rl, rh) in zip(X, R):
        assert Fraction(rl) ** 2 <= Fraction(xl) < Fraction(_next_up(rl)) ** 2
        assert Fraction(_next_dn(rh)) ** 2 < Fraction(xh) <= Fraction(rh) ** 2


@pytest.mark.parametrize("fn", ["exp", "log"])
def test_transcendental_enclosure_one_ulp(fn):
    """Tight exp/log enclose the true value (mpmath, 50 digits) with each end at
    most one ulp away; the fast mode encloses it within three ulps."""
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    if fn == "exp":
        x = np.concatenate([rng.uniform(-30, 30, 400), rng.uniform(-700, 700, 100), [0.0, 1.0, -745.5, 709.7]])
        lo, hi = oracle.exp_enclose(x, tight=True)
        flo, fhi = oracle.exp_enclose(x, tight=False)
    else:
        x = np.concatenate([10.0 ** rng.uniform(-300, 300, 400), rng.uniform(0.5, 2, 100), [1.0, 2.0]])
        lo, hi = oracle.log_enclose(x, tight=True)
        flo, fhi = oracle.log_enclose(x, tight=False)
    with mpmath.workdps(50):
        for xi, l, h, fl, fh in zip(x, lo, hi, flo, fhi):
            t = mpmath.exp(mpmath.mpf(float(xi))) if fn == "exp" else mpmath.log(mpmath.mpf(float(xi)))
            assert mpmath.mpf(float(l)) <= t <= mpmath.mpf(float(h))
            assert mpmath.mpf(float(fl)) <= t <= mpmath.mpf(float(fh))
            if t != 0 and abs(t) > 1e-300:
                assert mpmath.mpf(float(_next_up(l))) >= t or l == 0.0  # lower end within one step
                assert mpmath.mpf(float(_next_dn(h))) <= t              # upper end within one step


@pytest.mark.parametrize("fn", ["exp", "log"])
@pytest.mark.parametrize("k", [2, 5])
def test_widened_bracket_is_k_minus_1_steps_beyond_tight(fn, k):
    """tight=k > 1 moves each tight end exactly k-1 representable steps
    outward (the exp lower end stays >= 0), counted here with numpy's own
    nextafter, and still encloses the true value"""
    rng = np.random.default_rng(12 + k)
    if fn == "exp":
        x = np.concatenate([rng.uniform(-30, 30, 300), [0.0, 1.0, -745.5, -800.0, 709.7, 710.0]])
        lo, hi = oracle.exp_enclose(x, tight=True)
        wlo, whi = oracle.exp_enclose(x, tight=k)
    else:
        x = np.concatenate([10.0 ** rng.uniform(-300, 300, 300), [1.0, 2.0, 0.5]])
        lo, hi = oracle.log_enclose(x, tight=True)
        wlo, whi = oracle.log_enclose(x, tight=k)
    elo, ehi = lo.copy(), hi.copy()
    for _ in range(k - 1):
        elo = np.nextafter(elo, -np.inf)
        ehi = np.nextafter(ehi, np.inf)
    if fn == "exp":
        elo = np.maximum(elo, 0.0)
    assert np.array_equal(wlo, elo) and np.array_equal(whi, ehi)
    assert np.all(wlo <= lo) and np.all(whi >= hi)


@pytest.mark.parametrize("config", [1, 2])
def test_widened_sweep_brackets_tight_sweep(config):
    """every operation other than exp/log is the same in both modes, so by
    isotonicity (Definition 2) the per-subdomain enclosures of the tight=5
    sweep contain the tight ones (F, f(c) and G), and a tape without exp/log
    gives identical bits"""
    t = W.config_tape(config)
    box = W.bisection_frontier(t.root_box, 4, seed=config)[1]
    splits = np.array([3] * t.n_vars, np.int32)
    F, Fc, G = oracle.enclose(t, box, splits, tight=True, want_fc=True, want_g=True)
    F5, Fc5, G5 = oracle.enclose(t, box, splits, tight=5, want_fc=True, want_g=True)
    for a, b in ((F, F5), (Fc, Fc5), (G, G5)):
        assert np.all(b[..., 0] <= a[..., 0]) and np.all(b[..., 1] >= a[..., 1])
    assert not np.array_equal(F, F5)
    r = W.random_problem(3, 40, 1, W.OPS_RATIONAL, [[-2, 2]] * 3, 4242, "rational")
    Fr, _, Gr = oracle.enclose(r, r.root_box, [3, 2, 4], tight=True, want_g=True)
    Fr5, _, Gr5 = oracle.enclose(r, r.root_box, [3, 2, 4], tight=5, want_g=True)
    assert np.array_equal(Fr, Fr5) and np.array_equal(Gr, Gr5)


# ------------------------------------------------------------ tape sweeps

def test_cubic_fig5_nie_textbook():
    """Fig. 5: natural interval extension of 3x^3+x^2-5x-1 on [-1,2] is [-23,32]
    (hand-computed, every operation exact) and encloses the exact range."""
    g = {r[0]: r[1:] for r in _golden("cubic_fig5.txt")}
    T = P.cubic_fig5()
    X = np.array([[float(v) for v in g["X"]]])
    V = oracle.value_sweep(T, X)
    assert V[T.out_idx[0]].tolist() == [float(v) for v in g["nie"]]
    lo, hi = P.cubic_range(X[0, 0], X[0, 1])
    assert V[T.out_idx[0], 0] <= lo and hi <= V[T.out_idx[0], 1]


def _excess(T, box, N, form, grad_mode="adjoint"):
    F, _, _ = oracle.enclose(T, box, [N], grad_mode=grad_mode, form=form)
    lo, hi = P.cubic_range(box[0][0], box[0][1])
    return (F[:, 0, 1].max() - F[:, 0, 0].min()) - (hi - lo)


def test_theorem1_convergence_orders():
    """Theorem 1: refinement excess width is O(w/N) for NIE and O((w/N)^2) for
    the Mean Value Form: doubling N halves NIE excess and quarters MVF excess."""
    T = P.cubic_fig5()
    box = [[-1.0, 2.0]]
    for form, lo_r, hi_r in (("nie", 1.8, 2.2), ("mvf", 3.5, 4.5)):
        e = [_excess(T, box, N, form) for N in (64, 128, 256)]
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert lo_r < r1 < hi_r and lo_r < r2 < hi_r, (form, e)


def test_mvf_definition_on_one_subdomain():
    """Definition 5 on a box where every operation is exact: f(c) + f'(X)(X-c)."""
    T = P.cubic_fig5()
    # X = [0, 1], c = 0.5: f(c) = 3/8 + 1/4 - 5/2 - 1 = -2.875
    # f'(X) by tangents: 3*(x*x*x)' = 3*((x*x)*1 + (x*x)'*x) ... computed by hand:
    # (x*x)' = 1*X + X*1 = [0,2]; (x*x*x)' = [0,2]*X + (x*x)*1 = [0,2]+[0,1] = [0,3]
    # 3*(.)' = [0,9]; (x^2)' = 2X*1 = [0,2]; sum = [0,11]; (5x)' = [5,5]; f' = [-5,6]
    # MVF = -2.875 + [-5,6]*[-0.5,0.5] = -2.875 + [-3,3] = [-5.875, 0.125]
    F, Fc, G = oracle.enclose(T, [[0.0, 1.0]], [1], grad_mode="forward", want_fc=True, want_g=True)
    assert Fc[0, 0].tolist() == [-2.875, -2.875]
    assert G[0, 0, 0].tolist() == [-5.0, 6.0]
    assert F[0, 0].tolist() == [-5.875, 0.125]


def _inside(v, iv_):
    return iv_[0] <= v <= iv_[1]


@pytest.mark.parametrize("config", [1, 2, 4])
@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_inclusion_of_sampled_values_and_gradients(config, grad_mode):
    """Definition 1 (inclusion): on random subdomains the MVF enclosure, the
    point enclosure f(c) and the gradient enclosure contain values and gradients
    evaluated independently in mpmath at points sampled in X_k."""
    mpmath = pytest.importorskip("mpmath")
    T = W.config_tape(config)
    rng = np.random.default_rng(config)
    nodes = W.bisection_frontier(T.root_box, 6, seed=config)
    for nd in nodes[:3]:
        splits = np.full(T.n_vars, 3 if T.n_vars <= 4 else 1, np.int32)
        S = int(np.prod(splits))
        ks = rng.integers(0, S, 2)
        for k in ks:
            F, Fc, G = oracle.enclose(T, nd, splits, first=int(k), count=1, grad_mode=grad_mode,
                                      want_fc=True, want_g=True)
            X, c = oracle.decode(nd, splits, int(k))
            fcv = P.mp_eval(T, c, dps=40)
            for o in range(T.n_out):
                assert mpmath.mpf(float(Fc[0, o, 0])) <= fcv[o] <= mpmath.mpf(float(Fc[0, o, 1]))
            for _ in range(4):
                x = rng.uniform(X[:, 0], X[:, 1])
                fv, gv = P.mp_eval(T, x, dps=40, grad=True)
                for o in range(T.n_out):
                    assert mpmath.mpf(float(F[0, o, 0])) <= fv[o] <= mpmath.mpf(float(F[0, o, 1]))
                    for i in range(T.n_vars):
                        assert mpmath.mpf(float(G[0, o, i, 0])) <= gv[o][i] <= mpmath.mpf(float(G[0, o, i, 1]))


@pytest.mark.parametrize("config", [1, 2, 3])
def test_isotonicity_of_nie_and_gradients(config):
    """Definition 2 (inclusion isotonicity): Y in X implies F(Y) in F(X), for the
    natural extension of every node and for both gradient enclosures; the
    degenerate [x,x] is the extreme case (Definition 3)."""
    T = W.config_tape(config)
    rng = np.random.default_rng(30 + config)
    X = T.root_box.copy()
    for _ in range(3):
        w = X[:, 1] - X[:, 0]
        lo = X[:, 0] + rng.uniform(0, 0.5, T.n_vars) * w
        Y = np.stack([lo, lo + rng.uniform(0, 0.5, T.n_vars) * w], 1)
        x = rng.uniform(Y[:, 0], Y[:, 1])
        Z = np.stack([x, x], 1)
        VX, VY, VZ = (oracle.value_sweep(T, B) for B in (X, Y, Z))
        assert np.all(VX[:, 0] <= VY[:, 0]) and np.all(VY[:, 1] <= VX[:, 1])
        assert np.all(VY[:, 0] <= VZ[:, 0]) and np.all(VZ[:, 1] <= VY[:, 1])
        for gm in ("forward", "adjoint"):
            GX, GY = oracle.gradient(T, X, gm), oracle.gradient(T, Y, gm)
            assert np.all(GX[..., 0] <= GY[..., 0]) and np.all(GY[..., 1] <= GX[..., 1])
        X = Y


def test_brute_force_minimum_tiny_grid():
    """n=2, 16x16 subdomains: the refinement lower end is below every sampled
    value (10^6 points), and the gap closes as the grid is refined."""
    T = W.config_tape(1)
    box = T.root_box
    g = np.linspace(box[0, 0], box[0, 1], 1001)
    h = np.linspace(box[1, 0], box[1, 1], 1001)
    XX, YY = np.meshgrid(g, h)
    vals = P.np_eval(T, np.stack([XX.ravel(), YY.ravel()], 1))[:, 0]
    fmin = vals.min()
    gaps = []
    for N in (16, 32, 64):
        r = oracle.bound_nodes(T, box[None], [N, N], grad_mode="forward")
        assert r["lb"][0] <= fmin
        gaps.append(fmin - r["lb"][0])
    assert gaps[0] > gaps[1] > gaps[2]


def test_shifted_squares_lb_converges_to_zero():
    """sum (x_i - a_i)^2 with a in the box: lower bound <= 0 and -> 0 as the
    subdomains shrink (quadratically for the MVF)."""
    a = [0.3, -1.1, 0.7]
    T = P.shifted_squares(3, a, [[-2, 2]] * 3)
    lbs = [oracle.bound_nodes(T, T.root_box[None], [N] * 3)["lb"][0] for N in (4, 8, 16)]
    assert all(v <= 0 for v in lbs)
    assert -lbs[0] > -lbs[1] > -lbs[2]
    assert 3.0 < lbs[0] / lbs[1] < 5.0


def test_point_sweep_is_exact_for_exact_tapes():
    """Interval extension (Definition 3): F([x,x]) = f(x) when no rounding occurs."""
    T = P.shifted_squares(2, [0.5, -0.25], [[-2, 2]] * 2)
    V = oracle.value_sweep(T, [[1.0, 1.0], [0.5, 0.5]])
    assert V[T.out_idx[0]].tolist() == [0.25 + 0.5625, 0.25 + 0.5625]


# ----------------------------------------------------- feasibility pins

def test_feasibility_flags():
    """Section 3.1 pruning: an inequality is violated when its refinement lower
    end is > 0; an equality when 0 is outside its refinement."""
    box = np.array([[-2.0, 2.0], [-2.0, 2.0]])
    for kind, expect in (("feasible", False), ("infeasible", True), ("eq_out", True), ("eq_in", False)):
        T = P.constrained_toy(kind)
        r = oracle.bound_nodes(T, box[None], [8, 8])
        assert bool(r["infeasible"][0]) is expect, kind
        assert r["lb"][0] <= -4.0                 # objective x0+x1 on the box
    # the feasible toy: the certified centre upper bound is a feasible value
    T = P.constrained_toy("feasible")
    r = oracle.bound_nodes(T, box[None], [8, 8])
    assert -math.sqrt(2) - 1e-12 <= r["ub"][0] < 0.0
    # a node outside the unit disc is infeasible
    r = oracle.bound_nodes(T, np.array([[[1.5, 2.0], [1.5, 2.0]]]), [4, 4])
    assert r["infeasible"][0]


def test_filter_never_loosens():
    T = P.constrained_toy("feasible")
    box = np.array([[[-2.0, 2.0], [-2.0, 2.0]]])
    r0 = oracle.bound_nodes(T, box, [16, 16])
    r1 = oracle.bound_nodes(T, box, [16, 16], filter=True)
    assert r1["lb"][0] >= r0["lb"][0]
    assert r1["lb"][0] <= -math.sqrt(2) + 1e-12        # true constrained minimum -sqrt(2)


# ----------------------------------------------------- Peaks (Section 4.1)

def test_peaks_bounds_and_mvf_vs_nie():
    """Section 4.1 / Fig. 6a: more subdomains give tighter root lower bounds;
    MVF is looser than NIE with few subdomains and tighter with many."""
    T = P.peaks()
    g = np.linspace(-3, 3, 1201)
    XX, YY = np.meshgrid(g, g)
    fmin = P.peaks_np(XX, YY).min()
    root = T.root_box[None]
    lb = {}
    for form in ("mvf", "nie"):
        for N in (2, 8, 32, 128):
            lb[form, N] = oracle.bound_nodes(T, root, [N, N], form=form)["lb"][0]
            assert lb[form, N] <= fmin
    for form in ("mvf", "nie"):
        assert lb[form, 2] < lb[form, 8] < lb[form, 32] < lb[form, 128]
    assert lb["mvf", 2] < lb["nie", 2]
    assert lb["mvf", 128] > lb["nie", 128]


# ----------------------------------------------------- point gradients

@pytest.mark.parametrize("config", [1, 2, 4])
def test_point_gradient_matches_mpmath_and_central_differences(config):
    """RN point gradient vs independent mpmath derivatives (rel 1e-9) and vs
    binary128 central differences, h = 1e-6 max(1,|x_i|), rel tol 1e-6."""
    pytest.importorskip("mpmath")
    T = W.config_tape(config)
    pts = W.sample_points(T.root_box, 4, seed=config)
    for x in pts:
        f, g = oracle.point_grad(T, x)
        fv, gv = P.mp_eval(T, x, dps=40, grad=True)
        h = 1e-6 * np.maximum(1.0, np.abs(x))
        gfd = oracle.central_diff_q(T, x, h)
        for o in range(T.n_out):
            assert abs(f[o] - float(fv[o])) <= 1e-9 * max(1.0, abs(float(fv[o])))
            for i in range(T.n_vars):
                gi = float(gv[o][i])
                assert abs(g[o, i] - gi) <= 1e-9 * max(1.0, abs(gi))
                assert abs(g[o, i] - gfd[o, i]) <= 1e-6 * max(1.0, abs(g[o, i]))


# ----------------------------------------------------------------- B&B

def test_bnb_shifted_squares_converges_to_zero():
    T = P.shifted_squares(2, [0.3, -1.1], [[-2, 2]] * 2)
    r = oracle.bnb(T, splits=[8, 8], eps_abs=1e-6, eps_rel=0.0, grad_mode="forward", max_nodes=20000)
    assert r["converged"]
    assert r["lb"] <= 0.0 <= r["ub"] and r["ub"] - r["lb"] <= 1e-6


def test_bnb_separable_quartic_closed_form():
    n = 2
    T = P.separable_quartic(n, [[-2, 2]] * n)
    fstar = n * P.quartic_min_1d(-2.0, 2.0)
    r = oracle.bnb(T, splits=[8, 8], eps_abs=1e-6, eps_rel=0.0, grad_mode="adjoint", max_nodes=20000)
    assert r["converged"]
    assert r["lb"] - 1e-12 <= fstar <= r["ub"] + 1e-12
    assert r["ub"] - r["lb"] <= 1e-6


def test_bnb_tiny_config_against_grid():
    """Config 1 (tiny): B&B to absolute gap 1e-4 brackets the dense-grid minimum."""
    wl = W.config_workload(1)
    T = wl.tape
    r = oracle.bnb(T, splits=wl.splits, eps_abs=wl.gap_abs, eps_rel=0.0, grad_mode="forward", max_nodes=50000)
    assert r["converged"] and r["ub"] - r["lb"] <= wl.gap_abs
    g = np.linspace(-2, 2, 2001)
    XX, YY = np.meshgrid(g, g)
    vals = P.np_eval(T, np.stack([XX.ravel(), YY.ravel()], 1))[:, 0]
    assert r["lb"] <= vals.min()
    assert r["ub"] >= r["lb"]


def test_generator_is_deterministic_and_sized():
    """the seeded generator gives identical tapes and exact entry counts"""
    for cfg, n_ops in ((1, 20), (2, 4 + 4 * 56), (4, 400)):
        t1, t2 = W.config_tape(cfg), W.config_tape(cfg)
        assert t1.n_ops == n_ops
        assert np.array_equal(t1.op, t2.op) and np.array_equal(t1.c, t2.c)
        assert np.array_equal(t1.a, t2.a) and np.array_equal(t1.b, t2.b)
        # operands refer to earlier entries only
        idx = np.arange(t1.n_ops)
        interior = t1.op >= W.OP_ADD
        assert np.all(t1.a[interior] < idx[interior])
        assert np.all(t1.b[interior] < idx[interior])
    assert W.Xoshiro256ss(1).next_u64() == W.Xoshiro256ss(1).next_u64()


# ------------------------------------------------ constraint propagation

def _toy(n, build, box):
    B = P.Builder(n)
    build(B, [B.x(i) for i in range(n)])
    return B.tape(box, "toy")


def test_propagation_closed_forms():
    """hand-derived tightenings: the unit disc, a linear cut, an equality,
    an objective cut, an impossible constraint"""
    def disc(B, x):
        B.output(B.add(x[0], x[1]), P.KIND_OBJ)
        B.output(B.sub(B.add(B.sqr(x[0]), B.sqr(x[1])), B.const(1.0)), P.KIND_INEQ)
    t = _toy(2, disc, [[-2.0, 2.0], [-2.0, 2.0]])
    bx, inf = oracle.propagate(t, t.root_box)
    assert not inf[0] and np.array_equal(bx[0], [[-1.0, 1.0], [-1.0, 1.0]])

    def cut(B, x):   # x0 + x1 + 3 <= 0 on [-2, 2]^2: both in [-2, -1]
        B.output(B.mul(x[0], x[1]), P.KIND_OBJ)
        B.output(B.add(B.add(x[0], x[1]), B.const(3.0)), P.KIND_INEQ)
    t = _toy(2, cut, [[-2.0, 2.0], [-2.0, 2.0]])
    bx, inf = oracle.propagate(t, t.root_box)
    assert not inf[0] and np.array_equal(bx[0], [[-2.0, -1.0], [-2.0, -1.0]])

    def eq(B, x):    # x0 - x1 = 0 on [0, 2] x [1, 3]: both in [1, 2]
        B.output(B.add(x[0], x[1]), P.KIND_OBJ)
        B.output(B.sub(x[0], x[1]), P.KIND_EQ)
    t = _toy(2, eq, [[0.0, 2.0], [1.0, 3.0]])
    bx, inf = oracle.propagate(t, t.root_box)
    assert not inf[0] and np.array_equal(bx[0], [[1.0, 2.0], [1.0, 2.0]])

    def obj(B, x):   # f = x0 (a variable entry), cut f <= 0.5
        B.output(x[0], P.KIND_OBJ)
    t = _toy(1, obj, [[-1.0, 1.0]])
    bx, inf = oracle.propagate(t, t.root_box, ub=0.5)
    assert not inf[0] and np.array_equal(bx[0], [[-1.0, 0.5]])
    bx, inf = oracle.propagate(t, t.root_box, ub=-2.0)
    assert inf[0]

    def never(B, x):  # x0^2 + 1 <= 0 has no solution
        B.output(x[0], P.KIND_OBJ)
        B.output(B.add(B.sqr(x[0]), B.const(1.0)), P.KIND_INEQ)
    t = _toy(1, never, [[-3.0, 3.0]])
    assert oracle.propagate(t, t.root_box)[1][0]


def test_propagation_through_exp_log_div_sqrt():
    """exp(x0) <= 2 gives x0 <= log 2 (within the widening); log(x0) >= 1
    gives x0 >= e; x0 / x1 <= 1 with x1 in [1, 2] gives x0 <= 2;
    sqrt(x0) <= 3 gives x0 <= 9"""
    def f(B, x):
        B.output(B.add(x[0], x[1]), P.KIND_OBJ)
        B.output(B.sub(B.exp(x[0]), B.const(2.0)), P.KIND_INEQ)
    t = _toy(2, f, [[-3.0, 3.0], [-1.0, 1.0]])
    bx, _ = oracle.propagate(t, t.root_box)
    assert math.log(2.0) <= bx[0, 0, 1] <= math.log(2.0) * (1 + 8e-16) and bx[0, 0, 0] == -3.0

    def g(B, x):
        B.output(x[0], P.KIND_OBJ)
        B.output(B.sub(B.const(1.0), B.log(x[0])), P.KIND_INEQ)
    t = _toy(1, g, [[0.5, 10.0]])
    bx, _ = oracle.propagate(t, t.root_box)
    assert math.e * (1 - 8e-16) <= bx[0, 0, 0] <= math.e and bx[0, 0, 1] == 10.0

    def h(B, x):
        B.output(x[0], P.KIND_OBJ)
        B.output(B.sub(B.div(x[0], x[1]), B.const(1.0)), P.KIND_INEQ)
        B.output(B.sub(B.sqrt(B.add(x[0], B.const(5.0))), B.const(3.0)), P.KIND_INEQ)
    t = _toy(2, h, [[-4.0, 10.0], [1.0, 2.0]])
    bx, _ = oracle.propagate(t, t.root_box)
    assert bx[0, 0, 1] == 2.0 and bx[0, 1].tolist() == [1.0, 2.0]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_propagation_is_sound_on_sampled_points(seed):
    """brute force: every sampled point that certainly satisfies the
    constraints (and f <= ub) lies in the tightened box, boxes declared
    infeasible hold no such point, and no box grows"""
    t = W.random_problem(3, 60, 2, W.OPS_ALL, [[-3, 2]] * 3, 300 + seed, "sound")
    rng = np.random.default_rng(seed)
    boxes = W.bisection_frontier(t.root_box, 40, seed=seed)
    pts = np.concatenate([rng.uniform(boxes[:, :, 0][:, None, :], boxes[:, :, 1][:, None, :], (40, 400, 3))])
    vals = P.np_eval(t, pts.reshape(-1, 3)).reshape(40, 400, -1)
    ineq = [q for q in range(t.n_out) if t.out_kind[q] == W.KIND_INEQ]
    obj = [q for q in range(t.n_out) if t.out_kind[q] == W.KIND_OBJ][0]
    ub = float(np.median(vals[:, :, obj]))
    bx, inf = oracle.propagate(t, boxes, ub=ub)
    assert np.all(bx[:, :, 0] >= boxes[:, :, 0]) and np.all(bx[:, :, 1] <= boxes[:, :, 1])
    scale = 1e-9 * (1 + np.abs(vals))
    good = np.all(vals[:, :, ineq] <= -scale[:, :, ineq], axis=2) & (vals[:, :, obj] <= ub - scale[:, :, obj])
    assert good.sum() > 50   # the check has teeth
    for k in range(40):
        p = pts[k][good[k]]
        if inf[k]:
            assert len(p) == 0
        else:
            assert np.all(p >= bx[k, :, 0]) and np.all(p <= bx[k, :, 1])
    assert inf.sum() + (bx != boxes).any(axis=(1, 2)).sum() > 0   # and propagation did something


def test_bnb_with_propagation_brackets_closed_form_minima():
    """the oracle B&B with propagation still brackets the known minima"""
    T = P.shifted_squares(2, [0.3, -1.1], [[-2, 2]] * 2)
    r = oracle.bnb(T, splits=[8, 8], eps_abs=1e-6, eps_rel=0.0, grad_mode="adjoint", max_nodes=20000, propagate=3)
    assert r["converged"] and r["lb"] <= 0.0 <= r["ub"] and r["ub"] - r["lb"] <= 1e-6
    t = P.constrained_toy("feasible")   # min x0 + x1 on the unit disc: -sqrt(2)
    r = oracle.bnb(t, splits=[6, 6], eps_abs=1e-6, eps_rel=0.0, grad_mode="adjoint", max_nodes=50000, propagate=3)
    assert r["converged"] and r["lb"] - 1e-12 <= -math.sqrt(2.0) <= r["ub"] + 1e-12
    t = P.constrained_toy("infeasible")
    r = oracle.bnb(t, splits=[6, 6], eps_abs=1e-6, eps_rel=0.0, propagate=3)
    assert r["converged"] and r["lb"] == math.inf and r["nodes"] == 0
