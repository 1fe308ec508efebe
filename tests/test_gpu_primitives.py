"""The kernels' interval operations (through the C-ABI test hook ivb_eval_op)
against the oracle's, on large sets of random and special operands:
+ - * / sqr sqrt and the reciprocal bit for bit (directed rounding is unique);
exp and log contain the oracle's tight enclosure, each end within 4 ulps;
+ - * sqr with the integer-pipe emulation of the endpoint operations bit for
bit, signed zeros included."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_20769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_20769_gb300 import build as B  # noqa: E402

B.build()
from paper_2507_20769_gb300 import ivb  # noqa: E402

DEV = torch.device("cuda:0")
RECIP = 100


def random_doubles(rng, n, emin=-1074, emax=1023, sign=True):
    """finite doubles with log-uniform magnitudes over [2^emin, 2^emax]"""
    e = rng.uniform(emin, emax, n)
    m = rng.uniform(1.0, 2.0, n)
    v = np.ldexp(m, np.floor(e).astype(np.int64))
    if sign:
        v *= rng.choice([-1.0, 1.0], n)
    return v


def specials():
    tiny = np.nextafter(0.0, 1.0)
    big = np.finfo(np.float64).max
    v = [0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0, 1.5, tiny, -tiny, big, -big, 2.0 ** -1022, 2.0 ** 1023,
         np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), np.nextafter(2.0, 0.0), np.nextafter(0.5, 1.0), 1.0 / 3.0]
    return np.array(v)


def intervals(rng, n, emin=-1074, emax=1023, positive=False):
    a = random_doubles(rng, n, emin, emax, sign=not positive)
    b = random_doubles(rng, n, emin, emax, sign=not positive)
    # a third are points (directed rounding of single operations), a third narrow
    pts = rng.random(n) < 0.33
    b[pts] = a[pts]
    nar = (~pts) & (rng.random(n) < 0.5)
    b[nar] = a[nar] * (1.0 + rng.uniform(-1e-6, 1e-6, nar.sum()))
    X = np.stack([np.minimum(a, b), np.maximum(a, b)], 1)
    s = specials()
    if positive:
        s = s[s > 0]
    S = np.array([[p, q] for p in s for q in s if p <= q])
    return np.concatenate([X, S])


def gpu(opcode, X, Y=None):
    x = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    y = None if Y is None else torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    r = ivb.ivb_eval_op(opcode, x, y)
    return r.cpu().numpy()


@pytest.mark.parametrize("opcode", [W.OP_ADD, W.OP_SUB, W.OP_MUL, W.OP_DIV])
def test_binary_ops_bit_exact(opcode):
    rng = np.random.default_rng(opcode)
    n = 200000
    X = intervals(rng, n, -540, 500)
    Y = intervals(rng, n, -540, 500)
    m = min(len(X), len(Y))
    X, Y = X[:m], Y[:m]
    R = gpu(opcode, X, Y)
    Ro = oracle.iv_op(opcode, X, Y)
    bad = ~((R == Ro) | (np.isnan(R) & np.isnan(Ro))).all(axis=1)
    assert not bad.any(), (X[bad][:3], Y[bad][:3], R[bad][:3], Ro[bad][:3])


def test_division_exact_and_binade_cases():
    """quotients that are exact, powers of two, or next to them"""
    rng = np.random.default_rng(9)
    y = random_doubles(rng, 20000, -300, 300, sign=False)
    k = rng.integers(1, 64, y.size).astype(np.float64)
    xs = [k * y, np.ldexp(y, rng.integers(-20, 20, y.size)), np.nextafter(y, 0) * 2.0, np.nextafter(2 * y, 10 * y)]
    for x in xs:
        X = np.stack([x, x], 1)
        Y = np.stack([y, y], 1)
        for sgn in (1.0, -1.0):
            R = gpu(W.OP_DIV, sgn * X, Y)
            assert np.array_equal(R, oracle.iv_op(W.OP_DIV, sgn * X, Y))


def test_sqrt_and_reciprocal_exact_and_neighbouring_cases():
    """square roots of exact squares (zero remainder) and of their neighbours
    (remainder of one unit), reciprocals of products of powers of two and
    short odd integers and of their neighbours: the cases where the sign of
    the remainder decides the directed result"""
    rng = np.random.default_rng(21)
    g = random_doubles(rng, 30000, -400, 400, sign=False)
    g = (g.view(np.int64) & ~np.int64(0x7FFFFFF)).view(np.float64)      # 26-bit significands: g^2 exact
    sq = g * g
    x = np.concatenate([sq, np.nextafter(sq, 0.0), np.nextafter(sq, np.inf)])
    X = np.stack([x, x], 1)
    assert np.array_equal(gpu(W.OP_SQRT, X), oracle.iv_op(W.OP_SQRT, X))
    odd = rng.integers(1, 1 << 20, 30000) * 2 + 1
    y = np.ldexp(odd.astype(np.float64), rng.integers(-300, 300, odd.size))
    y = np.concatenate([y, np.nextafter(y, 0.0), np.nextafter(y, np.inf), np.ldexp(1.0, rng.integers(-900, 900, 100))])
    for sgn in (1.0, -1.0):
        Y = np.stack([sgn * y, sgn * y], 1)
        assert np.array_equal(gpu(RECIP, Y), oracle.iv_op(RECIP, Y))


@pytest.mark.parametrize("opcode", [W.OP_SQR, W.OP_SQRT, RECIP, W.OP_NEG])
def test_unary_ops_bit_exact(opcode):
    rng = np.random.default_rng(50 + opcode)
    X = intervals(rng, 200000, -1074, 1023, positive=(opcode == W.OP_SQRT))
    if opcode == RECIP:
        X = X[(X[:, 0] > 0) | (X[:, 1] < 0)]
    R = gpu(opcode, X)
    Ro = oracle.iv_op(opcode, X)
    bad = ~((R == Ro) | (np.isnan(R) & np.isnan(Ro))).all(axis=1)
    assert not bad.any(), (X[bad][:3], R[bad][:3], Ro[bad][:3])


def test_fused_accumulation_bit_exact():
    """acc + x*y with one directed rounding per end (IVB_EVAL_FMA, the adjoint,
    tangent and Mean Value Form accumulation) equals the oracle's: every sign
    case of x and y, zero endpoints, points, wide exponent ranges, infinite
    factor ends and special operands"""
    rng = np.random.default_rng(105)
    n = 200000
    X = intervals(rng, n, -300, 300)
    Y = intervals(rng, n, -300, 300)
    Z = intervals(rng, n, -300, 300)
    m = min(len(X), len(Y), len(Z))
    X, Y, Z = X[:m], Y[:m], Z[:m]
    X[::11, 0] = 0.0                                         # zero lower ends ...
    X[::11, 1] = np.abs(X[::11, 1])                          # ... of valid intervals
    Y[5::13, 1] = 0.0
    Y[5::13, 0] = np.minimum(Y[5::13, 0], 0.0)
    Z[3::17] = -Z[3::17, ::-1]                               # addends of both signs
    x = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    y = torch.from_numpy(np.ascontiguousarray(Y)).to(DEV)
    z = torch.from_numpy(np.ascontiguousarray(Z)).to(DEV)
    R = ivb.ivb_eval_op(ivb.IVB_EVAL_FMA, x, y, acc=z).cpu().numpy()
    Ro = oracle.iv_fma(X, Y, Z)
    bad = ~((R == Ro) | (np.isnan(R) & np.isnan(Ro))).all(axis=1)
    assert not bad.any(), (X[bad][:3], Y[bad][:3], Z[bad][:3], R[bad][:3], Ro[bad][:3])
    # infinite factor ends with finite addends
    F = np.array([[-np.inf, 1.0], [0.0, np.inf], [-2.0, np.inf], [-np.inf, np.inf], [1.0, 1.0], [0.0, 0.0]])
    A = np.array([[-1.0, 2.0], [0.5, 0.75], [-0.0, 0.0]])
    Xs = np.repeat(F, len(F) * len(A), axis=0)
    Ys = np.tile(np.repeat(F, len(A), axis=0), (len(F), 1))
    Zs = np.tile(A, (len(F) * len(F), 1))
    R = ivb.ivb_eval_op(ivb.IVB_EVAL_FMA, torch.from_numpy(Xs).to(DEV), torch.from_numpy(Ys).to(DEV),
                        acc=torch.from_numpy(Zs).to(DEV)).cpu().numpy()
    Ro = oracle.iv_fma(Xs, Ys, Zs)
    assert (((R == Ro) | (np.isnan(R) & np.isnan(Ro))).all(axis=1)).all()


def ulps(a, b):
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    ia = np.where(ia < 0, np.int64(-(2 ** 63)) - ia, ia)
    ib = np.where(ib < 0, np.int64(-(2 ** 63)) - ib, ib)
    return np.abs(ia - ib)


@pytest.mark.parametrize("fn", ["exp", "log"])
def test_exp_log_contain_oracle_within_4_ulps(fn):
    rng = np.random.default_rng(77)
    if fn == "exp":
        pts = np.concatenate([rng.uniform(-745, 710, 150000), rng.uniform(-1, 1, 50000),
                              np.ldexp(rng.uniform(-1, 1, 20000), -rng.integers(1, 60, 20000)),
                              np.array([0.0, -0.0, 700.0, -700.0, 709.7, -745.0, 1e-300])])
        opcode = W.OP_EXP
    else:
        pts = np.concatenate([random_doubles(rng, 150000, -1074, 1023, sign=False),
                              1.0 + rng.uniform(-0.01, 0.01, 50000), 1.0 + np.ldexp(rng.uniform(-1, 1, 20000), -30),
                              np.array([1.0, 2.0, 0.5, 1.5, 0.75, np.nextafter(1.0, 0), np.nextafter(1.0, 2)])])
        opcode = W.OP_LOG
    X = np.stack([pts, pts], 1)
    R = gpu(opcode, X)
    Ro = oracle.iv_op(opcode, X, tight=True)
    assert np.all(R[:, 0] <= Ro[:, 0]) and np.all(R[:, 1] >= Ro[:, 1])
    fin = np.isfinite(Ro[:, 0]) & (Ro[:, 0] != 0)
    assert np.all(ulps(R[fin, 0], Ro[fin, 0]) <= 4)
    fin = np.isfinite(Ro[:, 1]) & (Ro[:, 1] != 0)
    assert np.all(ulps(R[fin, 1], Ro[fin, 1]) <= 4)


# ---------------------------------------- integer-pipe emulation (option emulate)

def emulation_operands(rng, n):
    """pairs aimed at the emulated add and multiply: every exponent difference
    up to 70 with both signs (alignment, sticky bits, carries), near-cancelling
    sums, all-ones and power-of-two significands (rounding carries into the
    exponent), products and sums near overflow and underflow, subnormals,
    zeros, infinities"""
    def sig(k, kind):
        m = rng.uniform(1.0, 2.0, k)
        if kind == 1:
            m = np.full(k, np.nextafter(2.0, 1.0))
        elif kind == 2:
            m = np.ones(k)
        return m
    xs, ys = [], []
    # exponent differences 0..70, random signs and significand classes
    k = n // 4
    ex = rng.integers(-60, 60, k)
    d = rng.integers(0, 71, k)
    kx, ky = rng.integers(0, 3, k), rng.integers(0, 3, k)
    x = np.ldexp(np.where(kx == 0, sig(k, 0), np.where(kx == 1, sig(k, 1), 1.0)), ex)
    y = np.ldexp(np.where(ky == 0, sig(k, 0), np.where(ky == 1, sig(k, 1), 1.0)), ex - d)
    xs.append(x * rng.choice([-1.0, 1.0], k))
    ys.append(y * rng.choice([-1.0, 1.0], k))
    # near cancellation: y = -x (1 + tiny), and y = -x exactly
    x = np.ldexp(rng.uniform(1.0, 2.0, k), rng.integers(-100, 100, k))
    rel = np.where(rng.random(k) < 0.1, 0.0, rng.choice([-1.0, 1.0], k) * 2.0 ** rng.uniform(-53, -2, k))
    xs.append(x)
    ys.append(-x * (1.0 + rel))
    # near overflow / underflow of products and sums
    e1 = rng.integers(-1022, 1024, k)
    e2 = np.where(rng.random(k) < 0.5, 1023 - e1 + rng.integers(-2, 3, k), -1022 - e1 + rng.integers(-2, 3, k))
    xs.append(np.ldexp(rng.uniform(1.0, 2.0, k), e1) * rng.choice([-1.0, 1.0], k))
    ys.append(np.ldexp(rng.uniform(1.0, 2.0, k), np.clip(e2, -1074, 1023)) * rng.choice([-1.0, 1.0], k))
    # full range, subnormals included
    xs.append(random_doubles(rng, k, -1074, 1023))
    ys.append(random_doubles(rng, k, -1074, 1023))
    x, y = np.concatenate(xs), np.concatenate(ys)
    s = np.concatenate([specials(), [np.inf, -np.inf]])
    sx, sy = np.meshgrid(s, s)
    x, y = np.concatenate([x, sx.ravel()]), np.concatenate([y, sy.ravel()])
    return x, y


def same_bits_or_nan(a, b):
    return (a.view(np.int64) == b.view(np.int64)) | (np.isnan(a) & np.isnan(b))


@pytest.mark.parametrize("name,opcode,emu", [("add", W.OP_ADD, ivb.IVB_EVAL_EMU_ADD), ("sub", W.OP_SUB, ivb.IVB_EVAL_EMU_SUB),
                                             ("mul", W.OP_MUL, ivb.IVB_EVAL_EMU_MUL), ("sqr", W.OP_SQR, ivb.IVB_EVAL_EMU_SQR)])
def test_emulated_ops_bit_exact(name, opcode, emu):
    """+ - * sqr with every endpoint operation emulated on the integer pipes
    equal the oracle's directed operations bit for bit (signed zeros
    included), on points (single directed operations) and on intervals"""
    rng = np.random.default_rng(1000 + opcode)
    x, y = emulation_operands(rng, 1_600_000)
    # points: [x, x] op [y, y] gives the directed operation at both ends
    X, Y = np.stack([x, x], 1), np.stack([y, y], 1)
    XI = intervals(rng, 400000, -1074, 1023)
    YI = intervals(rng, 400000, -1074, 1023)
    m = min(len(XI), len(YI))
    X, Y = np.concatenate([X, XI[:m]]), np.concatenate([Y, YI[:m]])
    unary = opcode == W.OP_SQR
    R = gpu(emu, X, None if unary else Y)
    Ro = oracle.iv_op(opcode, X, None if unary else Y)
    bad = ~same_bits_or_nan(R, Ro).all(axis=1)
    assert not bad.any(), (name, int(bad.sum()), X[bad][:3], Y[bad][:3], R[bad][:3], Ro[bad][:3])
    # the hardware path gives the same bits
    Rh = gpu(opcode, X, None if unary else Y)
    assert same_bits_or_nan(R, Rh).all()
