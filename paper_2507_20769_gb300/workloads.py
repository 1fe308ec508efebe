"""Seeded synthetic inputs: op tapes of factorable functions and B&B node batches.

This module only *builds problems*: it holds none of the bounding method's
arithmetic (no interval operations, no derivatives, no partitioning). Both the
CUDA path and the CPU oracle consume what it returns.

The paper's test problems (ANN surrogates of Peaks and Alpine02, Sections 4.1
and 4.3) need trained weights that were not released, so the workloads are
seeded random factorable functions (Definition 4) of the sizes stated below,
written as op tapes (Section 3.2, Fig. 5: the objective and constraints as
sub-graphs of one DAG). Structure: a node's operands come from a window of
recent nodes of the same function or from the input variables, which gives the
layer-to-layer locality of the paper's feed-forward ANN surrogates.

Randomness: xoshiro256** (Blackman and Vigna, 2018) seeded through SplitMix64,
implemented here from its published definition so that a seed gives the same
tape on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# tape alphabet (mirrors the opcodes declared in include/ivb.h)
OP_VAR, OP_CONST, OP_ADD, OP_SUB, OP_MUL, OP_DIV = 0, 1, 2, 3, 4, 5
OP_SQR, OP_SQRT, OP_EXP, OP_LOG, OP_NEG = 6, 7, 8, 9, 10
OP_NAMES = {OP_VAR: "var", OP_CONST: "const", OP_ADD: "add", OP_SUB: "sub", OP_MUL: "mul",
            OP_DIV: "div", OP_SQR: "sqr", OP_SQRT: "sqrt", OP_EXP: "exp", OP_LOG: "log",
            OP_NEG: "neg"}
BINARY = (OP_ADD, OP_SUB, OP_MUL, OP_DIV)
KIND_OBJ, KIND_INEQ, KIND_EQ = 0, 1, 2

OPS_RATIONAL = (OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_SQR, OP_SQRT)
OPS_TINY = (OP_ADD, OP_SUB, OP_MUL, OP_SQR, OP_EXP)
OPS_ALL = (OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_SQR, OP_SQRT, OP_EXP, OP_LOG)

_M64 = (1 << 64) - 1

# layout of one tape entry in the C ABI (ivb_op): u8 op, 3 pad, i32 a, i32 b, f64 c
IVB_OP_DTYPE = np.dtype({"names": ["op", "a", "b", "c"],
                         "formats": ["u1", "<i4", "<i4", "<f8"],
                         "offsets": [0, 4, 8, 16], "itemsize": 24})


class Xoshiro256ss:
    """xoshiro256** 1.0 with SplitMix64 seeding (Blackman & Vigna, 2018)."""

    def __init__(self, seed: int):
        z = seed & _M64
        self.s = []
        for _ in range(4):
            z = (z + 0x9E3779B97F4A7C15) & _M64
            x = z
            x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _M64
            x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _M64
            self.s.append(x ^ (x >> 31))

    @staticmethod
    def _rotl(x: int, k: int) -> int:
        return ((x << k) | (x >> (64 - k))) & _M64

    def next_u64(self) -> int:
        s = self.s
        result = (self._rotl((s[1] * 5) & _M64, 7) * 9) & _M64
        t = (s[1] << 17) & _M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = self._rotl(s[3], 45)
        return result

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * 2.0 ** -53)

    def randint(self, n: int) -> int:
        """uniform integer in [0, n) (multiply-shift; bias below 2^-40 for n < 2^24)"""
        return (self.next_u64() * n) >> 64

    def choice(self, seq):
        return seq[self.randint(len(seq))]


@dataclass
class Tape:
    """Flattened DAG: entry t is (op[t], a[t], b[t], c[t]); operands index
    earlier entries (VAR: a = variable index; CONST: value c)."""
    n_vars: int
    op: np.ndarray
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    out_idx: np.ndarray
    out_kind: np.ndarray
    root_box: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_ops(self) -> int:
        return int(self.op.shape[0])

    @property
    def n_out(self) -> int:
        return int(self.out_idx.shape[0])

    def records(self) -> np.ndarray:
        r = np.zeros(self.n_ops, dtype=IVB_OP_DTYPE)
        r["op"], r["a"], r["b"], r["c"] = self.op, self.a, self.b, self.c
        return r

    def op_histogram(self) -> dict:
        u, k = np.unique(self.op, return_counts=True)
        return {OP_NAMES[int(x)]: int(y) for x, y in zip(u, k)}


class TapeBuilder:
    """Appends entries and keeps a crude upper bound M[t] on |node t| over the
    root box (plain float arithmetic on magnitudes, used only to place scaling
    constants so that intermediate values stay moderate)."""

    def __init__(self, n_vars: int, root_box):
        self.n_vars = n_vars
        self.op, self.a, self.b, self.c, self.M = [], [], [], [], []
        for i in range(n_vars):
            self._push(OP_VAR, i, 0, 0.0, max(abs(root_box[i][0]), abs(root_box[i][1])))

    def _push(self, op, a, b, c, m):
        self.op.append(op); self.a.append(a); self.b.append(b); self.c.append(c)
        self.M.append(m)
        return len(self.op) - 1

    def const(self, v: float) -> int:
        return self._push(OP_CONST, 0, 0, float(v), abs(v))

    def unary(self, op, x, m) -> int:
        return self._push(op, x, 0, 0.0, m)

    def binary(self, op, x, y, m) -> int:
        return self._push(op, x, y, 0.0, m)


LIMIT = 1.0e3      # post-scale any node whose magnitude bound exceeds this
EXP_ARG = 4.0      # exp arguments are pre-scaled to |arg| <= EXP_ARG


def _pow2_at_most(r: float) -> float:
    """largest power of two <= r (r > 0)"""
    return 2.0 ** math.floor(math.log2(r))


class _DagGen:
    """One random function of K tape entries (its share of the n shared VAR
    entries included) appended to a builder."""

    def __init__(self, bld: TapeBuilder, rng: Xoshiro256ss, ops, window=12, p_recent=0.5,
                 p_const=0.15, p_var=0.25):
        self.bld, self.rng, self.ops = bld, rng, ops
        self.window, self.p_recent, self.p_const, self.p_var = window, p_recent, p_const, p_var
        self.pool = []          # recent interior nodes of this function
        self.unconsumed = []    # interior nodes not yet used as an operand (ordered)
        self.acc = None         # running sum of nodes that left the window unused
        self.emitted = 0

    # -- bookkeeping ----------------------------------------------------
    def _consume(self, x):
        if x in self.unconsumed:
            self.unconsumed.remove(x)

    def _u(self):
        return len(self.unconsumed)

    def _emit_node(self, t):
        self.unconsumed.append(t)
        self.pool.append(t)
        if len(self.pool) > self.window:
            old = self.pool.pop(0)
            if old in self.unconsumed:           # fold it into the accumulator now
                if self.acc is None:
                    self.acc = old
                else:
                    self._consume(old); self._consume(self.acc)
                    m = self.bld.M[old] + self.bld.M[self.acc]
                    self.acc = self.bld.binary(OP_ADD, self.acc, old, m)
                    self.emitted += 1
                    self.unconsumed.append(self.acc)

    # -- operand choice ---------------------------------------------------
    def _operand(self, allow_const=True):
        r = self.rng
        if self.pool and r.uniform() < self.p_recent:
            return self.pool[-1]
        if allow_const and r.uniform() < self.p_const:
            return ("const", r.uniform(-2.0, 2.0))
        if not self.pool or r.uniform() < self.p_var:
            return r.randint(self.bld.n_vars)
        return r.choice(self.pool)

    # -- candidate ops: returns a plan of (kind, ...) steps and its cost -----
    def _plan(self, op):
        a = self._operand(allow_const=False)
        b = self._operand() if op in BINARY else None
        return op, a, b

    def _cost(self, plan):
        op, a, b = plan
        e = 1
        new_consts = 0
        if isinstance(b, tuple):
            new_consts += 1
        if op in (OP_SQRT, OP_LOG):
            e += 3        # sqr, const, add guard
        if op == OP_DIV:
            e += 3
        if op == OP_EXP and self.bld.M[a] > EXP_ARG:
            e += 2        # const, mul pre-scale
        e += new_consts
        cons = {a} if b is None or isinstance(b, tuple) else {a, b}
        du = 1 - sum(1 for x in cons if x in self.unconsumed)
        return e + du, e

    def _materialize(self, x):
        if isinstance(x, tuple):
            return self.bld.const(x[1])
        return x

    def _guard_positive(self, t):
        """sqr(t) + kappa, kappa ~ U[0.5, 2]: a strictly positive argument"""
        bld = self.bld
        kap = self.rng.uniform(0.5, 2.0)
        s = bld.unary(OP_SQR, t, bld.M[t] ** 2)
        k = bld.const(kap)
        g = bld.binary(OP_ADD, s, k, bld.M[s] + kap)
        self.emitted += 3
        return g, kap

    def _emit(self, plan):
        op, a, b = plan
        bld = self.bld
        self._consume(a)
        bm = None
        if b is not None:
            if isinstance(b, tuple):
                b = self._materialize(b)
                self.emitted += 1
            else:
                self._consume(b)
            bm = bld.M[b]
        am = bld.M[a]
        if op == OP_ADD or op == OP_SUB:
            t = bld.binary(op, a, b, am + bm)
        elif op == OP_MUL:
            t = bld.binary(op, a, b, am * bm)
        elif op == OP_DIV:
            g, kap = self._guard_positive(b)
            t = bld.binary(OP_DIV, a, g, am / kap)
        elif op == OP_SQR:
            t = bld.unary(OP_SQR, a, am * am)
        elif op == OP_SQRT:
            g, kap = self._guard_positive(a)
            t = bld.unary(OP_SQRT, g, math.sqrt(bld.M[g]))
        elif op == OP_LOG:
            g, kap = self._guard_positive(a)
            t = bld.unary(OP_LOG, g, max(abs(math.log(kap)), abs(math.log(bld.M[g]))))
        elif op == OP_EXP:
            if am > EXP_ARG:
                s = _pow2_at_most(EXP_ARG / am)
                k = bld.const(s)
                a = bld.binary(OP_MUL, a, k, am * s)
                self.emitted += 2
                am = bld.M[a]
            t = bld.unary(OP_EXP, a, math.exp(am))
        elif op == OP_NEG:
            t = bld.unary(OP_NEG, a, am)
        else:
            raise ValueError(op)
        self.emitted += 1
        self._emit_node(t)
        return t

    def _post_scale(self, t, budget_left):
        """multiply by a power of two when the magnitude bound is large"""
        bld = self.bld
        if bld.M[t] <= LIMIT or budget_left < 2:
            return 0
        s = _pow2_at_most(LIMIT / bld.M[t])
        self._consume(t)
        self.pool.remove(t)
        k = bld.const(s)
        u = bld.binary(OP_MUL, t, k, bld.M[t] * s)
        self.emitted += 2
        self.unconsumed.append(u)
        self.pool.append(u)
        return 2

    def build(self, K_own: int) -> int:
        """append exactly K_own entries; returns the function's root entry"""
        rng = self.rng
        while True:
            u = self._u()
            remaining = K_own - self.emitted - max(u - 1, 0)
            if remaining <= 0:
                break
            plan = self._plan(self.ops[rng.randint(len(self.ops))])
            cost, _ = self._cost(plan)
            if cost > remaining:
                # cheapest fallback: binary op of an unconsumed node with a variable
                cand = [x for x in self.unconsumed if x != self.acc]
                x = cand[-1] if cand else rng.randint(self.bld.n_vars)
                plan = (rng.choice((OP_ADD, OP_SUB, OP_MUL)), x, rng.randint(self.bld.n_vars))
                cost, _ = self._cost(plan)
                if cost > remaining:
                    break
            t = self._emit(plan)
            u = self._u()
            self._post_scale(t, K_own - self.emitted - max(u - 1, 0))
        # fold every node still unused, oldest first, into one sum
        rest = list(self.unconsumed)
        root = rest[0]
        for x in rest[1:]:
            root = self.bld.binary(OP_ADD, root, x, self.bld.M[root] + self.bld.M[x])
            self.emitted += 1
        self.unconsumed = [root]
        return root


def _point_value(bld: TapeBuilder, root: int, x) -> float:
    """round-to-nearest value of entry `root` at the point x (problem
    construction only: places the constraint offsets)"""
    v = {}
    for t in range(root + 1):
        op, a, b = bld.op[t], bld.a[t], bld.b[t]
        if op == OP_VAR: v[t] = x[a]
        elif op == OP_CONST: v[t] = bld.c[t]
        elif op == OP_ADD: v[t] = v[a] + v[b]
        elif op == OP_SUB: v[t] = v[a] - v[b]
        elif op == OP_MUL: v[t] = v[a] * v[b]
        elif op == OP_DIV: v[t] = v[a] / v[b]
        elif op == OP_SQR: v[t] = v[a] * v[a]
        elif op == OP_SQRT: v[t] = math.sqrt(v[a])
        elif op == OP_EXP: v[t] = math.exp(v[a])
        elif op == OP_LOG: v[t] = math.log(v[a])
        elif op == OP_NEG: v[t] = -v[a]
    return v[root]


def random_problem(n_vars: int, K: int, n_ineq: int, ops, root_box, base_seed: int,
                   name: str = "", window: int = 12) -> Tape:
    """Objective plus n_ineq inequality constraints g_o(x) <= 0, each a random
    function of K tape entries (K counts the n shared VAR entries too).
    Function o uses seed base_seed + o. Constraint o is r_o(x) - C_o with
    C_o = floor(r_o(x0) * 2^20) / 2^20 + 0.5 at a seeded x0 in the box, so x0 is
    strictly feasible and the problem is feasible."""
    if K < n_vars + 3:
        raise ValueError("K too small for the variable count")
    root_box = np.asarray(root_box, dtype=np.float64).reshape(n_vars, 2)
    bld = TapeBuilder(n_vars, root_box)
    out_idx, out_kind = [], []
    rng0 = Xoshiro256ss(base_seed + 999)
    x0 = [rng0.uniform(root_box[i][0], root_box[i][1]) for i in range(n_vars)]
    for o in range(1 + n_ineq):
        rng = Xoshiro256ss(base_seed + o)
        gen = _DagGen(bld, rng, ops, window=window)
        if o == 0:
            root = gen.build(K - n_vars)
            out_kind.append(KIND_OBJ)
        else:
            r = gen.build(K - n_vars - 2)
            val = _point_value(bld, r, x0)
            off = math.floor(val * 2.0 ** 20) / 2.0 ** 20 + 0.5
            k = bld.const(off)
            root = bld.binary(OP_SUB, r, k, bld.M[r] + abs(off))
            out_kind.append(KIND_INEQ)
        out_idx.append(root)
    tape = Tape(n_vars=n_vars,
                op=np.asarray(bld.op, dtype=np.uint8), a=np.asarray(bld.a, dtype=np.int32),
                b=np.asarray(bld.b, dtype=np.int32), c=np.asarray(bld.c, dtype=np.float64),
                out_idx=np.asarray(out_idx, dtype=np.int32), out_kind=np.asarray(out_kind, dtype=np.uint8),
                root_box=root_box, name=name, meta={"K": K, "x0": x0, "seed": base_seed})
    return tape


# ------------------------------------------------------------------ configs

def config_seed(config: int) -> int:
    return 20769 * 1000 + config * 10


@dataclass
class Workload:
    name: str
    tape: Tape
    splits: np.ndarray | None     # fixed splits per dim for every node (or None)
    grad_mode: str                # "forward" (plain) or "adjoint"
    gap_abs: float
    gap_rel: float


def config_tape(config: int) -> Tape:
    s = config_seed(config)
    if config == 1:
        return random_problem(2, 20, 0, OPS_TINY, [[-2, 2]] * 2, s, "tiny n=2 K=20")
    if config == 2:
        return random_problem(4, 60, 3, OPS_ALL, [[-5, 5]] * 4, s, "plain n=4 1+3x60")
    if config == 3:
        return random_problem(6, 150, 5, OPS_ALL, [[-10, 10]] * 6, s, "batching n=6 1+5x150")
    if config == 4:
        return random_problem(16, 400, 0, OPS_ALL, [[-2, 2]] * 16, s, "differentiation n=16 K=400")
    if config == 5:
        return random_problem(8, 1000, 10, OPS_ALL, [[-10, 10]] * 8, s, "full n=8 1+10x1000")
    raise ValueError(config)


def config_workload(config: int) -> Workload:
    t = config_tape(config)
    if config == 1:
        return Workload(t.name, t, np.array([16, 16], np.int32), "forward", 1e-4, 0.0)
    if config == 2:
        return Workload(t.name, t, np.array([16] * 4, np.int32), "forward", 0.0, 1e-3)
    if config == 3:
        return Workload(t.name, t, None, "adjoint", 0.0, 1e-3)
    if config == 4:
        return Workload(t.name, t, np.array([4] * 4 + [2] * 12, np.int32), "adjoint", 0.0, 1e-3)
    if config == 5:
        return Workload(t.name, t, None, "adjoint", 0.0, 1e-3)
    raise ValueError(config)


def uneven_nodes(n_vars: int, n_nodes: int, root_box, seed: int, log10_w=(-4.0, 1.0),
                 log2_s=(10, 20)):
    """Batch of B&B nodes of uneven widths: per dim width 10^U[log10_w], centre
    uniform in the root box, clipped to it; per node a subdomain target
    2^U{log2_s}. Returns boxes [n_nodes][n][2] and targets [n_nodes]."""
    rng = Xoshiro256ss(seed)
    root_box = np.asarray(root_box, dtype=np.float64).reshape(n_vars, 2)
    boxes = np.empty((n_nodes, n_vars, 2))
    targets = np.empty(n_nodes, dtype=np.int64)
    for k in range(n_nodes):
        for i in range(n_vars):
            lo, hi = root_box[i]
            w = 10.0 ** rng.uniform(*log10_w)
            ctr = rng.uniform(lo, hi)
            a, b = max(lo, ctr - 0.5 * w), min(hi, ctr + 0.5 * w)
            if not b > a:
                a, b = lo, hi
            boxes[k, i] = (a, b)
        targets[k] = 1 << (log2_s[0] + rng.randint(log2_s[1] - log2_s[0] + 1))
    return boxes, targets


def bisection_frontier(root_box, n_nodes: int, seed: int):
    """n_nodes boxes that tile the root box, made by repeatedly bisecting a
    random open box along its widest dimension (the shape of a B&B frontier)."""
    rng = Xoshiro256ss(seed)
    boxes = [np.asarray(root_box, dtype=np.float64).copy()]
    while len(boxes) < n_nodes:
        k = rng.randint(len(boxes))
        bx = boxes.pop(k)
        w = bx[:, 1] - bx[:, 0]
        i = int(np.argmax(w))
        mid = bx[i, 0] + 0.5 * (bx[i, 1] - bx[i, 0])
        l, r = bx.copy(), bx.copy()
        l[i, 1] = mid
        r[i, 0] = mid
        boxes += [l, r]
    return np.stack(boxes)


def full_scale_splits(box, root_box, wide: int = 8, rest: int = 4, n_wide: int = 2) -> np.ndarray:
    """Per-dimension split counts of one node of the full-scale workload
    (n = 8, 2^18 subdomains per node, 64 nodes = 2^24 per B&B iteration):
    `wide` on the `n_wide` dimensions of largest width relative to the root
    box (ties: lowest index), `rest` elsewhere -- 8^2 * 4^6 = 2^18."""
    box = np.asarray(box, dtype=np.float64)
    root_box = np.asarray(root_box, dtype=np.float64)
    rel = (box[:, 1] - box[:, 0]) / (root_box[:, 1] - root_box[:, 0])
    order = sorted(range(box.shape[0]), key=lambda i: (-rel[i], i))
    out = np.full(box.shape[0], rest, np.int32)
    out[order[:n_wide]] = wide
    return out


def sample_points(box, count: int, seed: int) -> np.ndarray:
    """count points uniform in a box [n][2]"""
    rng = Xoshiro256ss(seed)
    box = np.asarray(box, dtype=np.float64)
    n = box.shape[0]
    pts = np.empty((count, n))
    for k in range(count):
        for i in range(n):
            pts[k, i] = rng.uniform(box[i, 0], box[i, 1])
    return pts
