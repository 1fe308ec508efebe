"""Thin ctypes binding of libivb.so, the C ABI in include/ivb.h.

Argument marshalling only: every step of the bounding runs in the library's
CUDA kernels. Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
the library detects the pointer kind. CUDA tensors are processed on torch's
current stream. Importing this module fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

IVB_OK, IVB_EINVAL, IVB_ENOMEM, IVB_ECUDA, IVB_ETAPE, IVB_ETIMEOUT, IVB_ENOTSUP = range(7)
STATUS_NAMES = {0: "IVB_OK", 1: "IVB_EINVAL", 2: "IVB_ENOMEM", 3: "IVB_ECUDA", 4: "IVB_ETAPE",
                5: "IVB_ETIMEOUT", 6: "IVB_ENOTSUP"}
IVB_GRAD_FORWARD, IVB_GRAD_ADJOINT = 0, 1
IVB_FORM_MVF, IVB_FORM_NIE, IVB_FORM_MVF_NIE = 0, 1, 2
IVB_SPLIT_UNIFORM, IVB_SPLIT_LARGEST, IVB_SPLIT_ADAPTIVE = 0, 1, 2
GRAD = {"forward": IVB_GRAD_FORWARD, "adjoint": IVB_GRAD_ADJOINT}
FORM = {"mvf": IVB_FORM_MVF, "nie": IVB_FORM_NIE, "mvf_nie": IVB_FORM_MVF_NIE}
SPLIT = {"uniform": IVB_SPLIT_UNIFORM, "largest": IVB_SPLIT_LARGEST, "adaptive": IVB_SPLIT_ADAPTIVE}


class IvbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ivb_options(ctypes.Structure):
    _fields_ = [("grad_mode", ctypes.c_int32), ("form", ctypes.c_int32), ("filter", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("max_nodes", ctypes.c_int32), ("frame_in_shared", ctypes.c_int32), ("specialize", ctypes.c_int32),
                ("emulate", ctypes.c_int32), ("recompute", ctypes.c_int32), ("seg_chunk", ctypes.c_int32),
                ("seg_regs", ctypes.c_int32), ("threads_per_subdomain", ctypes.c_int32), ("seg_sync", ctypes.c_int32),
                ("seg_ilp", ctypes.c_int32), ("seg_outline", ctypes.c_int32)]


class ivb_tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("frame_in_shared", ctypes.c_int32), ("threads_per_subdomain", ctypes.c_int32),
                ("subdomains_per_pass", ctypes.c_int32), ("chunk_sync", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("candidates", ctypes.c_int32),
                ("best_ms", ctypes.c_float), ("worst_ms", ctypes.c_float)]


class ivb_tape(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("n_ops", ctypes.c_int32), ("n_outputs", ctypes.c_int32),
                ("ops", ctypes.c_void_p), ("out_idx", ctypes.c_void_p), ("out_kind", ctypes.c_void_p)]


class ivb_bnb_options(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("split_mode", ctypes.c_int32), ("splits", ctypes.c_void_p),
                ("target", ctypes.c_int64), ("eps_abs", ctypes.c_double), ("eps_rel", ctypes.c_double),
                ("max_nodes", ctypes.c_int64), ("time_limit", ctypes.c_double), ("corner_ub", ctypes.c_int32),
                ("propagate", ctypes.c_int32), ("overlap", ctypes.c_int32)]


class ivb_bnb_result(ctypes.Structure):
    _fields_ = [("lb", ctypes.c_double), ("ub", ctypes.c_double), ("iterations", ctypes.c_int64),
                ("nodes_bounded", ctypes.c_int64), ("subdomains", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("converged", ctypes.c_int32), ("open_nodes", ctypes.c_int64), ("split_target", ctypes.c_int64)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded libivb.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise IvbError(IVB_ENOTSUP, f"{path} is not built; run paper_2507_20769_gb300.build.build() "
                                        "(needs the CUDA toolkit)")
        L = ctypes.CDLL(path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.ivb_options_default.argtypes = [P]
        L.ivb_create_problem.argtypes = [P, P, P]
        L.ivb_bound_nodes.argtypes = [P, I32, P, P, P, P, P]
        L.ivb_bound_nodes_ex.argtypes = [P, I32, P, P, P, P, P, P, P, P]
        L.ivb_enclose.argtypes = [P, P, P, I64, I64, P, P, P, P]
        L.ivb_point_grad.argtypes = [P, I64, P, P, P, P]
        L.ivb_pick_splits.argtypes = [I32, P, P, I64, I32, P]
        L.ivb_get_tuning.argtypes = [P, P, P, P, P]
        L.ivb_launch_count.argtypes = [P]
        L.ivb_launch_count.restype = I64
        L.ivb_last_error.argtypes = [P]
        L.ivb_last_error.restype = ctypes.c_char_p
        L.ivb_destroy.argtypes = [P]
        L.ivb_bound_nodes_noalloc.argtypes = [P, I32, P, P, P, P, P]
        L.ivb_eval_op.argtypes = [I32, I64, P, P, P, P]
        L.ivb_op_counts.argtypes = [P, P]
        L.ivb_fp64_probe.argtypes = [I32, I32, P]
        L.ivb_bnb_options_default.argtypes = [P]
        L.ivb_bnb_solve.argtypes = [P, I32, P, P, P, P]
        L.ivb_get_specialization.argtypes = [P, P, P, P, P, P]
        L.ivb_propagate.argtypes = [P, I32, P, D, I32, P, P]
        L.ivb_host_gradient.argtypes = [P, P, I32, I32, P]
        L.ivb_specialize_compile.argtypes = [P, I32, I32, P, P, P]
        L.ivb_get_segmentation.argtypes = [P, P, P, P, P, P, P, P]
        L.ivb_get_tuning_ex.argtypes = [P, P]
        for f in ("ivb_create_problem", "ivb_bound_nodes", "ivb_bound_nodes_ex", "ivb_enclose", "ivb_point_grad",
                  "ivb_pick_splits", "ivb_get_tuning", "ivb_bnb_solve", "ivb_op_counts", "ivb_fp64_probe",
                  "ivb_bound_nodes_noalloc", "ivb_eval_op", "ivb_get_specialization", "ivb_specialize_compile",
                  "ivb_get_segmentation", "ivb_get_tuning_ex",
                  "ivb_propagate", "ivb_host_gradient"):
            getattr(L, f).restype = I32
        _lib = L
    return _lib


# ----------------------------------------------------------------- marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _stream_for(*xs):
    for x in xs:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return None


def _check(status: int, handle=None):
    if status != IVB_OK:
        msg = lib().ivb_last_error(handle)
        raise IvbError(status, msg.decode() if msg else "")


def _as(x, dtype):
    """numpy array of dtype, or a torch tensor checked for dtype"""
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        return x.contiguous()
    return np.ascontiguousarray(x, dtype=dtype)


def _empty_like_kind(ref, shape, dtype):
    if ref is not None and _is_torch(ref):
        import torch
        tdt = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


# -------------------------------------------------------------------- the ABI

def ivb_options_default(**overrides) -> ivb_options:
    o = ivb_options()
    lib().ivb_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "grad_mode" and isinstance(v, str):
            v = GRAD[v]
        if k == "form" and isinstance(v, str):
            v = FORM[v]
        setattr(o, k, int(v))
    return o


def ivb_create_problem(tape, options: ivb_options | None = None, **overrides) -> "Problem":
    return Problem(tape, options, **overrides)


def ivb_pick_splits(box, target: int, strategy="adaptive", ref_widths=None) -> np.ndarray:
    box = np.ascontiguousarray(box, dtype=np.float64).reshape(-1, 2)
    n = box.shape[0]
    ref = None if ref_widths is None else np.ascontiguousarray(ref_widths, dtype=np.float64)
    out = np.empty(n, dtype=np.int32)
    s = SPLIT[strategy] if isinstance(strategy, str) else int(strategy)
    _check(lib().ivb_pick_splits(n, _ptr(box), _ptr(ref), int(target), s, _ptr(out)))
    return out


CNT_NAMES = ("addsub", "mul", "div", "rcp", "sqrt", "exp", "log", "rn")
PROBE = {"dadd": 0, "dmul": 1, "dfma": 2, "ddiv": 3, "drcp": 4, "dsqrt": 5, "exp": 6, "log": 7,
         "own_rcp": 8, "own_div": 9, "own_sqrt": 10, "own_exp": 11, "own_log": 12,
         "emu_mul": 13, "mixed_mul": 14, "emu_add": 15, "mixed_add": 16}


def ivb_fp64_probe(which: str, iters: int = 1024) -> float:
    """lane operations per second of one FP64 primitive on the current GPU"""
    v = ctypes.c_double()
    _check(lib().ivb_fp64_probe(PROBE[which], int(iters), ctypes.byref(v)))
    return v.value


IVB_EVAL_RECIP = 100
IVB_EVAL_EMU_ADD, IVB_EVAL_EMU_SUB, IVB_EVAL_EMU_MUL, IVB_EVAL_EMU_SQR = 101, 102, 103, 104
IVB_EVAL_FMA = 105


def ivb_eval_op(opcode: int, x, y=None, acc=None):
    """test hook: one interval operation of the kernels' arithmetic on CUDA
    tensors of intervals [n, 2]; returns a new [n, 2] tensor (IVB_EVAL_FMA:
    acc + x*y, acc required)"""
    import torch
    if not (_is_torch(x) and x.is_cuda):
        raise TypeError("ivb_eval_op takes CUDA tensors")
    x = x.contiguous()
    y = None if y is None else y.contiguous()
    if opcode == IVB_EVAL_FMA:
        if acc is None:
            raise ValueError("IVB_EVAL_FMA needs the addend acc")
        r = acc.contiguous().clone()
    else:
        r = torch.empty_like(x)
    _check(lib().ivb_eval_op(int(opcode), int(x.shape[0]), _ptr(x), _ptr(y), _ptr(r), _stream_for(x)))
    return r


def ivb_specialize_compile(tape, grad_mode="adjoint", compact=True, variant=None) -> dict:
    """generate and compile (NVRTC, no GPU needed) the tape-specialised
    kernel of a tape: ptxas registers, spill-store bytes, compile seconds.
    variant: the `specialize` value it is built as (1 compact, 2 inlined,
    3 segmented; 4: segmented with two subdomains per thread in the paired
    dual-pipe form, emulate = 15); by default 1 or 2 from `compact`"""
    recs = tape.records()
    oi = np.ascontiguousarray(tape.out_idx, dtype=np.int32)
    ok = np.ascontiguousarray(tape.out_kind, dtype=np.uint8)
    t = ivb_tape(int(tape.n_vars), int(recs.shape[0]), int(oi.shape[0]), recs.ctypes.data, oi.ctypes.data,
                 ok.ctypes.data)
    regs, spill, secs = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    g = GRAD[grad_mode] if isinstance(grad_mode, str) else int(grad_mode)
    code = {1: 1, 2: 0, 3: 3, 4: 4}[int(variant)] if variant is not None else int(bool(compact))
    _check(lib().ivb_specialize_compile(ctypes.byref(t), g, code, ctypes.byref(regs),
                                        ctypes.byref(spill), ctypes.byref(secs)))
    return {"registers": regs.value, "spill_bytes": spill.value, "seconds": secs.value}


def _c_tape(tape):
    recs = tape.records()
    oi = np.ascontiguousarray(tape.out_idx, dtype=np.int32)
    ok = np.ascontiguousarray(tape.out_kind, dtype=np.uint8)
    t = ivb_tape(int(tape.n_vars), int(recs.shape[0]), int(oi.shape[0]), recs.ctypes.data, oi.ctypes.data,
                 ok.ctypes.data)
    return t, (recs, oi, ok)


def ivb_propagate(tape, boxes, ub=float("inf"), passes=4):
    """constraint propagation on the host (no GPU): tightened boxes
    [k, n, 2] and infeasible flags [k]"""
    bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, int(tape.n_vars), 2)
    out = np.empty_like(bx)
    inf = np.empty(bx.shape[0], dtype=np.uint8)
    t, keep = _c_tape(tape)
    _check(lib().ivb_propagate(ctypes.byref(t), bx.shape[0], _ptr(bx), float(ub), int(passes), _ptr(out),
                               _ptr(inf)))
    return out, inf.astype(bool)


def ivb_host_gradient(tape, box, output=0, grad_mode="adjoint"):
    """gradient enclosure [n, 2] of one output over one box, on the host (no GPU)"""
    bx = np.ascontiguousarray(box, dtype=np.float64).reshape(int(tape.n_vars), 2)
    G = np.empty_like(bx)
    t, keep = _c_tape(tape)
    _check(lib().ivb_host_gradient(ctypes.byref(t), _ptr(bx), int(output), GRAD[grad_mode], _ptr(G)))
    return G


def ivb_last_error(problem=None) -> str:
    h = None if problem is None else problem._h
    m = lib().ivb_last_error(h)
    return m.decode() if m else ""


class Problem:
    """An ivb_problem handle (ivb_create_problem / ivb_destroy)."""

    def __init__(self, tape, options: ivb_options | None = None, **overrides):
        L = lib()
        if options is None:
            options = ivb_options_default(**overrides)
        else:
            for k, v in overrides.items():
                setattr(options, k, int(v))
        self.options = options
        self.n_vars, self.n_out = int(tape.n_vars), int(tape.out_idx.shape[0])
        self._recs = tape.records()
        self._oi = np.ascontiguousarray(tape.out_idx, dtype=np.int32)
        self._ok = np.ascontiguousarray(tape.out_kind, dtype=np.uint8)
        t = ivb_tape(self.n_vars, int(self._recs.shape[0]), self.n_out, self._recs.ctypes.data,
                     self._oi.ctypes.data, self._ok.ctypes.data)
        h = ctypes.c_void_p()
        st = L.ivb_create_problem(ctypes.byref(t), ctypes.byref(options), ctypes.byref(h))
        if st != IVB_OK:
            raise IvbError(st, L.ivb_last_error(None).decode())
        self._h = h

    # -- lifecycle
    def destroy(self):
        if getattr(self, "_h", None):
            lib().ivb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()

    # -- bounding
    def ivb_bound_nodes_ex(self, boxes, splits, want_ub=True, want_hull=False, out=None, stream=None):
        boxes = _as(boxes, np.float64)
        splits = _as(splits, np.int32)
        nn = int(boxes.shape[0]) if boxes.ndim == 3 else int(np.prod(boxes.shape)) // (2 * self.n_vars)
        out = out or {}
        lb = out.get("lb", _empty_like_kind(boxes, (nn,), np.float64))
        inf = out.get("infeasible", _empty_like_kind(boxes, (nn,), np.uint8))
        ub = out.get("ub", _empty_like_kind(boxes, (nn,), np.float64)) if want_ub else None
        mn = _empty_like_kind(boxes, (nn, self.n_out), np.float64) if want_hull else None
        mx = _empty_like_kind(boxes, (nn, self.n_out), np.float64) if want_hull else None
        s = stream if stream is not None else _stream_for(boxes, splits, lb)
        _check(lib().ivb_bound_nodes_ex(self._h, nn, _ptr(boxes), _ptr(splits), _ptr(lb), _ptr(inf), _ptr(ub),
                                        _ptr(mn), _ptr(mx), s), self._h)
        r = {"lb": lb, "infeasible": inf}
        if want_ub:
            r["ub"] = ub
        if want_hull:
            r["minlo"], r["maxhi"] = mn, mx
        return r

    def ivb_bound_nodes(self, boxes, splits, stream=None):
        r = self.ivb_bound_nodes_ex(boxes, splits, want_ub=False, stream=stream)
        return r["lb"], r["infeasible"]

    def ivb_bound_nodes_noalloc(self, boxes, splits, out_lb, out_infeasible, stream=None):
        """allocation-free bounding for callers that cannot allocate device
        memory: all four arguments are CUDA tensors (outputs preallocated)"""
        import torch
        for x in (boxes, splits, out_lb, out_infeasible):
            if not (_is_torch(x) and x.is_cuda):
                raise TypeError("ivb_bound_nodes_noalloc takes CUDA tensors only")
        want = ((boxes, torch.float64, "boxes"), (splits, torch.int32, "splits"),
                (out_lb, torch.float64, "out_lb"), (out_infeasible, torch.uint8, "out_infeasible"))
        for x, dt, name in want:
            if x.dtype != dt:
                raise TypeError(f"{name} must be {dt}, got {x.dtype}")
            if not x.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            if x.device != boxes.device:
                raise ValueError(f"{name} is on {x.device}, boxes on {boxes.device}")
        if boxes.ndim != 3 or boxes.shape[1:] != (self.n_vars, 2):
            raise ValueError(f"boxes must have shape (nodes, {self.n_vars}, 2), got {tuple(boxes.shape)}")
        nn = int(boxes.shape[0])
        if tuple(splits.shape) != (nn, self.n_vars):
            raise ValueError(f"splits must have shape ({nn}, {self.n_vars}), got {tuple(splits.shape)}")
        for x, name in ((out_lb, "out_lb"), (out_infeasible, "out_infeasible")):
            if tuple(x.shape) != (nn,):
                raise ValueError(f"{name} must have shape ({nn},), got {tuple(x.shape)}")
        s = stream if stream is not None else _stream_for(boxes)
        _check(lib().ivb_bound_nodes_noalloc(self._h, nn, _ptr(boxes), _ptr(splits), _ptr(out_lb),
                                             _ptr(out_infeasible), s), self._h)
        return out_lb, out_infeasible

    def ivb_enclose(self, box, splits, first=0, count=None, want_fc=False, want_g=False, device=None):
        box = _as(box, np.float64)
        splits = _as(splits, np.int32)
        if count is None:
            sp = splits.cpu().numpy() if _is_torch(splits) else splits
            count = int(np.prod(sp.astype(np.int64))) - int(first)
        ref = box if _is_torch(box) else None
        F = _empty_like_kind(ref, (count, self.n_out, 2), np.float64)
        Fc = _empty_like_kind(ref, (count, self.n_out, 2), np.float64) if want_fc else None
        G = _empty_like_kind(ref, (count, self.n_out, self.n_vars, 2), np.float64) if want_g else None
        _check(lib().ivb_enclose(self._h, _ptr(box), _ptr(splits), int(first), int(count), _ptr(F), _ptr(Fc),
                                 _ptr(G), _stream_for(box, F)), self._h)
        return F, Fc, G

    def ivb_point_grad(self, x, want_grad=True, stream=None):
        x = _as(x, np.float64)
        m = int(x.shape[0])
        f = _empty_like_kind(x, (m, self.n_out), np.float64)
        g = _empty_like_kind(x, (m, self.n_out, self.n_vars), np.float64) if want_grad else None
        s = stream if stream is not None else _stream_for(x)
        _check(lib().ivb_point_grad(self._h, m, _ptr(x), _ptr(f), _ptr(g), s), self._h)
        return f, g

    def ivb_bnb_solve(self, root, splits=None, target=0, strategy="adaptive", batch=1, eps_abs=0.0,
                      eps_rel=1e-3, max_nodes=0, time_limit=0.0, corner_ub=1, propagate=0, overlap=0, stream=None):
        root = np.ascontiguousarray(root, dtype=np.float64)
        o = ivb_bnb_options()
        lib().ivb_bnb_options_default(ctypes.byref(o))
        sp = None
        if splits is not None:
            sp = np.ascontiguousarray(splits, dtype=np.int32)
            o.split_mode, o.splits = 0, sp.ctypes.data
        else:
            o.split_mode = 1 + (SPLIT[strategy] if isinstance(strategy, str) else int(strategy))
            o.target = int(target)
        o.batch, o.eps_abs, o.eps_rel = int(batch), float(eps_abs), float(eps_rel)
        o.max_nodes, o.time_limit, o.corner_ub = int(max_nodes), float(time_limit), int(corner_ub)
        o.propagate, o.overlap = int(propagate), int(overlap)
        r = ivb_bnb_result()
        _check(lib().ivb_bnb_solve(self._h, self.n_vars, _ptr(root), ctypes.byref(o), ctypes.byref(r), stream),
               self._h)
        return {"lb": r.lb, "ub": r.ub, "iterations": r.iterations, "nodes": r.nodes_bounded,
                "subdomains": r.subdomains, "seconds": r.seconds, "converged": bool(r.converged),
                "open": r.open_nodes, "split_target": r.split_target}

    def ivb_get_tuning(self):
        t = ivb_tuning()
        _check(lib().ivb_get_tuning_ex(self._h, ctypes.byref(t)), self._h)
        return {k: getattr(t, k) for k, _ in ivb_tuning._fields_}

    def ivb_get_specialization(self) -> dict:
        a, r, lb, sec, em = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        _check(lib().ivb_get_specialization(self._h, ctypes.byref(a), ctypes.byref(r), ctypes.byref(lb),
                                            ctypes.byref(sec), ctypes.byref(em)), self._h)
        return {"active": bool(a.value), "registers": r.value, "local_bytes": lb.value, "compile_seconds": sec.value,
                "emulate": em.value}

    def ivb_get_segmentation(self) -> dict:
        su, ch, rc, il = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ld, stv, re = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ivb_get_segmentation(self._h, ctypes.byref(su), ctypes.byref(ch), ctypes.byref(ld),
                                          ctypes.byref(stv), ctypes.byref(re), ctypes.byref(rc), ctypes.byref(il)),
               self._h)
        return {"state_units": su.value, "chunks": ch.value, "state_loads": ld.value, "state_stores": stv.value,
                "recomputed": re.value, "recompute": rc.value, "ilp": il.value}

    def ivb_op_counts(self) -> dict:
        c = (ctypes.c_int64 * 8)()
        _check(lib().ivb_op_counts(self._h, c), self._h)
        return dict(zip(CNT_NAMES, [int(v) for v in c]))

    def ivb_launch_count(self) -> int:
        return int(lib().ivb_launch_count(self._h))

    def ivb_last_error(self) -> str:
        return ivb_last_error(self)

    # short aliases
    bound_nodes = ivb_bound_nodes
    bound_nodes_ex = ivb_bound_nodes_ex
    enclose = ivb_enclose
    point_grad = ivb_point_grad
    bnb_solve = ivb_bnb_solve
    get_tuning = ivb_get_tuning
    get_specialization = ivb_get_specialization
    get_segmentation = ivb_get_segmentation
    launch_count = ivb_launch_count
    op_counts = ivb_op_counts
    bound_nodes_noalloc = ivb_bound_nodes_noalloc
