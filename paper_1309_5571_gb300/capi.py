"""ctypes binding of the C ABI declared in include/dmrg.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module only converts superblock
containers, torch device tensors and CUDA streams into the plain pointers and sizes of
the C ABI.  PyTorch provides device memory and streams.  If the shared library is
missing or CUDA is unavailable, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdmrg_gb300.so")

PREC = {"fp64": 0, "tf32": 1, "bf16x3": 2, "fp64tc": 3, "bf16x2": 4}
VEC = {"fp64": 0, "df": 1, "split": 2}
TILE_SCHEDULES = 27  # DMRG_TILE_SCHEDULES: candidate tile schedules per GEMM stage
IDENTITY = -1
MAX_SUBSPACE = 24

STATUS = {0: "ok", 1: "invalid argument", 2: "shape mismatch", 3: "out of memory",
          4: "CUDA error", 5: "not converged", 6: "numerical breakdown", 7: "unsupported"}


class DmrgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class NotConverged(DmrgError):
    pass


# ---------------------------------------------------------------- C structs
class Block(C.Structure):
    _fields_ = [("idx_in", C.c_int32), ("idx_out", C.c_int32), ("rows", C.c_int64),
                ("cols", C.c_int64), ("ld", C.c_int64), ("data", C.c_void_p)]


class Operator(C.Structure):
    _fields_ = [("nblocks", C.c_int32), ("blocks", C.POINTER(Block))]


class Term(C.Structure):
    _fields_ = [("coef", C.c_double), ("a_op", C.c_int32), ("b_op", C.c_int32)]


class SuperblockDesc(C.Structure):
    _fields_ = [("nL", C.c_int32), ("nR", C.c_int32),
                ("dimL", C.POINTER(C.c_int64)), ("dimR", C.POINTER(C.c_int64)),
                ("npairs", C.c_int32),
                ("pair_i", C.POINTER(C.c_int32)), ("pair_k", C.POINTER(C.c_int32)),
                ("nopsL", C.c_int32), ("nopsR", C.c_int32),
                ("opsL", C.POINTER(Operator)), ("opsR", C.POINTER(Operator)),
                ("nterms", C.c_int32), ("terms", C.POINTER(Term)),
                ("data_location", C.c_int32)]


class Term4(C.Structure):
    _fields_ = [("coef", C.c_double), ("l_op", C.c_int32), ("s1_op", C.c_int32),
                ("s2_op", C.c_int32), ("r_op", C.c_int32)]


class L11rDesc(C.Structure):
    _fields_ = [("nl", C.c_int32), ("nr", C.c_int32),
                ("diml", C.POINTER(C.c_int64)), ("dimr", C.POINTER(C.c_int64)),
                ("q", C.c_int32), ("nsegs", C.c_int32),
                ("seg_l", C.POINTER(C.c_int32)), ("seg_s1", C.POINTER(C.c_int32)),
                ("seg_s2", C.POINTER(C.c_int32)), ("seg_r", C.POINTER(C.c_int32)),
                ("nopsl", C.c_int32), ("nopsr", C.c_int32),
                ("opsl", C.POINTER(Operator)), ("opsr", C.POINTER(Operator)),
                ("nsops", C.c_int32), ("sops", C.POINTER(C.c_double)),
                ("nterms", C.c_int32), ("terms", C.POINTER(Term4)),
                ("data_location", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("max_subspace", C.c_int32), ("restart_keep", C.c_int32), ("fp64_refine", C.c_int32),
                ("refine_ratio", C.c_double), ("anchor_prec", C.c_int32),
                ("vector_arith", C.c_int32), ("autotune", C.c_int32), ("graphs", C.c_int32),
                ("anchor_update", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("energy", C.c_double), ("resnorm", C.c_double), ("iters", C.c_int32),
                ("projections", C.c_int32), ("fp64_projections", C.c_int32),
                ("restarts", C.c_int32), ("small_eig_sweeps", C.c_int32),
                ("converged", C.c_int32), ("anchor_updates", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("records", C.c_int64), ("flops", C.c_int64),
                ("tiles_stage1", C.c_int64), ("tiles_stage2", C.c_int64),
                ("device_bytes", C.c_int64), ("tc_schedule", C.c_int32 * 2),
                ("tc_tune_us", (C.c_float * TILE_SCHEDULES) * 2)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_[:6]}
        d["tc_schedule"] = list(self.tc_schedule)
        d["tc_tune_us"] = [list(r) for r in self.tc_tune_us]
        return d


# every exported symbol and its signature (checked by the CPU test suite)
SIGNATURES = {
    "dmrg_options_default": (None, [C.POINTER(Options)]),
    "dmrg_plan_create": (C.c_int, [C.POINTER(SuperblockDesc), C.POINTER(Options), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "dmrg_plan_create_l11r": (C.c_int, [C.POINTER(L11rDesc), C.POINTER(Options), C.c_void_p,
                                        C.POINTER(C.c_void_p)]),
    "dmrg_plan_destroy": (None, [C.c_void_p]),
    "dmrg_plan_trim": (C.c_int, [C.c_void_p]),
    "dmrg_plan_get_stats": (C.c_int, [C.c_void_p, C.POINTER(PlanStats)]),
    "dmrg_plan_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dmrg_plan_set_tile_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int32, C.c_int32, C.c_void_p]),
    "dmrg_project": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_project_prec": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_project_digits": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_diagonal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_gemv_trans": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "dmrg_gemv_trans_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_state_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "dmrg_state_destroy": (None, [C.c_void_p]),
    "dmrg_davidson_step": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "dmrg_state_get_info": (C.c_int, [C.c_void_p, C.POINTER(SolveInfo)]),
    "dmrg_state_ritz": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg_davidson_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo),
                                      C.c_void_p]),
    "dmrg_davidson_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(SolveInfo), C.c_void_p]),
    "dmrg_davidson_solve_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32,
                                              C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                              C.POINTER(SolveInfo), C.c_void_p]),
    "dmrg_davidson_solve_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(SolveInfo), C.c_void_p]),
    "dmrg_precision_available": (C.c_int32, [C.c_int]),
    "dmrg_kernel_launches": (C.c_int64, []),
    "dmrg_status_string": (C.c_char_p, [C.c_int]),
    "dmrg_last_error": (C.c_char_p, []),
    "dmrg_version": (C.c_char_p, []),
}

_lib = None


def load(path: Optional[str] = None):
    """Load the shared library (no CUDA context is created here)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        msg = load().dmrg_last_error().decode()
        if status == 5:
            raise NotConverged(status, msg)
        raise DmrgError(status, msg)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA is not available: this library has no CPU path")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_vec(t, n, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {n} elements")


@dataclass
class _Marshalled:
    desc: object
    keep: list


def _ops_array(ops, keep):
    arr = (Operator * max(1, len(ops)))()
    for o, op in enumerate(ops):
        items = sorted(op.blocks.items())
        blocks = (Block * max(1, len(items)))()
        for b, ((i, j), M) in enumerate(items):
            M = np.ascontiguousarray(M, dtype=np.float64)
            keep.append(M)
            blocks[b] = Block(i, j, M.shape[0], M.shape[1], M.shape[1], M.ctypes.data)
        keep.append(blocks)
        arr[o] = Operator(len(items), blocks)
    keep.append(arr)
    return arr


def marshal_l11r(sb) -> _Marshalled:
    """l-1-1-r superblock container -> C descriptor (host data); keeps the arrays alive."""
    keep = []
    diml = np.ascontiguousarray(sb.dl, dtype=np.int64)
    dimr = np.ascontiguousarray(sb.dr, dtype=np.int64)
    segs = np.asarray(sb.segs, dtype=np.int32).reshape(-1, 4)
    cols = [np.ascontiguousarray(segs[:, c]) for c in range(4)]
    q = len(sb.qs)
    sops = np.ascontiguousarray(np.stack(sb.sops).reshape(-1) if sb.sops else np.zeros(1), dtype=np.float64)
    keep += [diml, dimr, sops, *cols]
    opsl, opsr = _ops_array(sb.opsl, keep), _ops_array(sb.opsr, keep)
    terms = (Term4 * max(1, len(sb.terms)))()
    for t, (coef, a, s1, s2, b) in enumerate(sb.terms):
        terms[t] = Term4(float(coef), int(a), int(s1), int(s2), int(b))
    keep.append(terms)
    i32 = C.POINTER(C.c_int32)
    desc = L11rDesc(len(diml), len(dimr), diml.ctypes.data_as(C.POINTER(C.c_int64)),
                    dimr.ctypes.data_as(C.POINTER(C.c_int64)), q, len(segs),
                    cols[0].ctypes.data_as(i32), cols[1].ctypes.data_as(i32),
                    cols[2].ctypes.data_as(i32), cols[3].ctypes.data_as(i32),
                    len(sb.opsl), len(sb.opsr), opsl, opsr, len(sb.sops),
                    sops.ctypes.data_as(C.POINTER(C.c_double)), len(sb.terms), terms, 0)
    return _Marshalled(desc, keep)


def marshal(sb) -> _Marshalled:
    """Superblock container -> C descriptor (host data); keeps the arrays alive."""
    keep = []
    dimL = np.ascontiguousarray(sb.dL, dtype=np.int64)
    dimR = np.ascontiguousarray(sb.dR, dtype=np.int64)
    pairs = np.asarray(sb.pairs, dtype=np.int32).reshape(-1, 2)
    pi = np.ascontiguousarray(pairs[:, 0])
    pk = np.ascontiguousarray(pairs[:, 1])
    keep += [dimL, dimR, pi, pk]

    def ops_array(ops):
        arr = (Operator * max(1, len(ops)))()
        for o, op in enumerate(ops):
            items = sorted(op.blocks.items())
            blocks = (Block * max(1, len(items)))()
            for b, ((i, j), M) in enumerate(items):
                M = np.ascontiguousarray(M, dtype=np.float64)
                keep.append(M)
                blocks[b] = Block(i, j, M.shape[0], M.shape[1], M.shape[1], M.ctypes.data)
            keep.append(blocks)
            arr[o] = Operator(len(items), blocks)
        keep.append(arr)
        return arr

    opsL, opsR = ops_array(sb.opsL), ops_array(sb.opsR)
    terms = (Term * max(1, len(sb.terms)))()
    for t, (coef, a, b) in enumerate(sb.terms):
        terms[t] = Term(float(coef), int(a), int(b))
    keep.append(terms)
    desc = SuperblockDesc(
        len(dimL), len(dimR),
        dimL.ctypes.data_as(C.POINTER(C.c_int64)), dimR.ctypes.data_as(C.POINTER(C.c_int64)),
        len(pi), pi.ctypes.data_as(C.POINTER(C.c_int32)), pk.ctypes.data_as(C.POINTER(C.c_int32)),
        len(sb.opsL), len(sb.opsR), opsL, opsR, len(sb.terms), terms, 0)
    return _Marshalled(desc, keep)


def options(prec="fp64", tol=1e-10, max_iter=1000, max_subspace=20, restart_keep=2, fp64_refine=True,
            refine_ratio=0.0, anchor_prec="fp64", vector_arith="split", autotune=True,
            graphs=True, anchor_update=True) -> Options:
    o = Options()
    load().dmrg_options_default(C.byref(o))
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.tol = tol
    o.max_iter = max_iter
    o.max_subspace = max_subspace
    o.restart_keep = restart_keep
    o.fp64_refine = int(bool(fp64_refine))
    o.refine_ratio = refine_ratio
    o.anchor_prec = PREC[anchor_prec] if isinstance(anchor_prec, str) else int(anchor_prec)
    o.vector_arith = VEC[vector_arith] if isinstance(vector_arith, str) else int(vector_arith)
    o.autotune = int(bool(autotune))
    o.graphs = int(bool(graphs))
    o.anchor_update = int(bool(anchor_update))
    return o


class Plan:
    """A planned superblock problem on the current CUDA device: dmrg_plan_create for an LR
    superblock, dmrg_plan_create_l11r for one in the l-1-1-r form (a container with
    ``segs`` and ``sops``)."""

    def __init__(self, sb, stream=None, **opts):
        torch = _torch()
        self.lib = load()
        self.opt = options(**opts)
        h = C.c_void_p()
        if hasattr(sb, "segs"):
            m = marshal_l11r(sb)
            _check(self.lib.dmrg_plan_create_l11r(C.byref(m.desc), C.byref(self.opt),
                                                  _stream_ptr(stream), C.byref(h)))
        else:
            m = marshal(sb)
            _check(self.lib.dmrg_plan_create(C.byref(m.desc), C.byref(self.opt), _stream_ptr(stream),
                                             C.byref(h)))
        self.handle = h
        st = PlanStats()
        _check(self.lib.dmrg_plan_get_stats(self.handle, C.byref(st)))
        self.stats = st.as_dict()
        self.n = int(st.n)
        self.device = torch.cuda.current_device()

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dmrg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def trim(self):
        """dmrg_plan_trim: free the Davidson workspace and host-solve vectors kept between
        solves."""
        _check(self.lib.dmrg_plan_trim(self.handle))

    def get_stats(self):
        st = PlanStats()
        _check(self.lib.dmrg_plan_get_stats(self.handle, C.byref(st)))
        self.stats = st.as_dict()
        return self.stats

    def autotune(self, prec="bf16x3", stream=None):
        """dmrg_plan_autotune: time the tile schedules of the tensor-core GEMM stages."""
        _check(self.lib.dmrg_plan_autotune(self.handle, PREC[prec] if isinstance(prec, str) else int(prec),
                                           _stream_ptr(stream)))
        return self.get_stats()

    def set_tile_schedule(self, stage1, stage2, prec="bf16x3", stream=None):
        """dmrg_plan_set_tile_schedule: fix the tile schedules of the two GEMM stages."""
        _check(self.lib.dmrg_plan_set_tile_schedule(
            self.handle, PREC[prec] if isinstance(prec, str) else int(prec), int(stage1), int(stage2),
            _stream_ptr(stream)))
        return self.get_stats()

    def project(self, x, y=None, prec=None, stream=None):
        torch = _torch()
        _check_vec(x, self.n, "x")
        if y is None:
            y = torch.empty_like(x)
        _check_vec(y, self.n, "y")
        p = self.opt.prec if prec is None else (PREC[prec] if isinstance(prec, str) else prec)
        _check(self.lib.dmrg_project_prec(self.handle, int(p), x.data_ptr(), y.data_ptr(),
                                          _stream_ptr(stream)))
        return y

    def project_digits(self, x, digits, y=None, stream=None):
        """dmrg_project_digits: y = H x on the FP64_TC path with the leading `digits` digits."""
        torch = _torch()
        _check_vec(x, self.n, "x")
        if y is None:
            y = torch.empty_like(x)
        _check_vec(y, self.n, "y")
        _check(self.lib.dmrg_project_digits(self.handle, int(digits), x.data_ptr(), y.data_ptr(),
                                            _stream_ptr(stream)))
        return y

    def diagonal(self, stream=None):
        torch = _torch()
        d = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(self.lib.dmrg_diagonal(self.handle, d.data_ptr(), _stream_ptr(stream)))
        return d

    def solve(self, x0, x_out=None, stream=None, raise_on_nonconvergence=True):
        torch = _torch()
        _check_vec(x0, self.n, "x0")
        if x_out is None:
            x_out = torch.empty_like(x0)
        _check_vec(x_out, self.n, "x_out")
        info = SolveInfo()
        st = self.lib.dmrg_davidson_solve(self.handle, x0.data_ptr(), x_out.data_ptr(),
                                          C.byref(info), _stream_ptr(stream))
        if st == 5 and not raise_on_nonconvergence:
            return x_out, info.as_dict()
        _check(st)
        return x_out, info.as_dict()

    def solve_host(self, x0: np.ndarray, x_out: Optional[np.ndarray] = None, stream=None):
        """Solve with host buffers: the copies in and out are part of the call."""
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        if x0.shape != (self.n,):
            raise ValueError("x0 has the wrong length")
        if x_out is None:
            x_out = np.empty(self.n, dtype=np.float64)
        info = SolveInfo()
        _check(self.lib.dmrg_davidson_solve_host(self.handle, x0.ctypes.data, x_out.ctypes.data,
                                                 C.byref(info), _stream_ptr(stream)))
        return x_out, info.as_dict()

    def solve_block(self, X0, nev, X_out=None, stream=None, raise_on_nonconvergence=True):
        """dmrg_davidson_solve_block: the nev lowest eigenpairs from a start block X0 given as a
        contiguous CUDA float64 tensor of shape (block, n) (row c = start vector c, i.e. a
        column-major n x block matrix).  Returns (X of shape (nev, n), energies, resnorms, info)."""
        torch = _torch()
        if not (isinstance(X0, torch.Tensor) and X0.is_cuda and X0.dtype == torch.float64
                and X0.is_contiguous() and X0.dim() == 2 and X0.shape[1] == self.n):
            raise ValueError(f"X0 must be a contiguous CUDA float64 tensor of shape (block, {self.n})")
        block = X0.shape[0]
        if X_out is None:
            X_out = torch.empty((nev, self.n), dtype=torch.float64, device=X0.device)
        if not (X_out.is_contiguous() and tuple(X_out.shape) == (nev, self.n) and X_out.dtype == torch.float64):
            raise ValueError(f"X_out must be a contiguous float64 tensor of shape ({nev}, {self.n})")
        e = (C.c_double * nev)()
        r = (C.c_double * nev)()
        info = SolveInfo()
        st = self.lib.dmrg_davidson_solve_block(self.handle, int(nev), int(block), X0.data_ptr(), self.n,
                                                X_out.data_ptr(), self.n, e, r, C.byref(info),
                                                _stream_ptr(stream))
        if not (st == 5 and not raise_on_nonconvergence):
            _check(st)
        return X_out, list(e), list(r), info.as_dict()

    def state(self, x0, stream=None) -> "DavidsonState":
        return DavidsonState(self, x0, stream)


class DavidsonState:
    def __init__(self, plan: Plan, x0, stream=None):
        _check_vec(x0, plan.n, "x0")
        self.plan = plan
        self.lib = plan.lib
        h = C.c_void_p()
        _check(self.lib.dmrg_state_create(plan.handle, x0.data_ptr(), _stream_ptr(stream), C.byref(h)))
        self.handle = h

    def step(self, stream=None) -> bool:
        conv = C.c_int32(0)
        _check(self.lib.dmrg_davidson_step(self.handle, _stream_ptr(stream), C.byref(conv)))
        return bool(conv.value)

    def info(self) -> dict:
        info = SolveInfo()
        _check(self.lib.dmrg_state_get_info(self.handle, C.byref(info)))
        return info.as_dict()

    def ritz(self, stream=None):
        torch = _torch()
        x = torch.empty(self.plan.n, dtype=torch.float64, device="cuda")
        _check(self.lib.dmrg_state_ritz(self.handle, x.data_ptr(), _stream_ptr(stream)))
        return x

    def close(self):
        if getattr(self, "handle", None):
            self.lib.dmrg_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans, x0s, x_outs=None, stream=None, raise_on_nonconvergence=True):
    """dmrg_davidson_solve_batched over a list of plans and device start vectors."""
    torch = _torch()
    nb = len(plans)
    if len(x0s) != nb:
        raise ValueError("one start vector per plan")
    if x_outs is None:
        x_outs = [torch.empty_like(x) for x in x0s]
    for p, x, y in zip(plans, x0s, x_outs):
        _check_vec(x, p.n, "x0")
        _check_vec(y, p.n, "x_out")
    hp = (C.c_void_p * max(1, nb))(*[p.handle.value for p in plans])
    hx = (C.c_void_p * max(1, nb))(*[x.data_ptr() for x in x0s])
    hy = (C.c_void_p * max(1, nb))(*[y.data_ptr() for y in x_outs])
    infos = (SolveInfo * max(1, nb))()
    st = load().dmrg_davidson_solve_batched(hp, nb, hx, hy, infos, _stream_ptr(stream))
    if not (st == 5 and not raise_on_nonconvergence):
        _check(st)
    return x_outs, [infos[i].as_dict() for i in range(nb)]


def tc_available(prec: str = "bf16x3") -> bool:
    return bool(load().dmrg_precision_available(PREC[prec]))


def kernel_launches() -> int:
    return int(load().dmrg_kernel_launches())


def gemv_trans(V, k: int, w, stream=None):
    """s = V[:, :k]^T w for a column-major V given as a (kcols, ldv) row-major tensor."""
    torch = _torch()
    if V.dtype != torch.float64 or not V.is_cuda or not V.is_contiguous():
        raise ValueError("V must be a contiguous CUDA float64 tensor of shape (columns, ldv)")
    n = w.numel()
    ldv = V.shape[1]
    s = torch.empty(k, dtype=torch.float64, device="cuda")
    _check(load().dmrg_gemv_trans(V.data_ptr(), ldv, n, k, w.data_ptr(), s.data_ptr(),
                                  _stream_ptr(stream)))
    return s


def gemv_trans_noalloc(V, k: int, w, s=None, stream=None):
    """Same product as gemv_trans through the allocation-free entry point; the library
    allocates nothing (pass ``s`` to keep the caller's side free of allocations too)."""
    torch = _torch()
    if V.dtype != torch.float64 or not V.is_cuda or not V.is_contiguous():
        raise ValueError("V must be a contiguous CUDA float64 tensor of shape (columns, ldv)")
    n = w.numel()
    if s is None:
        s = torch.empty(k, dtype=torch.float64, device="cuda")
    _check(load().dmrg_gemv_trans_noalloc(V.data_ptr(), V.shape[1], n, k, w.data_ptr(),
                                          s.data_ptr(), _stream_ptr(stream)))
    return s
