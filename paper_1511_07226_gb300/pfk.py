"""Thin ctypes binding of the C ABI in include/pfk.h (argument marshalling only).

Every computation runs in the CUDA kernels of libpfk.so; this module only
converts Python / NumPy / PyTorch arguments to pointers and sizes.  There is no
fallback: if the library is missing or no GPU is present, calls raise.

Names follow the C ABI: ``create_context``, ``create_operator``,
``create_preconditioner``, ``solve``; the classes wrap the opaque handles.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfk.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pfk.h")

PFK_OK, PFK_PENDING = 0, 1
STATUS_NAMES = {0: "ok", 1: "pending", -1: "invalid", -2: "oom", -3: "cuda", -4: "breakdown",
                -5: "not_converged", -6: "timeout", -7: "cancelled", -8: "busy"}
METHODS = {"fcg": 0, "pipefcg": 1, "gcr": 2, "pipegcr": 3, "fgmres": 4, "pipefgmres": 5, "pipefcg_naive": 6,
           "pipegcr_w": 7, "pipefcg_theta": 8}
PC_KINDS = {"none": 0, "jacobi": 1, "inner_pcg": 2, "chebyshev": 3, "noisy": 4, "block_upper": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}
OP_KINDS = {"stencil2d": 0, "stencil3d": 1, "csr": 2}
STORAGE = {"matrix_free": 0, "csr": 1}
HISTORY_FIELDS = 4
MAX_MMAX = 32


class OperatorDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("storage", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("nz", C.c_int32), ("eta", C.c_void_p), ("eta_on_device", C.c_int32), ("vel", C.c_double * 3),
                ("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("vals", C.c_void_p), ("csr_on_device", C.c_int32)]


class PcDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("inner_iters", C.c_int32), ("precision", C.c_int32),
                ("cheb_lo", C.c_double), ("cheb_hi", C.c_double)]


class SolveParams(C.Structure):
    _fields_ = [("method", C.c_int32), ("mmax", C.c_int32), ("truncation", C.c_int32), ("norm", C.c_int32),
                ("rtol", C.c_double), ("atol", C.c_double), ("maxit", C.c_int32), ("max_restarts", C.c_int32),
                ("sigma", C.c_double), ("true_residual_check", C.c_int32), ("graph_iters", C.c_int32),
                ("history", C.c_void_p), ("history_capacity", C.c_int32), ("profile", C.c_int32),
                ("persistent", C.c_int32), ("barrier_timeout_us", C.c_int32)]


class InnerSolve(C.Structure):
    _fields_ = [("method", C.c_int32), ("mmax", C.c_int32), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("pad", C.c_int32)]


class ServerParams(C.Structure):
    _fields_ = [("workers", C.c_int32), ("queue_capacity", C.c_int32), ("memory_budget", C.c_int64),
                ("order", C.c_int32), ("group_max_n", C.c_int32), ("group_ctas", C.c_int32),
                ("reserved", C.c_int32)]


SERVE_ORDERS = {"fifo": 0, "smallest_first": 1}
PERSISTENT = {"auto": 0, "off": 1, "on": 2}


class Request(C.Structure):
    _fields_ = [("op", OperatorDesc), ("pc", PcDesc), ("params", SolveParams), ("b", C.c_void_p),
                ("x0", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("restarts", C.c_int32),
                ("breakdowns", C.c_int32), ("replacements", C.c_int32), ("history_len", C.c_int32),
                ("rho0", C.c_double), ("rho_final", C.c_double), ("rnorm_true", C.c_double),
                ("bnorm", C.c_double), ("time_ms", C.c_double), ("pass_launches", C.c_int32),
                ("kernel_launches", C.c_int32), ("pass_bytes", C.c_double), ("pass_flops", C.c_double),
                ("pass_ms", C.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_lib = None

_SIGS = {
    "pfk_abi_version": (C.c_int, []),
    "pfk_last_error": (C.c_char_p, [C.c_void_p]),
    "pfk_create_context": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pfk_destroy_context": (C.c_int, [C.c_void_p]),
    "pfk_create_operator": (C.c_int, [C.c_void_p, C.POINTER(OperatorDesc), C.POINTER(C.c_void_p)]),
    "pfk_destroy_operator": (C.c_int, [C.c_void_p]),
    "pfk_operator_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "pfk_operator_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfk_create_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(PcDesc), C.POINTER(C.c_void_p)]),
    "pfk_destroy_preconditioner": (C.c_int, [C.c_void_p]),
    "pfk_create_noisy_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int, C.c_int,
                                                  C.POINTER(C.c_void_p)]),
    "pfk_create_block_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                  C.POINTER(InnerSolve), C.POINTER(C.c_void_p)]),
    "pfk_pc_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pfk_default_params": (C.c_int, [C.POINTER(SolveParams)]),
    "pfk_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveParams), C.c_void_p, C.c_void_p,
                            C.c_int, C.POINTER(SolveInfo)]),
    "pfk_method_storage_vectors": (C.c_int, [C.c_int, C.c_int]),
    "pfk_solve_workspace_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_int64)]),
    "pfk_pc_workspace_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "pfk_pc_apply_inner_pcg_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "pfk_solve_batched": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(PcDesc),
                                    C.POINTER(SolveParams), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                    C.c_int, C.POINTER(SolveInfo)]),
    "pfk_solve_grouped": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(PcDesc),
                                    C.POINTER(SolveParams), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                    C.c_int, C.POINTER(SolveInfo)]),
    "pfk_server_create": (C.c_int, [C.c_void_p, C.POINTER(ServerParams), C.POINTER(C.c_void_p)]),
    "pfk_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "pfk_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(SolveInfo), C.POINTER(C.c_double),
                           C.c_int]),
    "pfk_server_destroy": (C.c_int, [C.c_void_p]),
    "pfk_probe_fp64_fma": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
}


def header_symbols() -> list:
    """Function names declared in include/pfk.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pfk_\w+)\s*\(", src)))


def load():
    """Loads libpfk.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() first")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PfkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, ctx=None):
    if status != PFK_OK:
        lib = load()
        msg = lib.pfk_last_error(ctx).decode(errors="replace")
        raise PfkError(status, msg)


def _torch():
    import torch
    return torch


def _is_cuda_tensor(a) -> bool:
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(a, torch.Tensor) and a.is_cuda


def _dev_f64(a, device):
    """A contiguous float64 CUDA tensor holding `a` (copied from host if needed)."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=torch.float64)
    else:
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    return t.contiguous()


class Context:
    """pfk_context on one CUDA device, ordered on a CUDA stream (torch's current one by default)."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the pfk library has no CPU path")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(lib.pfk_create_context(device, C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().pfk_destroy_context(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    def __init__(self, ctx: Context, desc: OperatorDesc, keep=()):
        self.ctx = ctx
        h = C.c_void_p()
        _check(load().pfk_create_operator(ctx.h, C.byref(desc), C.byref(h)), ctx.h)
        self.h = h
        n = C.c_int64()
        _check(load().pfk_operator_size(h, C.byref(n)))
        self.n = int(n.value)

    @classmethod
    def stencil(cls, ctx: Context, dims, eta, vel=(0.0, 0.0, 0.0), storage: str = "matrix_free"):
        nx, ny, nz = (tuple(int(d) for d in dims) + (1, 1))[:3]
        d = OperatorDesc()
        d.kind = OP_KINDS["stencil3d" if nz > 1 else "stencil2d"]
        d.storage = STORAGE[storage]
        d.nx, d.ny, d.nz = nx, ny, nz
        if _is_cuda_tensor(eta):
            e = _dev_f64(eta, ctx.device)
            d.eta, d.eta_on_device = e.data_ptr(), 1
        else:
            e = np.ascontiguousarray(eta, dtype=np.float64)
            d.eta, d.eta_on_device = e.ctypes.data, 0
        for i in range(3):
            d.vel[i] = float((tuple(vel) + (0.0, 0.0, 0.0))[i])
        op = cls(ctx, d)
        op.dims = (nx, ny, nz)
        return op

    @classmethod
    def csr(cls, ctx: Context, rowptr, colidx, vals):
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        va = np.ascontiguousarray(vals, dtype=np.float64)
        d = OperatorDesc()
        d.kind = OP_KINDS["csr"]
        d.n, d.nnz = len(rp) - 1, len(va)
        d.rowptr, d.colidx, d.vals, d.csr_on_device = rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0
        return cls(ctx, d)

    def apply(self, x):
        """y = A x on the device (x: array or tensor of length n); returns a CUDA tensor."""
        torch = _torch()
        xd = _dev_f64(x, self.ctx.device)
        y = torch.empty_like(xd)
        _check(load().pfk_operator_apply(self.ctx.h, self.h, C.c_void_p(xd.data_ptr()), C.c_void_p(y.data_ptr())),
               self.ctx.h)
        return y

    def close(self):
        if getattr(self, "h", None):
            load().pfk_destroy_operator(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Preconditioner:
    def __init__(self, ctx: Context, op: Operator, kind: str = "jacobi", inner_iters: int = 4,
                 precision: str = "fp64", cheb_lo: float = 0.0, cheb_hi: float = 0.0):
        self.ctx, self.op = ctx, op
        d = PcDesc()
        d.kind = PC_KINDS[kind]
        d.inner_iters = int(inner_iters)
        d.precision = PRECISIONS[precision]
        d.cheb_lo, d.cheb_hi = float(cheb_lo), float(cheb_hi)
        h = C.c_void_p()
        _check(load().pfk_create_preconditioner(ctx.h, op.h, C.byref(d), C.byref(h)), ctx.h)
        self.h = h
        self.kind, self.precision = kind, precision

    @classmethod
    def noisy(cls, ctx: Context, op: Operator, eta: float, bank):
        """B(r) = r + eta ||r|| xi_j / ||xi_j||, xi_j = row j mod count of `bank` (the toy experiment's
        preconditioner); j counts applications since creation."""
        bk = np.ascontiguousarray(bank, dtype=np.float64)
        self = cls.__new__(cls)
        self.ctx, self.op = ctx, op
        h = C.c_void_p()
        _check(load().pfk_create_noisy_preconditioner(ctx.h, op.h, float(eta), C.c_void_p(bk.ctypes.data),
                                                      int(bk.shape[0]), 0, C.byref(h)), ctx.h)
        self.h = h
        self.kind, self.precision = "noisy", "fp64"
        return self

    @classmethod
    def block_upper(cls, ctx: Context, K: Operator, Bt: Operator, schur_diag, inner_method: str = "pipefcg",
                    inner_mmax: int = 30, inner_rtol: float = 1e-3, inner_maxit: int = 100):
        """[K_hat B^T; 0 S_hat]^-1 with K_hat^-1 an inner solve (the Stokes nesting of Sec. 6)."""
        sd = np.ascontiguousarray(schur_diag, dtype=np.float64)
        inner = InnerSolve()
        inner.method, inner.mmax = METHODS[inner_method], int(inner_mmax)
        inner.rtol, inner.maxit = float(inner_rtol), int(inner_maxit)
        self = cls.__new__(cls)
        self.ctx, self.op, self.keep = ctx, Bt, (K, Bt)
        h = C.c_void_p()
        _check(load().pfk_create_block_preconditioner(ctx.h, K.h, Bt.h, C.c_void_p(sd.ctypes.data), C.byref(inner),
                                                      C.byref(h)), ctx.h)
        self.h = h
        self.kind, self.precision = "block_upper", "fp64"
        return self

    def apply(self, v):
        torch = _torch()
        vd = _dev_f64(v, self.ctx.device)
        y = torch.empty_like(vd)
        _check(load().pfk_pc_apply(self.ctx.h, self.h, C.c_void_p(vd.data_ptr()), C.c_void_p(y.data_ptr())),
               self.ctx.h)
        return y

    def close(self):
        if getattr(self, "h", None):
            load().pfk_destroy_preconditioner(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_params() -> SolveParams:
    p = SolveParams()
    _check(load().pfk_default_params(C.byref(p)))
    return p


def make_params(method="pipefcg", mmax=30, truncation="standard", norm="natural", rtol=1e-8, atol=0.0,
                maxit=10000, max_restarts=20, sigma=float("nan"), true_residual_check=True,
                graph_iters=8, profile=False, persistent="auto", barrier_timeout_us=0) -> SolveParams:
    p = default_params()
    p.method = METHODS[method]
    p.mmax = int(mmax)
    p.truncation = 0 if truncation == "standard" else 1
    p.norm = 0 if norm == "natural" else 1
    p.rtol, p.atol = float(rtol), float(atol)
    p.maxit, p.max_restarts = int(maxit), int(max_restarts)
    p.sigma = float(sigma)
    p.true_residual_check = 1 if true_residual_check else 0
    p.graph_iters = int(graph_iters)
    p.profile = 1 if profile else 0
    p.persistent = PERSISTENT[persistent]
    p.barrier_timeout_us = int(barrier_timeout_us)
    return p


def solve(ctx: Context, op: Operator, pc: Preconditioner | None, b, x0=None, history: int = 0,
          raise_on_error: bool = False, **kw):
    """Solves A x = b.

    b (and x0) may be NumPy arrays (host path: the library stages them) or CUDA
    tensors (device path).  Returns (x, info dict, history array or None).
    """
    lib = load()
    prm = make_params(**kw)
    hist = None
    if history:
        hist = np.full((history, HISTORY_FIELDS), np.nan)
        prm.history = hist.ctypes.data
        prm.history_capacity = history
    info = SolveInfo()
    if _is_cuda_tensor(b):
        torch = _torch()
        bd = _dev_f64(b, ctx.device)
        xd = torch.zeros_like(bd) if x0 is None else _dev_f64(x0, ctx.device).clone()
        st = lib.pfk_solve(ctx.h, op.h, pc.h if pc else None, C.byref(prm), C.c_void_p(bd.data_ptr()),
                           C.c_void_p(xd.data_ptr()), 1, C.byref(info))
        x = xd
    else:
        bh = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(bh) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        st = lib.pfk_solve(ctx.h, op.h, pc.h if pc else None, C.byref(prm), C.c_void_p(bh.ctypes.data),
                           C.c_void_p(x.ctypes.data), 0, C.byref(info))
    d = info.as_dict()
    if st not in (PFK_OK, -4, -5) or (raise_on_error and st != PFK_OK):
        _check(st, ctx.h)
    d["message"] = lib.pfk_last_error(ctx.h).decode(errors="replace") if st != PFK_OK else ""
    if hist is not None:
        hist = hist[:min(info.history_len, history)]
    return x, d, hist


def probe_fp64_fma(ctx: Context, iters: int = 1 << 16) -> dict:
    """Measured FP64 FMA throughput of the device (the ALU roofline's denominator)."""
    tf, ms = C.c_double(), C.c_double()
    _check(load().pfk_probe_fp64_fma(ctx.h, int(iters), C.byref(tf), C.byref(ms)), ctx.h)
    return {"tflops": tf.value, "ms": ms.value, "iters": int(iters)}


NOALLOC_MAX_N = 262144


def pc_apply_inner_pcg_noalloc(ctx: Context, op: Operator, inner_iters: int, v, y=None):
    """y = B(v), FP64 inner Jacobi-PCG, through the allocation-free entry point.

    The library allocates nothing for this call (its scratch is a static device
    array); `y` may be given preallocated (a CUDA float64 tensor), otherwise this
    helper allocates it with torch before the call.
    """
    torch = _torch()
    vd = _dev_f64(v, ctx.device)
    if y is None:
        y = torch.empty_like(vd)
    _check(load().pfk_pc_apply_inner_pcg_noalloc(ctx.h, op.h, int(inner_iters), C.c_void_p(vd.data_ptr()),
                                                 C.c_void_p(y.data_ptr())), ctx.h)
    return y


def solve_batched(ctx: Context, ops, bs, x0s=None, pc_kind="inner_pcg", inner_iters=4, precision="fp64",
                  history: int = 0, block_threads: int = 0, **kw):
    """Solves independent systems ops[j] x_j = bs[j] in one persistent launch (PIPEFCG).

    bs / x0s are NumPy arrays (host path).  Returns (xs, infos, histories)."""
    lib = load()
    nsys = len(ops)
    prm = make_params(**kw)
    hist = None
    if history:
        hist = np.full((nsys, history, HISTORY_FIELDS), np.nan)
        prm.history = hist.ctypes.data
        prm.history_capacity = history
    d = PcDesc()
    d.kind = PC_KINDS[pc_kind]
    d.inner_iters = int(inner_iters)
    d.precision = PRECISIONS[precision]
    bh = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    xs = [np.zeros_like(b) if x0s is None else np.array(x0s[j], dtype=np.float64, copy=True)
          for j, b in enumerate(bh)]
    oparr = (C.c_void_p * nsys)(*[op.h.value for op in ops])
    barr = (C.c_void_p * nsys)(*[b.ctypes.data for b in bh])
    xarr = (C.c_void_p * nsys)(*[x.ctypes.data for x in xs])
    infos = (SolveInfo * nsys)()
    st = lib.pfk_solve_batched(ctx.h, nsys, oparr, C.byref(d), C.byref(prm), barr, xarr, 0, int(block_threads),
                               infos)
    if st not in (PFK_OK, -4, -5):
        _check(st, ctx.h)
    out = [infos[j].as_dict() for j in range(nsys)]
    hs = None
    if hist is not None:
        hs = [hist[j][:min(out[j]["history_len"], history)] for j in range(nsys)]
    return xs, out, hs


def solve_grouped(ctx: Context, ops, bs, x0s=None, pc_kind="inner_pcg", inner_iters=4, precision="fp64",
                  history: int = 0, ctas_per_system: int = 0, **kw):
    """Solves independent stencil systems ops[j] x_j = bs[j] with PIPEFCG,
    PIPEGCR or PIPEFGMRES (method=...) on the grouped persistent kernel (a
    group of CTAs per system, the systems sharing cooperative launches;
    ctas_per_system 1..64, 0 = about one per 4,096 cells, -1 = chosen by
    timing and cached).  bs / x0s are NumPy arrays (host path); the inner PCG
    runs in FP64 or FP32 (precision).  Returns (xs, infos, histories)."""
    lib = load()
    nsys = len(ops)
    prm = make_params(**kw)
    hist = None
    if history:
        hist = np.full((nsys, history, HISTORY_FIELDS), np.nan)
        prm.history = hist.ctypes.data
        prm.history_capacity = history
    d = PcDesc()
    d.kind = PC_KINDS[pc_kind]
    d.inner_iters = int(inner_iters)
    d.precision = PRECISIONS[precision]
    bh = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    xs = [np.zeros_like(b) if x0s is None else np.array(x0s[j], dtype=np.float64, copy=True)
          for j, b in enumerate(bh)]
    oparr = (C.c_void_p * nsys)(*[op.h.value for op in ops])
    barr = (C.c_void_p * nsys)(*[b.ctypes.data for b in bh])
    xarr = (C.c_void_p * nsys)(*[x.ctypes.data for x in xs])
    infos = (SolveInfo * nsys)()
    st = lib.pfk_solve_grouped(ctx.h, nsys, oparr, C.byref(d), C.byref(prm), barr, xarr, 0, int(ctas_per_system),
                               infos)
    if st not in (PFK_OK, -4, -5, -6):
        _check(st, ctx.h)
    out = [infos[j].as_dict() for j in range(nsys)]
    hs = None
    if hist is not None:
        hs = [hist[j][:min(out[j]["history_len"], history)] for j in range(nsys)]
    return xs, out, hs


class Server:
    """Continuous-batching solve server (pfk_server_*): submit requests at any
    time, poll for results.  Requests carry host arrays, which are copied at
    submission; each result is bitwise that of the same request solved alone."""

    def __init__(self, ctx: Context, workers: int = 4, queue_capacity: int = 0, memory_budget: int = 0,
                 order: str = "fifo", group_max_n: int = 0, group_ctas: int = 0):
        self.ctx = ctx
        p = ServerParams()
        p.workers, p.queue_capacity, p.memory_budget = int(workers), int(queue_capacity), int(memory_budget)
        p.order = SERVE_ORDERS[order]
        p.group_max_n, p.group_ctas = int(group_max_n), int(group_ctas)
        h = C.c_void_p()
        _check(load().pfk_server_create(ctx.h, C.byref(p), C.byref(h)), ctx.h)
        self.h = h
        self._n = {}

    def submit(self, dims, eta, b, x0=None, vel=(0.0, 0.0, 0.0), pc_kind="inner_pcg", inner_iters=4,
               precision="fp64", **kw) -> int:
        """Queues the stencil problem -div(eta grad u) (+ advection vel) = b; returns the ticket."""
        nx, ny, nz = (tuple(int(d) for d in dims) + (1, 1))[:3]
        r = Request()
        r.op.kind = OP_KINDS["stencil3d" if nz > 1 else "stencil2d"]
        r.op.nx, r.op.ny, r.op.nz = nx, ny, nz
        e = np.ascontiguousarray(eta, dtype=np.float64)
        r.op.eta, r.op.eta_on_device = e.ctypes.data, 0
        for i in range(3):
            r.op.vel[i] = float((tuple(vel) + (0.0, 0.0, 0.0))[i])
        r.pc.kind = PC_KINDS[pc_kind]
        r.pc.inner_iters = int(inner_iters)
        r.pc.precision = PRECISIONS[precision]
        r.params = make_params(**kw)
        bh = np.ascontiguousarray(b, dtype=np.float64)
        r.b = bh.ctypes.data
        xh = None
        if x0 is not None:
            xh = np.ascontiguousarray(x0, dtype=np.float64)
            r.x0 = xh.ctypes.data
        t = C.c_uint64()
        _check(load().pfk_submit(self.h, C.byref(r), C.byref(t)))
        self._n[int(t.value)] = bh.size
        return int(t.value)

    def submit_csr(self, rowptr, colidx, vals, b, x0=None, pc_kind="jacobi", **kw) -> int:
        """Queues a general sparse system (CSR, host arrays) A x = b; returns the ticket."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        va = np.ascontiguousarray(vals, dtype=np.float64)
        r = Request()
        r.op.kind = OP_KINDS["csr"]
        r.op.n, r.op.nnz = len(rp) - 1, len(va)
        r.op.rowptr, r.op.colidx, r.op.vals, r.op.csr_on_device = rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0
        r.pc.kind = PC_KINDS[pc_kind]
        r.params = make_params(**kw)
        bh = np.ascontiguousarray(b, dtype=np.float64)
        r.b = bh.ctypes.data
        if x0 is not None:
            xh = np.ascontiguousarray(x0, dtype=np.float64)
            r.x0 = xh.ctypes.data
        t = C.c_uint64()
        _check(load().pfk_submit(self.h, C.byref(r), C.byref(t)))
        self._n[int(t.value)] = bh.size
        return int(t.value)

    def poll(self, ticket: int, wait_ms: int = -1):
        """(x, info dict, latency_ms) once the request is done, None while pending."""
        x = np.empty(self._n[ticket])
        info = SolveInfo()
        lat = C.c_double()
        st = load().pfk_poll(self.h, C.c_uint64(ticket), C.c_void_p(x.ctypes.data), C.byref(info), C.byref(lat),
                             int(wait_ms))
        if st == PFK_PENDING:
            return None
        if st not in (PFK_OK, -4, -5):
            _check(st)
        del self._n[ticket]
        return x, info.as_dict(), float(lat.value)

    def close(self):
        if getattr(self, "h", None):
            load().pfk_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def storage_vectors(method: str, mmax: int) -> int:
    return int(load().pfk_method_storage_vectors(METHODS[method], int(mmax)))


def workspace_bytes(method: str, mmax: int, n: int) -> int:
    out = C.c_int64()
    _check(load().pfk_solve_workspace_bytes(METHODS[method], int(mmax), int(n), C.byref(out)))
    return int(out.value)
