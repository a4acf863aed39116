"""Python binding of the randomized QLP C ABI (include/rqlp.h).

Argument marshalling only: every step of the factorization runs in the CUDA
kernels of librqlp.so.  Device memory (outputs and workspace) comes from
torch; the work is enqueued on torch's current CUDA stream.  There is no
CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librqlp.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "rqlp.h")

RQLP_OK = 0
RQLP_WARN_SHIFTED_CHOLQR = 1
STATUS = {0: "RQLP_OK", 1: "RQLP_WARN_SHIFTED_CHOLQR", -1: "RQLP_ERR_INVALID_ARG",
          -2: "RQLP_ERR_NONFINITE", -3: "RQLP_ERR_RANK_DEFICIENT", -4: "RQLP_ERR_TIMEOUT",
          -5: "RQLP_ERR_CUDA", -6: "RQLP_ERR_WORKSPACE", -7: "RQLP_ERR_UNSUPPORTED"}
PREC = {"fp64": 0, "bf16x3": 1, "bf16": 2, "fp8": 3, "tf32x3": 4, "tf32": 5, "fp64tc": 6}
F64, F32 = 0, 1

_c_i32, _c_i64, _c_sz, _c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p


class Opts(ctypes.Structure):
    _fields_ = [("q", _c_i32), ("d", _c_i32), ("pivot2", _c_i32), ("prec", _c_i32),
                ("block_b", _c_i32), ("debug_flags", _c_i32), ("spin_limit_ns", _c_i64),
                ("fixed_pivots", _c_i32), ("truncate_k", _c_i32), ("in_flight", _c_i32)]


class Problem(ctypes.Structure):
    """rqlp_problem: one problem of a batch (device pointers)."""
    _fields_ = [("A", _c_p), ("a_dtype", _c_i32), ("k", _c_i32), ("m", _c_i64), ("n", _c_i64),
                ("lda", _c_i64), ("p", _c_i32), ("reserved", _c_i32), ("Omega", _c_p),
                ("ldo", _c_i64), ("Q", _c_p), ("L", _c_p), ("P", _c_p), ("Lvalues", _c_p),
                ("piv0", _c_p), ("piv1", _c_p)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("branches", _c_i32), ("gemm_target_ctas", _c_i32), ("mma_max_splits", _c_i32),
                ("engine", _c_i32)]


# batch engines (include/rqlp.h, rqlp_batch_tuning.engine)
ENGINES = {"auto": 0, "graph": 1, "persistent": 2}


class RqlpError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, STATUS.get(code, "unknown"), code))


_lib = None

_SIGS = {
    "rqlp_status_string": (ctypes.c_char_p, [_c_i32]),
    "rqlp_version": (_c_i32, []),
    "rqlp_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i32, _c_i32, ctypes.POINTER(Opts)]),
    "rqlp": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_i32, _c_i32, _c_p, _c_i64,
                      ctypes.POINTER(Opts), _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p]),
    "rqlp_read_status": (_c_i32, [_c_p, _c_p]),
    "rqlp_rvalues": (_c_i32, [_c_p, _c_i64, _c_i64, _c_i32, _c_i32, ctypes.POINTER(Opts), _c_p,
                              _c_p]),
    "rqlp_brqlp_tol": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_i32, _c_i32,
                                ctypes.c_double, _c_p, _c_i64, ctypes.POINTER(Opts), _c_p, _c_p,
                                _c_p, _c_p, _c_p, _c_p, ctypes.POINTER(ctypes.c_int32), _c_p,
                                _c_sz, _c_p]),
    "rqlp_host_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i32, _c_i32, ctypes.POINTER(Opts),
                                         _c_i32]),
    "rqlp_host": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i32, _c_i32, _c_p,
                           ctypes.POINTER(Opts), _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz,
                           _c_p]),
    "rqlp_host_async": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i32, _c_i32, _c_p,
                                 ctypes.POINTER(Opts), _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                 _c_sz, _c_p]),
    "rqlp_stage_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i32, _c_i32]),
    "rqlp_sketch": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_p, _c_i64, _c_i32, _c_i32,
                             _c_p, _c_i64, _c_p, _c_sz, _c_p]),
    "rqlp_project": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_p, _c_i64, _c_i32, _c_i32,
                              _c_p, _c_i64, _c_p, _c_sz, _c_p]),
    "rqlp_orth": (_c_i32, [_c_p, _c_i64, _c_i32, _c_i64, _c_p, _c_i64, _c_p, _c_p, _c_sz, _c_p]),
    "rqlp_cpqr": (_c_i32, [_c_p, _c_i64, _c_i32, _c_i64, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p]),
    "rqlp_cpqr_static": (_c_i32, [_c_p, _c_i64, _c_i32, _c_i64, _c_p, _c_p, _c_p, _c_i32, _c_p]),
    "rqlp_selftest": (_c_i32, [_c_i32, _c_p, _c_p]),
    "rqlp_fp64_probe": (_c_i32, [_c_i32, _c_p, _c_p, _c_p]),
    "rqlp_batched_workspace_size": (_c_sz, [ctypes.POINTER(Problem), _c_i32, ctypes.POINTER(Opts),
                                            ctypes.POINTER(BatchTuning)]),
    "rqlp_batched_create": (_c_i32, [ctypes.POINTER(Problem), _c_i32, ctypes.POINTER(Opts),
                                     ctypes.POINTER(BatchTuning), _c_p, _c_sz, ctypes.POINTER(_c_p)]),
    "rqlp_batched_launch": (_c_i32, [_c_p, _c_p]),
    "rqlp_batched_status": (_c_i32, [_c_p, _c_p, _c_p]),
    "rqlp_batched_kernel_nodes": (_c_i32, [_c_p]),
    "rqlp_batched_engine": (_c_i32, [_c_p, ctypes.POINTER(_c_i64)]),
    "rqlp_batched_stage_times": (_c_i32, [_c_p, _c_p, _c_p, _c_p, _c_p]),
    "rqlp_batched_destroy": (None, [_c_p]),
    "rqlp_graph_create": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_i32, _c_i32, _c_p,
                                   _c_i64, ctypes.POINTER(Opts), _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                   _c_p, _c_sz, _c_p, ctypes.POINTER(_c_p)]),
    "rqlp_graph_launch": (_c_i32, [_c_p, _c_p]),
    "rqlp_graph_kernels": (_c_i32, [_c_p]),
    "rqlp_graph_destroy": (None, [_c_p]),
    "rqlp_backward_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i32, _c_i32, ctypes.POINTER(Opts)]),
    "rqlp_backward": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_i32, _c_i32, _c_p, _c_i64,
                               ctypes.POINTER(Opts), _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_i64,
                               _c_p, _c_sz, _c_p]),
    "rqlp_qlp_workspace_size": (_c_sz, [_c_i64, _c_i64, _c_i32, ctypes.POINTER(Opts)]),
    "rqlp_qlp": (_c_i32, [_c_p, _c_i32, _c_i64, _c_i64, _c_i64, _c_i32, ctypes.POINTER(Opts), _c_p,
                          _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p]),
    "rqlp_launch_count": (ctypes.c_longlong, []),
    "rqlp_profile_begin": (_c_i32, []),
    "rqlp_profile_end": (_c_i32, [_c_p, _c_p, _c_i32]),
}

PROFILE_CLASSES = ("products_with_A", "cpqr_of_B", "cholqr_gram", "cholqr_cholesky",
                   "cholqr_trinv", "cholqr_apply", "explicit_Q0", "prep_A", "assembly")


def launch_count() -> int:
    return int(lib().rqlp_launch_count())


def selftest(count: int = 1 << 20, stream=None):
    """Device arithmetic helpers against CUDA's operations (include/rqlp.h,
    rqlp_selftest): mismatches for FP64->FP32, FP32->FP64, reciprocal and
    reciprocal square root."""
    fails = (ctypes.c_int32 * 4)()
    _check(lib().rqlp_selftest(count, ctypes.cast(fails, _c_p), _stream(stream)), "rqlp_selftest")
    return list(fails)


def fp64_peak(iters: int = 1 << 14, reps: int = 5, stream=None) -> dict:
    """Measured FP64 FMA rate of this GPU in TFLOP/s (rqlp_fp64_probe timed
    with CUDA events on the launch stream; the best of `reps` launches after
    one warm-up)."""
    torch = _torch()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    flops = ctypes.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    best = None
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib().rqlp_fp64_probe(int(iters), _ptr(sink), ctypes.byref(flops), _stream(st)),
               "rqlp_fp64_probe")
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if r > 0 and (best is None or ms < best):
            best = ms
    return {"tflops": flops.value / (best / 1e3) / 1e12, "ms": best, "flops": flops.value,
            "how": "rqlp_fp64_probe: 8 independent FP64 FMA chains per thread, 4 x SMs CTAs "
                   "of 256 threads, %d steps; best of %d event-timed launches" % (iters, reps)}


def profile_begin():
    _check(lib().rqlp_profile_begin(), "rqlp_profile_begin")


def profile_end() -> dict:
    n = len(PROFILE_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(lib().rqlp_profile_end(ctypes.cast(ms, _c_p), ctypes.cast(cnt, _c_p), n),
           "rqlp_profile_end")
    return {name: (ms[i], int(cnt[i])) for i, name in enumerate(PROFILE_CLASSES)}


def header_symbols(path: str = HEADER):
    """Names of the functions include/rqlp.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rqlp\w*)\s*\(", text)))


def lib():
    """The loaded librqlp.so with its argument types declared (raises if not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librqlp.so is not built: run `python -m paper_1811_09334_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def opts(q=0, d=1, pivot2=True, prec="fp64", block_b=0, debug_flags=0, spin_limit_ns=0,
         fixed_pivots=False, truncate_k=False, in_flight=0) -> Opts:
    return Opts(int(q), int(d), 1 if pivot2 else 0, PREC[prec] if isinstance(prec, str) else int(prec),
                int(block_b), int(debug_flags), int(spin_limit_ns), 1 if fixed_pivots else 0,
                1 if truncate_k else 0, int(in_flight))


def _torch():
    import torch
    return torch


def _ptr(t) -> int:
    return t.data_ptr() if t is not None else None


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code: int, where: str):
    if code < 0:
        raise RqlpError(code, where)
    return code


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("A must be float64 or float32")


def _row_major(t, name):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s must be a 2-D row-major tensor (stride(1) == 1)" % name)
    return t.stride(0)


def workspace(nbytes: int, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def read_status(ws, stream=None) -> int:
    return lib().rqlp_read_status(ctypes.c_void_p(_ptr(ws)), _stream(stream))


def rqlp(A, k: int, p: int, Omega, q: int = 0, d: int = 1, pivot2: bool = True,
         prec: str = "fp64", block_b: int = 0, ws=None, out: Optional[dict] = None,
         stream=None, check: bool = True, debug_flags: int = 0, spin_limit_ns: int = 0,
         piv0=None, piv1=None, truncate_k: bool = False, rvalues: bool = True,
         in_flight: int = 0) -> dict:
    """Randomized QLP A ~= Q L P^T on the GPU (Algorithms 2.1, 2.2 and 4.1).

    A: (m, n) float64/float32 CUDA tensor, row-major.  Omega: (n, k + p)
    float64 CUDA tensor.  Returns a dict with Q, L, P, Lvalues, Rvalues (diag
    R0 of the CPQR of B), piv0, piv1, status (and ws, for reuse).  With
    check=True the stream is synchronized and a device-side error raises
    RqlpError.  Given piv0 (and piv1 for Algorithm 2.1), int32 CUDA tensors
    of at least k + p entries, the factorization is taken at those pivots
    (rqlp_opts.fixed_pivots).  truncate_k returns the rank-k truncation
    (Q m x k, L k x k, P n x k).  in_flight: how many factorizations the
    caller runs at once on separate streams (rqlp_opts.in_flight; the
    results do not change).
    """
    torch = _torch()
    m, n = A.shape
    l = k + p
    lda = _row_major(A, "A")
    ldo = _row_major(Omega, "Omega")
    if Omega.dtype != torch.float64 or tuple(Omega.shape) != (n, l):
        raise ValueError("Omega must be float64 of shape (n, k + p)")
    fixed = piv0 is not None
    if fixed:
        for t, need_n in ((piv0, l), (piv1, l)):
            if t is None:
                if pivot2:
                    raise ValueError("fixed pivots of Algorithm 2.1 need piv0 and piv1")
                continue
            if t.dtype != torch.int32 or not t.is_contiguous() or t.numel() < need_n:
                raise ValueError("given pivots must be contiguous int32 with >= k + p entries")
    o = opts(q, d, pivot2, prec, block_b, debug_flags, spin_limit_ns, fixed, truncate_k, in_flight)
    L_ = lib()
    need = L_.rqlp_workspace_size(m, n, k, p, ctypes.byref(o))
    if need == 0:
        raise RqlpError(-1, "rqlp_workspace_size")
    dev = A.device
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    w = k if truncate_k else l
    if out is None:
        out = dict(Q=torch.empty((m, w), dtype=torch.float64, device=dev),
                   L=torch.empty((w, w), dtype=torch.float64, device=dev),
                   P=torch.empty((n, w), dtype=torch.float64, device=dev),
                   Lvalues=torch.empty((w,), dtype=torch.float64, device=dev),
                   piv0=torch.empty((n,), dtype=torch.int32, device=dev),
                   piv1=torch.empty((l,), dtype=torch.int32, device=dev))
        if rvalues:
            out["Rvalues"] = torch.empty((w,), dtype=torch.float64, device=dev)
    if fixed:
        out["piv0"], out["piv1"] = piv0, piv1
    st = _stream(stream)
    code = L_.rqlp(_ptr(A), _dtype_code(A), m, n, lda, k, p, _ptr(Omega), ldo, ctypes.byref(o),
                   _ptr(out["Q"]), _ptr(out["L"]), _ptr(out["P"]), _ptr(out["Lvalues"]),
                   _ptr(out["piv0"]), _ptr(out.get("piv1")), _ptr(ws), ws.numel(), st)
    _check(code, "rqlp")
    if out.get("Rvalues") is not None:
        _check(L_.rqlp_rvalues(_ptr(ws), m, n, k, p, ctypes.byref(o), _ptr(out["Rvalues"]), st),
               "rqlp_rvalues")
    res = dict(out)
    res["ws"] = ws
    if check:
        status = L_.rqlp_read_status(_ptr(ws), st)
        _check(status, "rqlp (device status)")
        res["status"] = status
    return res


def brqlp_tol(A, b: int, l_max: int, tol: float, Omega, d: int = 1, pivot2: bool = True,
              prec: str = "fp64", ws=None, stream=None) -> dict:
    """Fixed-accuracy BRQLP: blocks of b columns (Algorithm 4.1) until
    ||A - V V^T A||_F <= tol ||A||_F (eq. 2.1) or l_max columns.  Omega is
    (n, l_max) float64.  Returns Q, L, P, Lvalues, piv1 cut to the l columns
    used, piv0, l and status.  Synchronizes the stream once per block."""
    torch = _torch()
    m, n = A.shape
    lda = _row_major(A, "A")
    ldo = _row_major(Omega, "Omega")
    if Omega.dtype != torch.float64 or tuple(Omega.shape) != (n, l_max):
        raise ValueError("Omega must be float64 of shape (n, l_max)")
    o = opts(0, d, pivot2, prec, b)
    L_ = lib()
    need = L_.rqlp_workspace_size(m, n, l_max, 0, ctypes.byref(o))
    if need == 0:
        raise RqlpError(-1, "rqlp_workspace_size")
    dev = A.device
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    out = dict(Q=torch.empty((m, l_max), dtype=torch.float64, device=dev),
               L=torch.empty((l_max, l_max), dtype=torch.float64, device=dev),
               P=torch.empty((n, l_max), dtype=torch.float64, device=dev),
               Lvalues=torch.zeros((l_max,), dtype=torch.float64, device=dev),
               piv0=torch.empty((n,), dtype=torch.int32, device=dev),
               piv1=torch.empty((l_max,), dtype=torch.int32, device=dev))
    used = ctypes.c_int32(0)
    code = L_.rqlp_brqlp_tol(_ptr(A), _dtype_code(A), m, n, lda, b, l_max, float(tol), _ptr(Omega),
                             ldo, ctypes.byref(o), _ptr(out["Q"]), _ptr(out["L"]), _ptr(out["P"]),
                             _ptr(out["Lvalues"]), _ptr(out["piv0"]), _ptr(out["piv1"]),
                             ctypes.byref(used), _ptr(ws), ws.numel(), _stream(stream))
    _check(code, "rqlp_brqlp_tol")
    l = int(used.value)
    return dict(Q=out["Q"][:, :l], L=out["L"][:l, :l], P=out["P"][:, :l],
                Lvalues=out["Lvalues"][:l], piv0=out["piv0"], piv1=out["piv1"][:l], l=l,
                status=code, ws=ws)


def _host_call(entry: str, A_host, k, p, Omega_host, q, d, pivot2, prec, block_b, ws, out,
               device, stream, in_flight=0) -> dict:
    torch = _torch()
    m, n = A_host.shape
    l = k + p
    if not A_host.is_contiguous() or not Omega_host.is_contiguous():
        raise ValueError("host inputs must be contiguous")
    o = opts(q, d, pivot2, prec, block_b, in_flight=in_flight)
    L_ = lib()
    if stream is None:
        stream = torch.cuda.current_stream()  # the wait must use the same stream
    dt = _dtype_code(A_host)
    need = L_.rqlp_host_workspace_size(m, n, k, p, ctypes.byref(o), dt)
    if need == 0:
        raise RqlpError(-1, "rqlp_host_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    if out is None:
        pin = dict(pin_memory=True)
        out = dict(Q=torch.empty((m, l), dtype=torch.float64, **pin),
                   L=torch.empty((l, l), dtype=torch.float64, **pin),
                   P=torch.empty((n, l), dtype=torch.float64, **pin),
                   Lvalues=torch.empty((l,), dtype=torch.float64, **pin),
                   piv0=torch.empty((n,), dtype=torch.int32, **pin),
                   piv1=torch.empty((l,), dtype=torch.int32, **pin))
    code = getattr(L_, entry)(_ptr(A_host), dt, m, n, k, p, _ptr(Omega_host), ctypes.byref(o),
                              _ptr(out["Q"]), _ptr(out["L"]), _ptr(out["P"]),
                              _ptr(out["Lvalues"]), _ptr(out["piv0"]), _ptr(out["piv1"]),
                              _ptr(ws), ws.numel(), _stream(stream))
    _check(code, entry)
    res = dict(out)
    res["ws"] = ws
    res["status"] = code
    res["stream"] = stream
    return res


def rqlp_host(A_host, k: int, p: int, Omega_host, q: int = 0, d: int = 1, pivot2: bool = True,
              prec: str = "fp64", block_b: int = 0, ws=None, out: Optional[dict] = None,
              device="cuda", stream=None) -> dict:
    """rqlp() on host tensors: copies in, factors, copies out, synchronizes.

    A_host / Omega_host are CPU tensors (pinned for full copy speed); the
    results come back in CPU tensors (pinned when `out` is not given).
    """
    return _host_call("rqlp_host", A_host, k, p, Omega_host, q, d, pivot2, prec, block_b, ws,
                      out, device, stream)


def rqlp_host_async(A_host, k: int, p: int, Omega_host, q: int = 0, d: int = 1,
                    pivot2: bool = True, prec: str = "fp64", block_b: int = 0, ws=None,
                    out: Optional[dict] = None, device="cuda", stream=None,
                    in_flight: int = 0) -> dict:
    """rqlp_host() without the final synchronization: everything is enqueued
    on `stream`.  The host tensors must stay alive and untouched, and the
    results are valid, only after host_wait() on the returned dict.  Calls
    with their own workspaces and streams overlap one problem's copies with
    another's factorization (in_flight: how many such calls run at once)."""
    return _host_call("rqlp_host_async", A_host, k, p, Omega_host, q, d, pivot2, prec, block_b,
                      ws, out, device, stream, in_flight)


def host_wait(res: dict) -> int:
    """Waits for an rqlp_host_async() call; raises on a device error."""
    code = lib().rqlp_read_status(_ptr(res["ws"]), _stream(res.get("stream")))
    _check(code, "rqlp_host_async (device status)")
    res["status"] = code
    return code


def qlp(A, t: int, pivot2: bool = False, ws=None, stream=None, check: bool = True) -> dict:
    """Deterministic pivoted QLP of A truncated at t steps (Section 1, eq. 1.2;
    the comparison method of Section 5) on the GPU.  A: (m, n) float64 CUDA
    tensor.  Returns Q (m, t), L (t, t), P (n, t), Lvalues, piv0, piv1, status."""
    torch = _torch()
    m, n = A.shape
    o = opts(pivot2=pivot2)
    L_ = lib()
    need = L_.rqlp_qlp_workspace_size(m, n, t, ctypes.byref(o))
    if need == 0:
        raise RqlpError(-1, "rqlp_qlp_workspace_size")
    dev = A.device
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    out = dict(Q=torch.empty((m, t), dtype=torch.float64, device=dev),
               L=torch.empty((t, t), dtype=torch.float64, device=dev),
               P=torch.empty((n, t), dtype=torch.float64, device=dev),
               Lvalues=torch.empty((t,), dtype=torch.float64, device=dev),
               piv0=torch.empty((n,), dtype=torch.int32, device=dev),
               piv1=torch.empty((t,), dtype=torch.int32, device=dev))
    st = _stream(stream)
    _check(L_.rqlp_qlp(_ptr(A), _dtype_code(A), m, n, _row_major(A, "A"), t, ctypes.byref(o),
                       _ptr(out["Q"]), _ptr(out["L"]), _ptr(out["P"]), _ptr(out["Lvalues"]),
                       _ptr(out["piv0"]), _ptr(out["piv1"]), _ptr(ws), ws.numel(), st), "rqlp_qlp")
    out["ws"] = ws
    if check:
        out["status"] = _check(L_.rqlp_read_status(_ptr(ws), st), "rqlp_qlp (device status)")
    return out


# ------------------------------------------------------------------ stages
def _stage_ws(rows, cols, l, prec, device, ws=None):
    need = lib().rqlp_stage_workspace_size(rows, cols, l, PREC[prec] if isinstance(prec, str) else prec)
    if need == 0:
        raise RqlpError(-1, "rqlp_stage_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, device)
    return ws


def sketch(A, W, prec="fp64", ws=None, stream=None):
    """Y = A W (Algorithm 2.1, step 2)."""
    torch = _torch()
    m, n = A.shape
    l = W.shape[1]
    ws = _stage_ws(m, n, l, prec, A.device, ws)
    Y = torch.empty((m, l), dtype=torch.float64, device=A.device)
    st = _stream(stream)
    _check(lib().rqlp_sketch(_ptr(A), _dtype_code(A), m, n, _row_major(A, "A"), _ptr(W),
                             _row_major(W, "W"), l, PREC[prec], _ptr(Y), l, _ptr(ws), ws.numel(), st),
           "rqlp_sketch")
    _check(lib().rqlp_read_status(_ptr(ws), st), "rqlp_sketch (device status)")
    return Y


def project(A, V, prec="fp64", ws=None, stream=None):
    """Z = A^T V = (V^T A)^T (Algorithm 2.1, step 4)."""
    torch = _torch()
    m, n = A.shape
    l = V.shape[1]
    ws = _stage_ws(m, n, l, prec, A.device, ws)
    Z = torch.empty((n, l), dtype=torch.float64, device=A.device)
    st = _stream(stream)
    _check(lib().rqlp_project(_ptr(A), _dtype_code(A), m, n, _row_major(A, "A"), _ptr(V),
                              _row_major(V, "V"), l, PREC[prec], _ptr(Z), l, _ptr(ws), ws.numel(),
                              st), "rqlp_project")
    _check(lib().rqlp_read_status(_ptr(ws), st), "rqlp_project (device status)")
    return Z


def orth(X, want_r=True, ws=None, stream=None):
    """Thin QR X = Q R by CholeskyQR2 (Algorithm 2.1, step 3); returns (Q, R, status)."""
    torch = _torch()
    rows, l = X.shape
    ws = _stage_ws(rows, l, l, "fp64", X.device, ws)
    Q = torch.empty((rows, l), dtype=torch.float64, device=X.device)
    R = torch.empty((l, l), dtype=torch.float64, device=X.device) if want_r else None
    st = _stream(stream)
    _check(lib().rqlp_orth(_ptr(X), rows, l, _row_major(X, "X"), _ptr(Q), l, _ptr(R), _ptr(ws),
                           ws.numel(), st), "rqlp_orth")
    status = _check(lib().rqlp_read_status(_ptr(ws), st), "rqlp_orth (device status)")
    return Q, R, status


def cpqr(B, ws=None, stream=None):
    """Column-pivoted QR of the l x n matrix B (Algorithm 2.1, step 5).

    Returns (Q0, R0, piv0) with B[:, piv0] = Q0 @ R0.
    """
    torch = _torch()
    l, n = B.shape
    Bt = B.t().contiguous()
    ws = _stage_ws(l, n, l, "fp64", B.device, ws)
    R0t = torch.empty((n, l), dtype=torch.float64, device=B.device)
    piv = torch.empty((n,), dtype=torch.int32, device=B.device)
    Q0 = torch.empty((l, l), dtype=torch.float64, device=B.device)
    st = _stream(stream)
    _check(lib().rqlp_cpqr(_ptr(Bt), n, l, l, _ptr(R0t), _ptr(piv), _ptr(Q0), _ptr(ws), ws.numel(),
                           st), "rqlp_cpqr")
    _check(lib().rqlp_read_status(_ptr(ws), st), "rqlp_cpqr (device status)")
    return Q0, R0t.t().contiguous(), piv


# ----------------------------------------------------------------- batches
class Batch:
    """Many independent factorizations in one CUDA graph launch.

    As: list of (m_i, n_i) CUDA tensors (float64/float32, row-major); ks: the
    target ranks; p: oversampling; Omegas: list of (n_i, k_i + p) float64
    CUDA tensors.  engine: "persistent" (one persistent kernel taking work
    items from a device list), "graph" (every problem's kernels recorded into
    the graph over `branches` parallel streams) or "auto" (the persistent
    kernel where it supports the batch).  Outputs are allocated here
    (self.out[i] holds Q, L, P, Lvalues, piv0, piv1).  launch() runs the whole
    batch with one cudaGraphLaunch; status() synchronizes and returns (worst,
    per-problem).
    """

    def __init__(self, As, ks, p, Omegas, q=0, d=1, pivot2=True, prec="fp64", branches=0,
                 gemm_target_ctas=0, mma_max_splits=0, engine="auto"):
        torch = _torch()
        L_ = lib()
        self.count = len(As)
        self._keep = [As, Omegas]
        self.out = []
        probs = (Problem * self.count)()
        for i, (A, k, Om) in enumerate(zip(As, ks, Omegas)):
            m, n = A.shape
            l = k + p
            dev = A.device
            o = dict(Q=torch.empty((m, l), dtype=torch.float64, device=dev),
                     L=torch.empty((l, l), dtype=torch.float64, device=dev),
                     P=torch.empty((n, l), dtype=torch.float64, device=dev),
                     Lvalues=torch.empty((l,), dtype=torch.float64, device=dev),
                     piv0=torch.empty((n,), dtype=torch.int32, device=dev),
                     piv1=torch.empty((l,), dtype=torch.int32, device=dev))
            self.out.append(o)
            probs[i] = Problem(_ptr(A), _dtype_code(A), int(k), m, n, _row_major(A, "A"), int(p), 0,
                               _ptr(Om), _row_major(Om, "Omega"), _ptr(o["Q"]), _ptr(o["L"]),
                               _ptr(o["P"]), _ptr(o["Lvalues"]), _ptr(o["piv0"]), _ptr(o["piv1"]))
        self._probs = probs
        self.opts = opts(q, d, pivot2, prec)
        self.tuning = BatchTuning(int(branches), int(gemm_target_ctas), int(mma_max_splits),
                                  ENGINES[engine])
        need = L_.rqlp_batched_workspace_size(probs, self.count, ctypes.byref(self.opts),
                                              ctypes.byref(self.tuning))
        if need == 0:
            raise RqlpError(-1, "rqlp_batched_workspace_size")
        self.ws = workspace(need, As[0].device)
        handle = _c_p()
        _check(L_.rqlp_batched_create(probs, self.count, ctypes.byref(self.opts),
                                      ctypes.byref(self.tuning), _ptr(self.ws), self.ws.numel(),
                                      ctypes.byref(handle)), "rqlp_batched_create")
        self.handle = handle

    @property
    def kernel_nodes(self) -> int:
        return int(lib().rqlp_batched_kernel_nodes(self.handle))

    @property
    def engine(self) -> str:
        code = int(lib().rqlp_batched_engine(self.handle, None))
        return {1: "graph", 2: "persistent"}.get(code, "unknown")

    STAGE_KINDS = {1: "prep_A", 2: "split_omega", 3: "products_with_A", 4: "gram", 5: "cholesky",
                   6: "solve", 7: "cpqr_of_B", 8: "qlp_l_by_l", 9: "assembly", 10: "status"}

    def stage_times(self, stream=None) -> dict:
        """Persistent engine: per stage kind of the last launch, the CTA time
        spent running items (busy_us) and taking them (wait_us: the queue and
        the previous stage), summed over CTAs, and the items that ran."""
        busy, wait, items = (ctypes.c_double * 16)(), (ctypes.c_double * 16)(), (_c_i64 * 16)()
        _check(lib().rqlp_batched_stage_times(self.handle, _stream(stream), ctypes.cast(busy, _c_p),
                                              ctypes.cast(wait, _c_p), ctypes.cast(items, _c_p)),
               "rqlp_batched_stage_times")
        return {name: {"busy_us": busy[k], "wait_us": wait[k], "items": int(items[k])}
                for k, name in self.STAGE_KINDS.items()}

    @property
    def work_items(self) -> int:
        n = _c_i64(0)
        lib().rqlp_batched_engine(self.handle, ctypes.byref(n))
        return int(n.value)

    def launch(self, stream=None):
        _check(lib().rqlp_batched_launch(self.handle, _stream(stream)), "rqlp_batched_launch")

    def status(self, stream=None):
        arr = (_c_i32 * self.count)()
        worst = lib().rqlp_batched_status(self.handle, _stream(stream), ctypes.cast(arr, _c_p))
        return worst, list(arr)

    def close(self):
        if getattr(self, "handle", None):
            lib().rqlp_batched_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """One factorization recorded into a CUDA graph and replayed
    (rqlp_graph_create / launch / destroy).

    Arguments as for rqlp() (no fixed pivots, no R-values).  The constructor
    factors A once on `stream` and records the call; launch() replays it on
    any stream with one graph launch.  The graph reads A and Omega and writes
    self.out and self.ws at their current addresses: copy new data into A
    (in place) and launch again.  status() reads the device status word.
    """

    def __init__(self, A, k: int, p: int, Omega, q: int = 0, d: int = 1, pivot2: bool = True,
                 prec: str = "fp64", block_b: int = 0, stream=None, in_flight: int = 0,
                 truncate_k: bool = False):
        torch = _torch()
        m, n = A.shape
        l = k + p
        lda = _row_major(A, "A")
        ldo = _row_major(Omega, "Omega")
        if Omega.dtype != torch.float64 or tuple(Omega.shape) != (n, l):
            raise ValueError("Omega must be float64 of shape (n, k + p)")
        self.opts = opts(q, d, pivot2, prec, block_b, truncate_k=truncate_k, in_flight=in_flight)
        L_ = lib()
        need = L_.rqlp_workspace_size(m, n, k, p, ctypes.byref(self.opts))
        if need == 0:
            raise RqlpError(-1, "rqlp_workspace_size")
        dev = A.device
        self.ws = workspace(need, dev)
        w = k if truncate_k else l
        self.out = dict(Q=torch.empty((m, w), dtype=torch.float64, device=dev),
                        L=torch.empty((w, w), dtype=torch.float64, device=dev),
                        P=torch.empty((n, w), dtype=torch.float64, device=dev),
                        Lvalues=torch.empty((w,), dtype=torch.float64, device=dev),
                        piv0=torch.empty((n,), dtype=torch.int32, device=dev),
                        piv1=torch.empty((l,), dtype=torch.int32, device=dev))
        self._keep = (A, Omega)
        o = self.out
        handle = _c_p()
        _check(L_.rqlp_graph_create(_ptr(A), _dtype_code(A), m, n, lda, k, p, _ptr(Omega), ldo,
                                    ctypes.byref(self.opts), _ptr(o["Q"]), _ptr(o["L"]),
                                    _ptr(o["P"]), _ptr(o["Lvalues"]), _ptr(o["piv0"]),
                                    _ptr(o["piv1"]), _ptr(self.ws), self.ws.numel(),
                                    _stream(stream), ctypes.byref(handle)), "rqlp_graph_create")
        self.handle = handle

    @property
    def kernels(self) -> int:
        return int(lib().rqlp_graph_kernels(self.handle))

    def launch(self, stream=None):
        _check(lib().rqlp_graph_launch(self.handle, _stream(stream)), "rqlp_graph_launch")

    def status(self, stream=None) -> int:
        return read_status(self.ws, stream)

    def close(self):
        if getattr(self, "handle", None):
            lib().rqlp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- adjoint
def vjp(A, k, p, Omega, dQ=None, dL=None, dP=None, q=0, prec="fp64", ws=None, stream=None,
        piv0=None, piv1=None):
    """dA = J^T (dQ, dL, dP) of A -> (Q, L, P) for RQLP (Algorithm 2.1) with
    fixed pivots, computed on the GPU (FP64 sweep, forward recomputed).  piv0
    / piv1 (int32 CUDA tensors, >= k + p entries each): the forward call's
    pivots, held fixed; None recomputes them from A."""
    torch = _torch()
    m, n = A.shape
    o = opts(q, 1, True, prec)
    L_ = lib()
    need = L_.rqlp_backward_workspace_size(m, n, k, p, ctypes.byref(o))
    if need == 0:
        raise RqlpError(-1, "rqlp_backward_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    dA = torch.empty((m, n), dtype=torch.float64, device=A.device)
    cont = lambda t: None if t is None else t.detach().to(torch.float64).contiguous()
    dQ, dL, dP = cont(dQ), cont(dL), cont(dP)
    if (piv0 is None) != (piv1 is None):
        raise ValueError("give both pivot arrays or neither")
    if piv0 is not None:
        piv0 = piv0.to(torch.int32).contiguous()
        piv1 = piv1.to(torch.int32).contiguous()
        if piv0.numel() < k + p or piv1.numel() < k + p:
            raise ValueError("pivot arrays need >= k + p entries")
    st = _stream(stream)
    _check(L_.rqlp_backward(_ptr(A), _dtype_code(A), m, n, _row_major(A, "A"), k, p, _ptr(Omega),
                            _row_major(Omega, "Omega"), ctypes.byref(o), _ptr(piv0), _ptr(piv1),
                            _ptr(dQ), _ptr(dL), _ptr(dP), _ptr(dA), n, _ptr(ws), ws.numel(), st),
           "rqlp_backward")
    _check(L_.rqlp_read_status(_ptr(ws), st), "rqlp_backward (device status)")
    return dA


def _autograd_function():
    torch = _torch()

    class RQLPFunction(torch.autograd.Function):
        """(Q, L, P) = RQLP(A) on the GPU with a hand-written adjoint (pivots fixed)."""

        @staticmethod
        def forward(ctx, A, Omega, k, p, q, prec):
            out = rqlp(A.detach(), k, p, Omega, q=q, pivot2=True, prec=prec, rvalues=False)
            # the backward sweep recomputes the forward at these pivots, so the
            # derivative belongs to the factorization returned here
            ctx.save_for_backward(A, Omega, out["piv0"], out["piv1"])
            ctx.cfg = (k, p, q, prec)
            return out["Q"], out["L"], out["P"]

        @staticmethod
        def backward(ctx, dQ, dL, dP):
            A, Omega, piv0, piv1 = ctx.saved_tensors
            k, p, q, prec = ctx.cfg
            dA = vjp(A.detach(), k, p, Omega, dQ, dL, dP, q=q, prec=prec, piv0=piv0, piv1=piv1)
            return dA.to(A.dtype), None, None, None, None, None

    return RQLPFunction


_RQLPFunction = None


def rqlp_autograd(A, k, p, Omega, q=0, prec="fp64"):
    """Differentiable (Q, L, P) = RQLP(A) (torch.autograd, pivots held fixed)."""
    global _RQLPFunction
    if _RQLPFunction is None:
        _RQLPFunction = _autograd_function()
    return _RQLPFunction.apply(A, Omega, k, p, q, prec)
