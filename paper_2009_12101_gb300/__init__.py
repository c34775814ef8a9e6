"""GB300 compressed-basis GMRES (CB-GMRES, arXiv 2009.12101) -- thin Python binding.

Every step of the solver runs in the CUDA library ``_lib/libcbgmres.so`` (C ABI in
``include/cbgmres.h``).  This module only marshals arguments: it hands device pointers
of torch tensors and the current CUDA stream to the library.  There is no CPU
fallback: if the library is missing or no GPU is visible the calls raise.

    import paper_2009_12101_gb300 as cb
    s = cb.Solver(rowptr, col, val, restart=100, fmt="f32")
    stats = s.solve(b, x, tol=1e-10, maxit=20000)    # b, x: CUDA float64 tensors
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB as _LIB_RELEASE
from .build import LIB_DEBUG as _LIB_DEBUG
from .build import build as _build

# CBG_DEBUG=1 in the environment selects the debug library (guard tails on the solver's
# device allocations checked after every solve, column-index checks in the SpMV)
DEBUG = os.environ.get("CBG_DEBUG", "0") == "1"
_LIB_PATH = _LIB_DEBUG if DEBUG else _LIB_RELEASE

FORMATS = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "e4m3": 4, "i32": 5, "i16": 6}
FORMAT_NAMES = {v: k for k, v in FORMATS.items()}
FORMAT_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "e4m3": 1, "i32": 4, "i16": 2}
PRECONDS = {"none": 0, "jacobi": 1, "spai": 2, "bj4": 3}
REORTH = {"always": 0, "conditional": 1, "never": 2}
ARITH = {"df32": 0, "fp64": 1}
ORTHO = {"cgs": 0, "mgs": 1}
STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "STAGNATED", -1: "ERR_ARG", -2: "ERR_NONFINITE", -3: "ERR_OOM",
          -4: "ERR_CUDA", -5: "ERR_TIMEOUT", -6: "ERR_UNSUPPORTED"}
TILE_ROWS = 4096   # padded rows per basis column (multiple of every kernel tile)


class CbgError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: status {status} ({STATUS.get(status, '?')})"
        if status == -4 and _lib is not None:
            msg += f": {_lib.cbgmres_last_error().decode()}"
        super().__init__(msg)
        self.status = status


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32), ("pad0", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("reorth", C.c_int32), ("precond", C.c_int32), ("arith", C.c_int32),
                ("spmv_group", C.c_int32), ("eta", C.c_double), ("breakdown_eps", C.c_double),
                ("stream", C.c_void_p), ("check_every", C.c_int32), ("use_graph", C.c_int32),
                ("profile", C.c_int32), ("stop_on_stagnation", C.c_int32), ("adapt", C.c_int32),
                ("pad1", C.c_int32), ("adapt_gap", C.c_double), ("ortho", C.c_int32), ("pad2", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("reorths", C.c_int64),
                ("true_relres", C.c_double), ("est_relres", C.c_double), ("ms_total", C.c_double),
                ("bytes_model", C.c_double), ("status", C.c_int32), ("fmt_final", C.c_int32),
                ("history", C.c_void_p), ("history_cap", C.c_int64), ("history_len", C.c_int64),
                ("kernel_launches", C.c_int64), ("promotions", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 5), ("bytes", C.c_double * 5), ("launches", C.c_int64 * 5)]


PROFILE_CLASSES = ("basis_dot", "basis_axpy", "spmv", "store", "other")


_lib = None
_lock = threading.Lock()


def ensure_built() -> str:
    """Compile libcbgmres.so (libcbgmres_debug.so when CBG_DEBUG=1) for sm_103a if it is
    missing or older than its sources."""
    return _build(debug=DEBUG)


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libcbgmres.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"{_LIB_PATH} is missing: build it with "
                                  "paper_2009_12101_gb300.ensure_built() (needs nvcc)")
            L = C.CDLL(_LIB_PATH)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.cbgmres_options_default.argtypes = [C.POINTER(Options)]
            L.cbgmres_options_default.restype = None
            L.cbgmres_status_string.argtypes = [i32]
            L.cbgmres_status_string.restype = C.c_char_p
            L.cbgmres_format_bytes.argtypes = [i32]
            L.cbgmres_last_error.argtypes = []
            L.cbgmres_last_error.restype = C.c_char_p
            L.cbgmres_create.argtypes = [C.POINTER(Csr), i32, i32, C.POINTER(Options), C.POINTER(vp)]
            L.cbgmres_set_spai.argtypes = [vp, vp, i32]
            L.cbgmres_solve.argtypes = [vp, vp, vp, d, i64, C.POINTER(Stats)]
            L.cbgmres_solve_host.argtypes = [vp, vp, vp, d, i64, C.POINTER(Stats)]
            L.cbgmres_arnoldi.argtypes = [vp, vp, vp, i32, vp, C.POINTER(C.c_int)]
            L.cbgmres_basis_column.argtypes = [vp, i32, vp]
            L.cbgmres_spmv.argtypes = [vp, vp, vp]
            L.cbgmres_profile.argtypes = [vp, C.POINTER(Profile), i32]
            L.cbgmres_test_stall.argtypes = [vp, i32, C.c_int64]
            L.cbgmres_spmv_group.argtypes = [vp]
            L.cbgmres_debug_guard_check.argtypes = [vp, i32]
            L.cbgmres_destroy.argtypes = [vp]
            L.cbgmres_destroy.restype = None
            L.cbg_encode.argtypes = [i32, i64, vp, d, vp, C.POINTER(d), vp]
            L.cbg_decode.argtypes = [i32, i64, vp, d, vp, vp]
            L.cbg_basis_dot.argtypes = [i32, i32, i64, i32, vp, i64, vp, vp, vp, vp]
            L.cbg_basis_axpy.argtypes = [i32, i32, i64, i32, vp, i64, vp, vp, vp, vp]
            L.cbg_basis_dot_noalloc.argtypes = [i32, i32, i64, i32, vp, i64, vp, vp, vp, vp]
            L.cbg_basis_dot_multi_workspace.argtypes = [i64, i32, i32]
            L.cbg_basis_dot_multi_workspace.restype = C.c_size_t
            L.cbg_basis_dot_multi.argtypes = [i32, i64, i32, vp, i64, vp, i32, vp, i64, vp, vp, C.c_size_t, vp]
            L.cbg_basis_dot_multi_path.argtypes = [i32, i64, i32, vp, i64, vp, i32, vp, i64, vp, vp, C.c_size_t,
                                                   vp, i32]
            L.cbgmres_create_batched.argtypes = [i32, vp, i32, i32, C.POINTER(Options), C.POINTER(vp)]
            L.cbgmres_solve_batched.argtypes = [vp, vp, vp, d, i64, vp]
            L.cbgmres_tune_batched.argtypes = [vp, vp, vp, d, i64, C.c_char_p, C.POINTER(C.c_int),
                                               C.POINTER(C.c_int)]
            L.cbgmres_batched_schedule.argtypes = [vp, i32, i32]
            L.cbgmres_batched_spmv_lanes.argtypes = [vp, i32]
            L.cbgmres_solve_fallback.argtypes = [vp, i32, vp, vp, d, i64, C.POINTER(Stats), C.POINTER(C.c_int)]
            L.cbg_spai_create.argtypes = [C.POINTER(Csr), i64, i64, C.POINTER(Options), C.POINTER(vp)]
            L.cbg_spai_add_pair.argtypes = [vp, vp, vp]
            L.cbg_spai_train.argtypes = [vp, i32, d, C.POINTER(d), C.POINTER(d)]
            L.cbg_spai_loss.argtypes = [vp, C.POINTER(d)]
            L.cbg_spai_values.argtypes = [vp, vp]
            L.cbg_spai_params.argtypes = [vp, vp, i32]
            L.cbg_spai_num_params.argtypes = []
            L.cbg_spai_destroy.argtypes = [vp]
            L.cbg_spai_destroy.restype = None
            L.cbg_mlp_forward.argtypes = [i64, vp, vp, vp, vp]
            L.cbg_mlp_backward.argtypes = [i64, vp, vp, vp, vp, vp]
            L.cbgmres_destroy_batched.argtypes = [vp]
            L.cbgmres_destroy_batched.restype = None
            _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CB-GMRES needs a CUDA GPU (no device visible)")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(rc: int, where: str):
    if rc < 0:
        raise CbgError(rc, where)
    return rc


def _dev_f64(t, n=None, name="vector"):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return C.c_void_p(t.data_ptr())


def options(precond="none", arith="df32", reorth="always", spmv_group=0, stream=None,
            check_every=4, eta=None, breakdown_eps=None, profile=False,
            stop_on_stagnation=False, adapt=False, adapt_gap=None, ortho="cgs") -> Options:
    o = Options()
    lib().cbgmres_options_default(C.byref(o))
    o.precond = PRECONDS[precond]
    o.arith = ARITH[arith]
    o.reorth = REORTH[reorth]
    o.ortho = ORTHO[ortho]
    o.spmv_group = spmv_group
    o.check_every = check_every
    o.profile = int(bool(profile))
    o.stop_on_stagnation = int(bool(stop_on_stagnation))
    o.adapt = int(bool(adapt))
    if adapt_gap is not None:
        o.adapt_gap = adapt_gap
    if eta is not None:
        o.eta = eta
    if breakdown_eps is not None:
        o.breakdown_eps = breakdown_eps
    o.stream = _stream_ptr(stream).value
    return o


def _stats_dict(st: Stats, hist=None) -> dict:
    out = {k: getattr(st, k) for k in ("iters", "restarts", "reorths", "true_relres", "est_relres",
                                       "ms_total", "bytes_model", "status", "kernel_launches", "promotions")}
    out["fmt_final"] = FORMAT_NAMES.get(st.fmt_final, st.fmt_final)
    if hist is not None:
        out["history"] = hist[: st.history_len].copy()
    return out


class Solver:
    """Handle on libcbgmres for one matrix, restart length and basis format.

    rowptr/col/val: CSR arrays (int32, int32, float64) as numpy arrays (copied from
    host) or CUDA tensors (copied device to device)."""

    def __init__(self, rowptr, col, val, *, restart: int = 100, fmt: str = "f64",
                 precond: str = "none", arith: str = "df32", reorth: str = "always",
                 spmv_group: int = 0, stream=None, check_every: int = 4, profile: bool = False,
                 stop_on_stagnation: bool = False, adapt: bool = False, adapt_gap: float | None = None,
                 ortho: str = "cgs", eta: float | None = None):
        torch = _torch()
        L = lib()
        self.fmt, self.restart, self.precond, self.arith = fmt, restart, precond, arith
        self.stream = stream
        keep = []
        if isinstance(rowptr, torch.Tensor):
            rp = rowptr.to(torch.int32).contiguous(); ci = col.to(torch.int32).contiguous()
            va = val.to(torch.float64).contiguous(); keep += [rp, ci, va]
            csr = Csr(rp.numel() - 1, ci.numel(), rp.data_ptr(), ci.data_ptr(), va.data_ptr(), 1, 0)
        else:
            rp = np.ascontiguousarray(rowptr, np.int32); ci = np.ascontiguousarray(col, np.int32)
            va = np.ascontiguousarray(val, np.float64); keep += [rp, ci, va]
            csr = Csr(rp.size - 1, ci.size, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, 0)
        self.n, self.nnz = int(csr.n), int(csr.nnz)
        self.ld = (self.n + TILE_ROWS - 1) // TILE_ROWS * TILE_ROWS
        opt = options(precond=precond, arith=arith, reorth=reorth, spmv_group=spmv_group,
                      stream=stream, check_every=check_every, profile=profile,
                      stop_on_stagnation=stop_on_stagnation, adapt=adapt, adapt_gap=adapt_gap,
                      ortho=ortho, eta=eta)
        h = C.c_void_p()
        _check(L.cbgmres_create(C.byref(csr), restart, FORMATS[fmt], C.byref(opt), C.byref(h)),
               "cbgmres_create")
        self._h = h

    @classmethod
    def from_csr(cls, A, **kw):
        """A: any object with rowptr, col, val arrays (e.g. workloads.CSR)."""
        return cls(A.rowptr, A.col, A.val, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().cbgmres_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_spai(self, pvals):
        torch = _torch()
        if isinstance(pvals, torch.Tensor):
            p = pvals.to(torch.float64).contiguous()
            _check(lib().cbgmres_set_spai(self._h, C.c_void_p(p.data_ptr()), 1), "cbgmres_set_spai")
        else:
            p = np.ascontiguousarray(pvals, np.float64)
            _check(lib().cbgmres_set_spai(self._h, C.c_void_p(p.ctypes.data), 0), "cbgmres_set_spai")

    def solve(self, b, x, tol: float = 1e-10, maxit: int = 100000, history: int = 0) -> dict:
        """b, x: CUDA float64 tensors (x: initial guess in, solution out)."""
        st = Stats()
        hist = None
        if history:
            hist = np.zeros(history); st.history = hist.ctypes.data; st.history_cap = history
        rc = lib().cbgmres_solve(self._h, _dev_f64(b, self.n, "b"), _dev_f64(x, self.n, "x"),
                                 tol, maxit, C.byref(st))
        _check(rc, "cbgmres_solve")
        return _stats_dict(st, hist)

    def solve_host(self, b: np.ndarray, x: np.ndarray, tol: float = 1e-10, maxit: int = 100000) -> dict:
        """b, x: host float64 arrays; host<->device copies happen inside the call."""
        b = np.ascontiguousarray(b, np.float64)
        if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise TypeError("x must be a contiguous float64 numpy array")
        st = Stats()
        rc = lib().cbgmres_solve_host(self._h, C.c_void_p(b.ctypes.data), C.c_void_p(x.ctypes.data),
                                      tol, maxit, C.byref(st))
        _check(rc, "cbgmres_solve_host")
        return _stats_dict(st)

    def arnoldi(self, b, x0, k: int) -> np.ndarray:
        """Raw (k+1) x k Hessenberg of the first k Arnoldi steps from x0."""
        H = np.zeros((k, k + 1))
        kd = C.c_int()
        _check(lib().cbgmres_arnoldi(self._h, _dev_f64(b, self.n, "b"), _dev_f64(x0, self.n, "x0"),
                                     k, C.c_void_p(H.ctypes.data), C.byref(kd)), "cbgmres_arnoldi")
        kd = kd.value
        flat = H.ravel()[: (kd + 1) * kd]
        return flat.reshape(kd, kd + 1).T.copy()

    def basis_column(self, col: int):
        torch = _torch()
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib().cbgmres_basis_column(self._h, col, C.c_void_p(out.data_ptr())),
               "cbgmres_basis_column")
        return out

    def profile(self, reset: bool = False) -> dict:
        """Per-kernel-class CUDA-event timings (needs profile=True at construction)."""
        p = Profile()
        _check(lib().cbgmres_profile(self._h, C.byref(p), int(reset)), "cbgmres_profile")
        return {c: {"ms": p.ms[i], "bytes": p.bytes[i], "launches": p.launches[i]}
                for i, c in enumerate(PROFILE_CLASSES)}

    def debug_guard_check(self, poke: bool = False) -> int:
        """Debug library: status of the guard tails of every live allocation (poke: first
        overwrite one guard byte of this handle's basis, as a test); CBG_ERR_UNSUPPORTED
        (-6) from the release library."""
        return int(lib().cbgmres_debug_guard_check(self._h, int(bool(poke))))

    def spmv_group(self) -> int:
        """Lanes per CSR row of this handle's SpMV (tuned at create on large matrices)."""
        return _check(lib().cbgmres_spmv_group(self._h), "cbgmres_spmv_group")

    def test_stall(self, dots: int = 1, wait_cycles: int = 2_000_000):
        """Failure-path test: the next `dots` pipelined dot launches withhold their first
        bulk-copy stage and give up their waits after `wait_cycles` clock cycles."""
        _check(lib().cbgmres_test_stall(self._h, int(dots), int(wait_cycles)), "cbgmres_test_stall")

    def spmv(self, x):
        torch = _torch()
        y = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib().cbgmres_spmv(self._h, _dev_f64(x, self.n, "x"), C.c_void_p(y.data_ptr())),
               "cbgmres_spmv")
        return y


# ------------------------------------------------------------------ codec / kernel access
CODE_TORCH = {"f64": "float64", "f32": "float32", "f16": "int16", "bf16": "int16", "e4m3": "uint8",
              "i32": "int32", "i16": "int16"}


def encode(fmt: str, v, vmax: float, stream=None):
    """Encode a normalised CUDA float64 vector; returns (codes tensor, scale)."""
    torch = _torch()
    codes = torch.empty(v.numel(), dtype=getattr(torch, CODE_TORCH[fmt]), device=v.device)
    scale = C.c_double()
    _check(lib().cbg_encode(FORMATS[fmt], v.numel(), _dev_f64(v), vmax, C.c_void_p(codes.data_ptr()),
                            C.byref(scale), _stream_ptr(stream)), "cbg_encode")
    return codes, scale.value


def decode(fmt: str, codes, scale: float, stream=None):
    torch = _torch()
    out = torch.empty(codes.numel(), dtype=torch.float64, device=codes.device)
    _check(lib().cbg_decode(FORMATS[fmt], codes.numel(), C.c_void_p(codes.data_ptr()), scale,
                            C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "cbg_decode")
    return out


def basis_dot(fmt: str, arith: str, n: int, V, ld: int, scales, w, stream=None) -> np.ndarray:
    """h = V^T w for a code matrix V (CUDA tensor, ncols x ld codes)."""
    ncols = V.shape[0]
    h = np.zeros(ncols)
    sc = np.ascontiguousarray(scales, np.float64)
    _check(lib().cbg_basis_dot(FORMATS[fmt], ARITH[arith], n, ncols, C.c_void_p(V.data_ptr()), ld,
                               C.c_void_p(sc.ctypes.data), _dev_f64(w), C.c_void_p(h.ctypes.data),
                               _stream_ptr(stream)), "cbg_basis_dot")
    return h


def basis_dot_noalloc(fmt: str, arith: str, n: int, V, ld: int, scales, w, stream=None) -> np.ndarray:
    """h = V^T w like basis_dot, through the entry point that allocates no device memory
    (its scratch is a static device array shared by all calls; see cbgmres.h)."""
    ncols = V.shape[0]
    h = np.zeros(ncols)
    sc = np.ascontiguousarray(scales, np.float64)
    _check(lib().cbg_basis_dot_noalloc(FORMATS[fmt], ARITH[arith], n, ncols, C.c_void_p(V.data_ptr()), ld,
                                       C.c_void_p(sc.ctypes.data), _dev_f64(w), C.c_void_p(h.ctypes.data),
                                       _stream_ptr(stream)), "cbg_basis_dot_noalloc")
    return h


def basis_dot_multi(fmt: str, n: int, V, ld: int, scales, W, stream=None, workspace=None, path: str = "auto",
                    out=None):
    """H = V^T W for k <= 64 vectors; V: code matrix (ncols x ld codes); W: CUDA float64
    tensor (k, ldw) whose row r holds vector r.  scales: host array or CUDA float64 tensor
    of the ncols decode factors.  Returns H (CUDA tensor, ncols x k; `out` if given)."""
    torch = _torch()
    ncols = V.shape[0]
    k, ldw = int(W.shape[0]), int(W.shape[1])
    if torch.is_tensor(scales) and scales.is_cuda and scales.dtype == torch.float64 and scales.is_contiguous():
        sc = scales
    else:
        sc = torch.as_tensor(np.ascontiguousarray(scales, np.float64)).cuda()
    if out is not None and (out.shape != (ncols, k) or out.dtype != torch.float64 or not out.is_cuda
                            or not out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA float64 tensor of shape (ncols, k)")
    H = torch.empty(ncols, k, dtype=torch.float64, device=W.device) if out is None else out
    ws_bytes = lib().cbg_basis_dot_multi_workspace(ld, ncols, k)
    if ws_bytes == 0:
        raise CbgError(-1, "cbg_basis_dot_multi_workspace")
    if workspace is None or workspace.numel() < ws_bytes:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=W.device)
    _check(lib().cbg_basis_dot_multi_path(FORMATS[fmt], n, ncols, C.c_void_p(V.data_ptr()), ld,
                                          C.c_void_p(sc.data_ptr()), k, C.c_void_p(W.data_ptr()), ldw,
                                          C.c_void_p(H.data_ptr()), C.c_void_p(workspace.data_ptr()),
                                          workspace.numel(), _stream_ptr(stream),
                                          {"auto": 0, "cuda": 1, "tensor": 2}[path]), "cbg_basis_dot_multi")
    return H


def basis_axpy(fmt: str, arith: str, n: int, V, ld: int, scales, h, w, stream=None):
    """w -= V h in place (w: CUDA float64 tensor of ld elements)."""
    ncols = V.shape[0]
    sc = np.ascontiguousarray(scales, np.float64)
    hh = np.ascontiguousarray(h, np.float64)
    _check(lib().cbg_basis_axpy(FORMATS[fmt], ARITH[arith], n, ncols, C.c_void_p(V.data_ptr()), ld,
                                C.c_void_p(sc.ctypes.data), C.c_void_p(hh.ctypes.data), _dev_f64(w),
                                _stream_ptr(stream)), "cbg_basis_axpy")
    return w


class BatchedSolver:
    """Many independent systems solved by one persistent cluster launch.

    mats: list of objects with rowptr/col/val (host numpy) -- e.g. workloads.CSR.
    Vectors are packed in the order of `mats` (offsets = prefix sums of the sizes)."""

    def __init__(self, mats, *, restart: int = 30, fmt: str = "f32", precond: str = "jacobi",
                 use_graph: bool = True, stream=None):
        _torch()
        self.mats = mats
        self.sizes = np.array([int(len(A.rowptr) - 1) for A in mats])
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        self.total = int(self.offsets[-1])
        self._keep = []
        arr = (Csr * len(mats))()
        for i, A in enumerate(mats):
            rp = np.ascontiguousarray(A.rowptr, np.int32); ci = np.ascontiguousarray(A.col, np.int32)
            va = np.ascontiguousarray(A.val, np.float64)
            self._keep += [rp, ci, va]
            arr[i] = Csr(rp.size - 1, ci.size, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, 0)
        opt = options(precond=precond, stream=stream)
        opt.use_graph = int(use_graph)
        h = C.c_void_p()
        _check(lib().cbgmres_create_batched(len(mats), C.cast(arr, C.c_void_p), restart, FORMATS[fmt],
                                            C.byref(opt), C.byref(h)), "cbgmres_create_batched")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().cbgmres_destroy_batched(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, b, x, tol: float = 1e-8, maxit: int = 100000) -> dict:
        st = (Stats * len(self.mats))()
        rc = lib().cbgmres_solve_batched(self._h, _dev_f64(b, self.total, "b"), _dev_f64(x, self.total, "x"),
                                         tol, maxit, C.cast(st, C.c_void_p))
        _check(rc, "cbgmres_solve_batched")
        return {"status": rc, "ms": st[0].ms_total,
                "iters": np.array([s.iters for s in st]), "restarts": np.array([s.restarts for s in st]),
                "relres": np.array([s.true_relres for s in st]), "statuses": np.array([s.status for s in st]),
                "kernel_launches": st[0].kernel_launches}

    def tune(self, b, x, tol: float = 1e-8, maxit: int = 100000, cache_path: str | None = None):
        c = C.c_int(); sr = C.c_int()
        _check(lib().cbgmres_tune_batched(self._h, _dev_f64(b, self.total, "b"), _dev_f64(x, self.total, "x"),
                                          tol, maxit, cache_path.encode() if cache_path else None,
                                          C.byref(c), C.byref(sr)), "cbgmres_tune_batched")
        return c.value, sr.value

    def schedule(self, cluster: int, split_rows: int):
        _check(lib().cbgmres_batched_schedule(self._h, cluster, split_rows), "cbgmres_batched_schedule")

    def spmv_lanes(self, lanes: int = 0) -> int:
        """SpMV lanes per row (1, 2, 4, 8); 0 only queries."""
        return _check(lib().cbgmres_batched_spmv_lanes(self._h, int(lanes)), "cbgmres_batched_spmv_lanes")


def solve_fallback(solvers, b, x, tol: float = 1e-10, maxit: int = 100000):
    """Try the solvers in order (same matrix), each from the current x; the FP64 explicit
    residual decides.  Returns (stats, index of the solver that finished)."""
    arr = (C.c_void_p * len(solvers))(*[s._h.value if s is not None else None for s in solvers])
    st = Stats()
    used = C.c_int()
    n = next(s for s in solvers if s is not None).n
    rc = lib().cbgmres_solve_fallback(C.cast(arr, C.c_void_p), len(solvers), _dev_f64(b, n, "b"),
                                      _dev_f64(x, n, "x"), tol, maxit, C.byref(st), C.byref(used))
    _check(rc, "cbgmres_solve_fallback")
    return _stats_dict(st), used.value


# ------------------------------------------------------------- learned SPAI preconditioner
MLP_NPARAM = 5127


class LearnedSpai:
    """Per-row MLP emitting a sparse approximate inverse on A's 7-point pattern, trained on
    (r, e) pairs from FP64 GMRES iterates (see cbgmres.h for the definition)."""

    def __init__(self, A, sx: int, sxy: int, stream=None):
        _torch()
        rp = np.ascontiguousarray(A.rowptr, np.int32); ci = np.ascontiguousarray(A.col, np.int32)
        va = np.ascontiguousarray(A.val, np.float64)
        self._keep = (rp, ci, va)
        csr = Csr(rp.size - 1, ci.size, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, 0)
        self.n, self.nnz = int(csr.n), int(csr.nnz)
        opt = options(stream=stream)
        h = C.c_void_p()
        _check(lib().cbg_spai_create(C.byref(csr), sx, sxy, C.byref(opt), C.byref(h)), "cbg_spai_create")
        self._h = h
        self.npairs = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().cbg_spai_destroy(self._h)
            self._h = None

    __del__ = close

    def add_pair(self, xstar, xk):
        _check(lib().cbg_spai_add_pair(self._h, _dev_f64(xstar, self.n), _dev_f64(xk, self.n)), "cbg_spai_add_pair")
        self.npairs += 1

    def loss(self) -> float:
        v = C.c_double()
        _check(lib().cbg_spai_loss(self._h, C.byref(v)), "cbg_spai_loss")
        return v.value

    def train(self, steps: int = 200, lr: float = 1e-3):
        a, b = C.c_double(), C.c_double()
        _check(lib().cbg_spai_train(self._h, steps, lr, C.byref(a), C.byref(b)), "cbg_spai_train")
        return a.value, b.value

    def values(self):
        torch = _torch()
        p = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        _check(lib().cbg_spai_values(self._h, C.c_void_p(p.data_ptr())), "cbg_spai_values")
        return p

    def params(self) -> np.ndarray:
        w = np.zeros(MLP_NPARAM, np.float32)
        _check(lib().cbg_spai_params(self._h, C.c_void_p(w.ctypes.data), 0), "cbg_spai_params")
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, np.float32)
        _check(lib().cbg_spai_params(self._h, C.c_void_p(w.ctypes.data), 1), "cbg_spai_params")

    def save(self, path: str):
        """Checkpoint: the FP32 master weights as a flat little-endian binary file."""
        self.params().astype("<f4").tofile(path)

    def load(self, path: str):
        self.set_params(np.fromfile(path, dtype="<f4"))


def collect_pairs(spai: LearnedSpai, solver64: "Solver", nrhs: int, iterates: int = 3, gen=None):
    """Fold nrhs x iterates (r, e) pairs into `spai`: for random x* ~ U[-1,1] (torch
    generator `gen`), b = A x*, the FP64-basis GMRES iterates x_0 = 0, x_1, ..., one Arnoldi
    step apart, give e = x* - x_k and r = A e.  Only the first iterates are used: later
    errors are dominated by smooth modes, and a per-row fit to them yields a P that
    amplifies the rough ones (its least-squares optimum stops GMRES from converging)."""
    torch = _torch()
    for _ in range(nrhs):
        xs = (torch.rand(spai.n, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1).contiguous()
        b = solver64.spmv(xs)
        x = torch.zeros(spai.n, dtype=torch.float64, device="cuda")
        spai.add_pair(xs, x)
        for _ in range(iterates - 1):
            solver64.solve(b, x, tol=0.0, maxit=1)
            spai.add_pair(xs, x)


def mlp_forward(feat, params):
    torch = _torch()
    out = torch.empty(feat.shape[0], 7, dtype=torch.float32, device="cuda")
    w = np.ascontiguousarray(params, np.float32)
    _check(lib().cbg_mlp_forward(feat.shape[0], C.c_void_p(feat.data_ptr()), C.c_void_p(w.ctypes.data),
                                 C.c_void_p(out.data_ptr()), _stream_ptr(None)), "cbg_mlp_forward")
    return out


def mlp_backward(feat, params, gout) -> np.ndarray:
    w = np.ascontiguousarray(params, np.float32)
    g = np.zeros(MLP_NPARAM)
    _check(lib().cbg_mlp_backward(feat.shape[0], C.c_void_p(feat.data_ptr()), C.c_void_p(w.ctypes.data),
                                  C.c_void_p(gout.data_ptr()), C.c_void_p(g.ctypes.data), _stream_ptr(None)),
           "cbg_mlp_backward")
    return g
