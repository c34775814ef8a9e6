"""Plain CPU FP64 oracle for compressed-basis GMRES (arXiv 2009.12101).

TEST INFRASTRUCTURE ONLY.  The oracle is a slow, plain restatement of the method
(Fig. 1, Sections 2-5), written in plain C (``cbg_oracle.c``) and loaded here with
ctypes.  Its loops over rows and over the fixed blocks of inner products may run on
several host threads (OpenMP); the results do not depend on the thread count.  Only
the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline may import it.  It shares no code with the CUDA library in
``paper_2009_12101_gb300``; neither imports the other.  Parity pins that tie the
oracle to the paper and to mathematics live in ``tests/test_oracle_*.py``.

Learned-preconditioner parts (MLP forward/backward) have no counterpart in the paper:
parity unpinned by the paper; they are pinned to finite differences and to a numpy
restatement in the tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbg_oracle.c")
_HDR = os.path.join(_HERE, "cbg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
# A prebuilt copy of the oracle to load instead of building this one: the planted-mistake
# tests (tests/test_oracle_mutants.py) point it at copies with one deliberate error each.
_LIB_OVERRIDE = os.environ.get("CBG_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

F64, F32, F16, BF16, E4M3, I32, I16 = range(7)
FORMATS = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "e4m3": E4M3, "i32": I32, "i16": I16}
CODE_DTYPE = {F64: np.float64, F32: np.float32, F16: np.uint16, BF16: np.uint16,
              E4M3: np.uint8, I32: np.int32, I16: np.int16}
PC_NONE, PC_JACOBI, PC_SPAI, PC_BJ4 = 0, 1, 2, 3
REORTH_ALWAYS, REORTH_CONDITIONAL, REORTH_NEVER = 0, 1, 2
ORTHO_CGS, ORTHO_MGS = 0, 1
OK, NOT_CONVERGED, ERR_ARG, ERR_NONFINITE = 0, 1, -1, -2


CFLAGS = ["-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP, no contraction of a*b+c into fma;
    no -march=native, so x86 and aarch64 builds round alike)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(__file__))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(t: int) -> None:
    """Host threads of the oracle's parallel loops (results do not depend on it)."""
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())


class GmresArgs(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("fmt", C.c_int32), ("precond", C.c_int32), ("reorth", C.c_int32),
        ("literal_fig1", C.c_int32), ("adapt", C.c_int32),
        ("eta", C.c_double), ("eps_bd", C.c_double), ("tol", C.c_double),
        ("maxit", C.c_int64), ("pvals", C.c_void_p),
        ("H1", C.c_void_p), ("V1", C.c_void_p), ("hist", C.c_void_p), ("hist_cap", C.c_int64),
        ("tres", C.c_void_p), ("tres_cap", C.c_int64),
        ("iters", C.c_int64), ("cycles", C.c_int64), ("reorths", C.c_int64), ("k1", C.c_int64),
        ("nhist", C.c_int64), ("ntres", C.c_int64),
        ("true_relres", C.c_double), ("est_relres", C.c_double),
        ("status", C.c_int32), ("pad1", C.c_int32),
        ("adapt_gap", C.c_double), ("fmt_final", C.c_int32), ("promotions", C.c_int32),
        ("ortho", C.c_int32), ("pad2", C.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_LIB_OVERRIDE or build())
            vp, i64, d = C.c_void_p, C.c_int64, C.c_double
            for name in ("or_vec_f64_to_f16", "or_vec_f16_to_f64", "or_vec_f32_to_bf16",
                         "or_vec_bf16_to_f64", "or_vec_f32_to_e4m3", "or_vec_e4m3_to_f64"):
                getattr(L, name).argtypes = [i64, vp, vp]
                getattr(L, name).restype = None
            L.or_encode.argtypes = [C.c_int, i64, vp, d, vp, C.POINTER(d)]
            L.or_decode.argtypes = [C.c_int, i64, vp, d, vp]
            L.or_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
            L.or_spmv.restype = None
            L.or_set_threads.argtypes = [C.c_int]
            L.or_set_threads.restype = None
            L.or_get_threads.argtypes = []
            L.or_get_threads.restype = C.c_int
            L.or_dot.argtypes = [i64, vp, vp]
            L.or_dot.restype = d
            L.or_gram_schmidt_pass.argtypes = [i64, vp, i64, C.c_int, vp, vp]
            L.or_gmres.argtypes = [i64, vp, vp, vp, vp, vp, C.POINTER(GmresArgs)]
            L.or_mlp_forward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.or_spai_slots.argtypes = [i64, vp, vp, i64, i64, vp]
            L.or_spai_accumulate.argtypes = [i64, vp, vp, vp, vp, vp, d, vp, vp, vp]
            L.or_spai_loss.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, d, vp]
            L.or_spai_loss.restype = d
            L.or_mlp_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                          vp, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------ codec
def f64_to_f16(x):
    x = _c(x, np.float64); out = np.empty(x.shape, np.uint16)
    lib().or_vec_f64_to_f16(x.size, _p(x), _p(out)); return out


def f16_to_f64(c):
    c = _c(c, np.uint16); out = np.empty(c.shape, np.float64)
    lib().or_vec_f16_to_f64(c.size, _p(c), _p(out)); return out


def f32_to_bf16(x):
    x = _c(x, np.float32); out = np.empty(x.shape, np.uint16)
    lib().or_vec_f32_to_bf16(x.size, _p(x), _p(out)); return out


def bf16_to_f64(c):
    c = _c(c, np.uint16); out = np.empty(c.shape, np.float64)
    lib().or_vec_bf16_to_f64(c.size, _p(c), _p(out)); return out


def f32_to_e4m3(x):
    x = _c(x, np.float32); out = np.empty(x.shape, np.uint8)
    lib().or_vec_f32_to_e4m3(x.size, _p(x), _p(out)); return out


def e4m3_to_f64(c):
    c = _c(c, np.uint8); out = np.empty(c.shape, np.float64)
    lib().or_vec_e4m3_to_f64(c.size, _p(c), _p(out)); return out


def encode(fmt: int, v, vmax: float | None = None):
    """Encode a normalised FP64 vector; returns (codes, scale)."""
    v = _c(v, np.float64)
    if vmax is None:
        vmax = float(np.max(np.abs(v))) if v.size else 0.0
    codes = np.empty(v.shape, CODE_DTYPE[fmt])
    scale = C.c_double()
    rc = lib().or_encode(fmt, v.size, _p(v), vmax, _p(codes), C.byref(scale))
    if rc:
        raise ValueError(f"or_encode failed ({rc})")
    return codes, scale.value


def decode(fmt: int, codes, scale: float):
    codes = _c(codes, CODE_DTYPE[fmt])
    out = np.empty(codes.shape, np.float64)
    rc = lib().or_decode(fmt, codes.size, _p(codes), scale, _p(out))
    if rc:
        raise ValueError(f"or_decode failed ({rc})")
    return out


def compress_roundtrip(fmt: int, w, h: float):
    """v = w * (1/h), encoded and decoded as the basis store does (readings R3-R6)."""
    w = _c(w, np.float64)
    v = w * (1.0 / h)
    codes, scale = encode(fmt, v, float(np.max(np.abs(v))) if v.size else 0.0)
    return codes, scale, decode(fmt, codes, scale)


# ----------------------------------------------------------------------- building blocks
def spmv(A, x):
    x = _c(x, np.float64); y = np.empty(A.n, np.float64)
    rp, ci, va = _c(A.rowptr, np.int32), _c(A.col, np.int32), _c(A.val, np.float64)
    lib().or_spmv(A.n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def dot(a, b):
    a = _c(a, np.float64); b = _c(b, np.float64)
    return lib().or_dot(a.size, _p(a), _p(b))


def gram_schmidt_pass(V, w, ortho=ORTHO_CGS):
    """One Gram-Schmidt pass of w against the columns of V (n x k): returns (coefficients,
    reduced w); CGS as Fig. 1 prints it or the MGS variant."""
    V = np.asarray(V, np.float64)
    n, k = V.shape
    Vc = np.asfortranarray(V)
    w = np.array(w, dtype=np.float64, copy=True)
    c = np.zeros(k)
    lib().or_gram_schmidt_pass(n, Vc.ctypes.data, k, ortho, _p(w), _p(c))
    return c, w


# -------------------------------------------------------------------------------- GMRES
def gmres(A, b, x0=None, *, m: int = 100, fmt: int = F64, precond: int = PC_NONE,
          pvals=None, reorth: int = REORTH_ALWAYS, eta: float = 2 ** -0.5,
          eps_bd: float = 2.0 ** -46, literal_fig1: bool = False, tol: float = 1e-10,
          maxit: int | None = None, want_H1: bool = False, want_V1: bool = False,
          hist_cap: int = 0, tres_cap: int = 0, adapt: bool = False, adapt_gap: float = 4.0,
          ortho: int = ORTHO_CGS) -> dict:
    """Run the oracle's GMRES(m).  Returns a dict with x, status, iters, cycles, reorths,
    true_relres, est_relres and the optional H1 ((m+1) x m raw Hessenberg of the first
    cycle), V1 (decoded basis of the first cycle), hist, tres."""
    n = A.n
    maxit = 20 * n if maxit is None else maxit
    b = _c(b, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rp, ci, va = _c(A.rowptr, np.int32), _c(A.col, np.int32), _c(A.val, np.float64)
    a = GmresArgs()
    a.m, a.fmt, a.precond, a.reorth = m, fmt, precond, reorth
    a.literal_fig1 = int(literal_fig1)
    a.adapt, a.adapt_gap = int(adapt), adapt_gap
    a.ortho = ortho
    a.eta, a.eps_bd, a.tol, a.maxit = eta, eps_bd, tol, maxit
    keep = []
    if pvals is not None:
        pv = _c(pvals, np.float64); keep.append(pv); a.pvals = pv.ctypes.data
    H1 = V1 = hist = tres = None
    if want_H1:
        H1 = np.zeros((m, m + 1)); a.H1 = H1.ctypes.data  # column-major (m+1) x m
    if want_V1:
        ncols = min(m, maxit) + 1
        V1 = np.zeros((ncols, n)); a.V1 = V1.ctypes.data
    if hist_cap:
        hist = np.zeros(hist_cap); a.hist = hist.ctypes.data; a.hist_cap = hist_cap
    if tres_cap:
        tres = np.zeros(tres_cap); a.tres = tres.ctypes.data; a.tres_cap = tres_cap
    lib().or_gmres(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), C.byref(a))
    out = dict(x=x, status=a.status, iters=a.iters, cycles=a.cycles, reorths=a.reorths,
               true_relres=a.true_relres, est_relres=a.est_relres, k1=a.k1,
               fmt_final=a.fmt_final, promotions=a.promotions)
    if H1 is not None:
        out["H1"] = H1.T.copy()            # (m+1) x m
    if V1 is not None:
        out["V1"] = V1.T[:, : a.k1 + 1].copy()
    if hist is not None:
        out["hist"] = hist[: a.nhist].copy()
    if tres is not None:
        out["tres"] = tres[: a.ntres].copy()
    return out


# ------------------------------------------------------------------ learned preconditioner
MLP_IN, MLP_H, MLP_OUT = 7, 64, 7


def mlp_forward(feat, W1, b1, W2, b2, W3, b3, want_acts: bool = False):
    feat = _c(feat, np.float64); rows = feat.shape[0]
    ps = [_c(t, np.float64) for t in (W1, b1, W2, b2, W3, b3)]
    out = np.empty((rows, MLP_OUT))
    a1 = np.empty((rows, MLP_H)) if want_acts else None
    a2 = np.empty((rows, MLP_H)) if want_acts else None
    lib().or_mlp_forward(rows, _p(feat), *[_p(t) for t in ps], _p(out),
                         _p(a1) if want_acts else None, _p(a2) if want_acts else None)
    return (out, a1, a2) if want_acts else out


def mlp_backward(feat, W1, b1, W2, b2, W3, b3, gout):
    feat = _c(feat, np.float64); gout = _c(gout, np.float64); rows = feat.shape[0]
    ps = [_c(t, np.float64) for t in (W1, b1, W2, b2, W3, b3)]
    g = [np.empty_like(t) for t in ps]
    lib().or_mlp_backward(rows, _p(feat), *[_p(t) for t in ps], _p(gout), *[_p(t) for t in g])
    return g


# ---------------------------------------------------- learned SPAI statistics and loss
def spai_slots(A, sx: int, sxy: int):
    rp, ci = _c(A.rowptr, np.int32), _c(A.col, np.int32)
    slot = np.empty(ci.size, np.int8)
    if lib().or_spai_slots(A.n, _p(rp), _p(ci), sx, sxy, _p(slot)):
        raise ValueError("pattern is not a 3D 7-point stencil with the given strides")
    return slot


def spai_accumulate(A, slot, r, e, G=None, c=None, d=None):
    """Add one (r, e) pair (weight 1/||e||^2) to the per-row statistics."""
    n = A.n
    G = np.zeros((n, 49)) if G is None else G
    c = np.zeros((n, 7)) if c is None else c
    d = np.zeros(n) if d is None else d
    rp, ci = _c(A.rowptr, np.int32), _c(A.col, np.int32)
    r = _c(r, np.float64); e = _c(e, np.float64)
    lib().or_spai_accumulate(n, _p(rp), _p(ci), _p(slot), _p(r), _p(e), 1.0 / float(e @ e),
                             _p(G), _p(c), _p(d))
    return G, c, d


def spai_loss(A, slot, out, diag, G, c, d, npairs, want_grad=False):
    rp = _c(A.rowptr, np.int32)
    out = _c(out, np.float64); diag = _c(diag, np.float64)
    gout = np.empty_like(out) if want_grad else None
    loss = lib().or_spai_loss(A.n, _p(rp), _p(slot), _p(out), _p(diag), _p(G), _p(c), _p(d),
                              float(npairs), _p(gout) if want_grad else None)
    return (loss, gout) if want_grad else loss
