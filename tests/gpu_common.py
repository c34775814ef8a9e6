"""Shared helpers for the GPU parity tests (imported by tests/test_gpu_*.py only)."""
import numpy as np
import pytest

FORMATS = ["f64", "f32", "f16", "bf16", "e4m3", "i32", "i16"]


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_12101_gb300 as cb
    cb.ensure_built()
    cb.lib()
    return torch, cb


def to_dev(torch, a, n_pad=None):
    a = np.ascontiguousarray(a, np.float64)
    t = torch.zeros(n_pad if n_pad else a.size, dtype=torch.float64, device="cuda")
    t[: a.size] = torch.from_numpy(a).cuda()
    return t


def col_relerr(Hg, Ho, k):
    """Column-wise relative difference of the first k Hessenberg columns."""
    out = []
    for j in range(k):
        a = Hg[: j + 2, j]; b = Ho[: j + 2, j]
        out.append(np.linalg.norm(a - b) / np.linalg.norm(b))
    return np.array(out)


def scaled_matrix(A, case):
    """A test matrix outside the usual scale: A times 2^-70 ("tiny") or 2^40 ("huge"), which
    the solvers normalise by a power of two, or with every 50th off-diagonal nonzero
    times 2^-80 ("wide": a dynamic range beyond 2^64, where the per-step SpMV keeps FP64
    products); "one" leaves A as it is."""
    import workloads as W
    v = A.val.copy()
    if case == "wide":
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        v[np.flatnonzero(A.col != rows)[::50]] *= 2.0 ** -80
    else:
        v *= {"one": 1.0, "tiny": 2.0 ** -70, "huge": 2.0 ** 40}[case]
    return W.CSR(A.n, A.rowptr, A.col, v)
