"""Multi-RHS basis product H = V^T W (k <= 64 vectors sharing one compressed basis, in
groups of 8) against the oracle's dot products, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_common import FORMATS, need_gpu

pytestmark = pytest.mark.gpu


def _basis(fmt, n, ncols, ld, seed):
    rng = np.random.default_rng(seed)
    f = O.FORMATS[fmt]
    itemsize = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "e4m3": 1, "i32": 4, "i16": 2}[fmt]
    codes = np.zeros((ncols, ld * itemsize), dtype=np.uint8)
    scales = np.zeros(ncols)
    dec = np.zeros((ncols, n))
    for c in range(ncols):
        w = rng.standard_normal(n) * np.exp(rng.uniform(-4, 2, n))
        cd, s, d = O.compress_roundtrip(f, w, np.linalg.norm(w))
        codes[c, : n * itemsize] = cd.view(np.uint8)
        scales[c] = s
        dec[c] = d
    return codes, scales, dec


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n,ncols,k", [(5000, 1, 1), (12289, 13, 3), (40000, 40, 8), (70001, 9, 5), (9000, 101, 4),
                                        (9000, 37, 16), (4096, 12, 21)])
def test_basis_dot_multi_matches_oracle(fmt, n, ncols, k):
    torch, cb = need_gpu()
    ld = (n + 4095) // 4096 * 4096
    codes, scales, dec = _basis(fmt, n, ncols, ld, seed=n + ncols + k)
    rng = np.random.default_rng(k)
    W = rng.standard_normal((k, n)) * np.exp(rng.uniform(-3, 3, (k, 1)))
    Vt = torch.from_numpy(codes).cuda()
    Wd = torch.from_numpy(W).cuda()
    H = cb.basis_dot_multi(fmt, n, Vt, ld, scales, Wd).cpu().numpy()
    ref = np.array([[O.dot(dec[c], W[r]) for r in range(k)] for c in range(ncols)])
    tol = 1e-13 * np.linalg.norm(dec, axis=1)[:, None] * np.linalg.norm(W, axis=1)[None, :]
    assert H.shape == (ncols, k)
    assert np.all(np.abs(H - ref) <= tol), np.max(np.abs(H - ref) / tol)


def test_basis_dot_multi_rejects_bad_arguments():
    torch, cb = need_gpu()
    V = torch.zeros((3, 4096 * 4), dtype=torch.uint8, device="cuda")
    W = torch.zeros((65, 4096), dtype=torch.float64, device="cuda")
    with pytest.raises(cb.CbgError):
        cb.basis_dot_multi("f32", 4096, V, 4096, np.ones(3), W)     # k = 65 > 64


@pytest.mark.parametrize("n,ncols,k", [(5000, 1, 1), (12289, 13, 3), (40000, 40, 8), (70001, 9, 5),
                                        (9000, 101, 4), (20480, 128, 8), (2049, 7, 2), (9000, 64, 16),
                                        (12289, 100, 20)])
def test_basis_dot_multi_tensor_cores(n, ncols, k):
    """The tcgen05 path (f16 basis): exact digit products on the tensor cores, compared with
    the oracle and with the double-float CUDA-core path."""
    torch, cb = need_gpu()
    ld = (n + 4095) // 4096 * 4096
    codes, scales, dec = _basis("f16", n, ncols, ld, seed=3 * n + ncols + k)
    rng = np.random.default_rng(k + 17)
    W = rng.standard_normal((k, n)) * np.exp(rng.uniform(-3, 3, (k, 1)))
    W[:, : n // 3] *= 1e-9                       # blocks of very different magnitude
    Vt = torch.from_numpy(codes).cuda()
    Wd = torch.from_numpy(W).cuda()
    Ht = cb.basis_dot_multi("f16", n, Vt, ld, scales, Wd, path="tensor").cpu().numpy()
    Hc = cb.basis_dot_multi("f16", n, Vt, ld, scales, Wd, path="cuda").cpu().numpy()
    ref = np.array([[O.dot(dec[c], W[r]) for r in range(k)] for c in range(ncols)])
    tol = 1e-13 * np.linalg.norm(dec, axis=1)[:, None] * np.linalg.norm(W, axis=1)[None, :]
    assert np.all(np.abs(Ht - ref) <= tol), np.max(np.abs(Ht - ref) / tol)
    assert np.all(np.abs(Ht - Hc) <= 2 * tol)


def _f16_codes(vals, ld):
    """Raw f16 codes (scale 1) of the columns of vals, zero-padded to ld rows."""
    ncols, n = vals.shape
    codes = np.zeros((ncols, ld), dtype=np.float16)
    codes[:, :n] = vals.astype(np.float16)
    return codes.view(np.uint8), codes[:, :n].astype(np.float64)


def test_basis_dot_multi_tensor_full_code_range():
    """Codes anywhere in [-1, 1] (subnormals, exact powers of two, the endpoints) are cut
    exactly; W spans a wide exponent range; many CTAs whose chunk ranges start inside
    512-row blocks."""
    torch, cb = need_gpu()
    n, ncols, k = 400_037, 24, 8
    ld = (n + 4095) // 4096 * 4096
    rng = np.random.default_rng(5)
    vals = rng.uniform(-1, 1, (ncols, n)) * np.exp2(rng.integers(-30, 1, (ncols, n)))
    vals[:, :8] = [1.0, -1.0, 2.0 ** -24, -(2.0 ** -24), 2.0 ** -14, 0.5, -0.5, 0.99951171875]
    raw, dec = _f16_codes(vals, ld)
    W = rng.standard_normal((k, n)) * np.exp2(rng.integers(-40, 40, (k, 1)))
    W[:, 100_000:200_000] *= np.exp2(rng.integers(-200, 60, (k, 1)))   # blocks far apart in scale
    Ht = cb.basis_dot_multi("f16", n, torch.from_numpy(raw).cuda(), ld, np.ones(ncols),
                            torch.from_numpy(W).cuda(), path="tensor").cpu().numpy()
    ref = np.array([[O.dot(dec[c], W[r]) for r in range(k)] for c in range(ncols)])
    tol = 1e-13 * np.linalg.norm(dec, axis=1)[:, None] * np.linalg.norm(W, axis=1)[None, :]
    assert np.all(np.abs(Ht - ref) <= tol), np.max(np.abs(Ht - ref) / tol)


@pytest.mark.parametrize("what", ["code_above_1", "w_inf", "w_nan"])
def test_basis_dot_multi_tensor_flags_inputs_outside_its_range(what):
    """Inputs the exact digit cut does not cover make the whole result NaN, not a silently
    wrong number."""
    torch, cb = need_gpu()
    n, ncols, k = 10_000, 5, 3
    ld = 12288
    rng = np.random.default_rng(6)
    vals = rng.uniform(-1, 1, (ncols, n))
    W = rng.standard_normal((k, n))
    if what == "code_above_1":
        vals[3, 7777] = 1.5
    elif what == "w_inf":
        W[1, 4321] = np.inf
    else:
        W[2, 9999] = np.nan
    raw, _ = _f16_codes(vals, ld)
    ws = torch.empty(cb.lib().cbg_basis_dot_multi_workspace(ld, ncols, k), dtype=torch.uint8, device="cuda")
    Ht = cb.basis_dot_multi("f16", n, torch.from_numpy(raw).cuda(), ld, np.ones(ncols),
                            torch.from_numpy(W).cuda(), workspace=ws, path="tensor").cpu().numpy()
    assert np.all(np.isnan(Ht))
    # the next call on the same workspace is clean again
    W2 = rng.standard_normal((k, n))
    vals[3, 7777] = 0.5
    raw, dec = _f16_codes(vals, ld)
    Ht = cb.basis_dot_multi("f16", n, torch.from_numpy(raw).cuda(), ld, np.ones(ncols),
                            torch.from_numpy(W2).cuda(), workspace=ws, path="tensor").cpu().numpy()
    ref = np.array([[O.dot(dec[c], W2[r]) for r in range(k)] for c in range(ncols)])
    assert np.allclose(Ht, ref, rtol=0, atol=1e-12)


def test_basis_dot_multi_tensor_path_limits():
    torch, cb = need_gpu()
    V = torch.zeros((3, 4096 * 4), dtype=torch.uint8, device="cuda")
    W = torch.zeros((2, 4096), dtype=torch.float64, device="cuda")
    with pytest.raises(cb.CbgError) as e:
        cb.basis_dot_multi("f32", 4096, V, 4096, np.ones(3), W, path="tensor")   # f16 only
    assert e.value.status == -6
