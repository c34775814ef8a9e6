"""The allocation-free basis dot product (cbg_basis_dot_noalloc) against the allocating
one (cbg_basis_dot), called through the C ABI.

The no-alloc variant exists for callers that cannot let a library call cudaMalloc /
cudaFree: applications whose device memory belongs to another allocator, and loops
that cannot take the device-wide synchronisation of cudaFree.  Its scratch is one
static device array shared by every call, so two calls in a row must both be right
(the second finds the first one's leftovers in the array).  This file is collected
last so that a failure here never hides the other tests."""
import numpy as np
import pytest

import oracle as O
from gpu_common import need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _basis(fmt, n, ncols, ld, seed):
    rng = np.random.default_rng(seed)
    f = O.FORMATS[fmt]
    codes = np.zeros((ncols, ld), dtype=O.CODE_DTYPE[f])
    scales = np.zeros(ncols)
    for k in range(ncols):
        w = rng.standard_normal(n)
        c, s, _ = O.compress_roundtrip(f, w, np.linalg.norm(w))
        codes[k, :n] = c
        scales[k] = s
    return codes, scales


@pytest.mark.parametrize("fmt,arith", [("f32", "df32"), ("i16", "df32"), ("f64", "fp64")])
def test_noalloc_dot_matches_allocating_dot_twice(fmt, arith):
    torch, cb = need_gpu()
    for call, (n, ncols) in enumerate([(70001, 57), (9000, 3)]):   # two calls in a row
        ld = (n + cb.TILE_ROWS - 1) // cb.TILE_ROWS * cb.TILE_ROWS
        codes, scales = _basis(fmt, n, ncols, ld, seed=11 + call)
        w = np.random.default_rng(5 + call).standard_normal(n)
        Vt = torch.from_numpy(codes.view(np.uint8).reshape(ncols, -1)).cuda()
        wd = to_dev(torch, w, ld)
        h_ref = cb.basis_dot(fmt, arith, n, Vt, ld, scales, wd)
        h_new = cb.basis_dot_noalloc(fmt, arith, n, Vt, ld, scales, wd)
        dec = np.stack([O.decode(O.FORMATS[fmt], codes[k, :n], scales[k]) for k in range(ncols)])
        tol = 1e-13 * np.linalg.norm(w) * np.linalg.norm(dec, axis=1)
        assert np.all(np.abs(h_new - h_ref) <= tol), (call, np.max(np.abs(h_new - h_ref) / tol))


def test_noalloc_rejects_too_many_columns():
    torch, cb = need_gpu()
    n, ncols = 4096, 257
    V = torch.zeros((ncols, 4096 * 4), dtype=torch.uint8, device="cuda")
    w = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(cb.CbgError) as e:
        cb.basis_dot_noalloc("f32", "df32", n, V, 4096, np.ones(ncols), w)
    assert e.value.status == -1
