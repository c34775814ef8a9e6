"""The allocation-free basis dot product (cbg_basis_dot_noalloc), called through the C
ABI, against the oracle's inner products of the decoded columns and against the
allocating entry point (cbg_basis_dot).

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


def _basis(fmt, n, ncols, ld, w, seed):
    """Random normalised columns stored in `fmt`; returns the codes, the scales, the
    oracle's inner products of the decoded columns with w and the columns' norms."""
    rng = np.random.default_rng(seed)
    f = O.FORMATS[fmt]
    codes = np.zeros((ncols, ld), dtype=O.CODE_DTYPE[f])
    scales = np.zeros(ncols)
    h_o = np.zeros(ncols)
    vnorm = np.zeros(ncols)
    for k in range(ncols):
        v = rng.standard_normal(n)
        c, s, dec = O.compress_roundtrip(f, v, np.linalg.norm(v))
        codes[k, :n] = c
        scales[k] = s
        h_o[k] = O.dot(dec, w)
        vnorm[k] = np.linalg.norm(dec)
    return codes, scales, h_o, vnorm


def _two_calls(torch, cb, fmt, arith, shapes):
    for call, (n, ncols) in enumerate(shapes):   # two calls in a row
        ld = (n + cb.TILE_ROWS - 1) // cb.TILE_ROWS * cb.TILE_ROWS
        w = np.random.default_rng(5 + call).standard_normal(n)
        codes, scales, h_o, vnorm = _basis(fmt, n, ncols, ld, w, seed=11 + call)
        Vt = torch.from_numpy(codes.view(np.uint8).reshape(ncols, -1)).cuda()
        wd = to_dev(torch, w, ld)
        h_new = cb.basis_dot_noalloc(fmt, arith, n, Vt, ld, scales, wd)
        h_ref = cb.basis_dot(fmt, arith, n, Vt, ld, scales, wd)
        # normwise bound, as for the allocating dot: |error| <= 1e-13 ||v|| ||w||
        tol = 1e-13 * np.linalg.norm(w) * vnorm
        assert np.all(np.abs(h_new - h_o) <= tol), (call, np.max(np.abs(h_new - h_o) / tol))
        assert np.all(np.abs(h_new - h_ref) <= tol), (call, np.max(np.abs(h_new - h_ref) / tol))


@pytest.mark.parametrize("fmt,arith", [("f32", "df32"), ("i16", "df32"), ("f64", "fp64")])
def test_noalloc_dot_matches_oracle_twice(fmt, arith):
    torch, cb = need_gpu()
    _two_calls(torch, cb, fmt, arith, [(70001, 57), (9000, 3)])


def test_noalloc_dot_full_scratch_span():
    """ld >= 304 x 1024 rows and 320 columns: the grid reaches its cap of 304 blocks and
    every region of the static scratch (all partial-sum rows, the scales, the result,
    the counter) is written, twice in a row."""
    torch, cb = need_gpu()
    _two_calls(torch, cb, "f16", "df32", [(401000, 320), (333333, 320)])


def test_noalloc_rejects_too_many_columns():
    torch, cb = need_gpu()
    n, ncols = 4096, 321
    V = torch.zeros((ncols, 4096 * 4), dtype=torch.uint8, device="cuda")
    w = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(cb.CbgError) as e:
        cb.basis_dot_noalloc("f32", "df32", n, V, 4096, np.ones(ncols), w)
    assert e.value.status == -1
