"""GPU parity of the basis accessor (Section 4.2) and of the basis products
(the CGS projection and re-orthogonalisation of Fig. 1) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_common import FORMATS, need_gpu, to_dev

pytestmark = pytest.mark.gpu


def _test_vectors(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(n) * np.exp(rng.uniform(-8, 3, n))
    v = w * (1.0 / np.linalg.norm(w))
    return v


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n", [1, 31, 1000, 4097, 65537])
def test_encode_decode_bit_exact(fmt, n):
    torch, cb = need_gpu()
    v = _test_vectors(n, 100 + n)
    if fmt == "f16" and n >= 1000:
        # exact f16 midpoints and subnormal-range values
        k = np.arange(1, 300, dtype=np.float64)
        v[:299] = np.concatenate([(2 * k + 1) * 2.0 ** -25, ])[:299] * np.where(k % 2 == 0, 1, -1)
    vmax = float(np.max(np.abs(v)))
    codes_o, scale_o = O.encode(O.FORMATS[fmt], v, vmax)
    vd = torch.from_numpy(v).cuda()
    codes_g, scale_g = cb.encode(fmt, vd, vmax)
    assert scale_g == scale_o
    cg = codes_g.cpu().numpy().view(codes_o.dtype)
    assert np.array_equal(cg, codes_o), f"{np.count_nonzero(cg != codes_o)} codes differ"
    dec_g = cb.decode(fmt, codes_g, scale_g).cpu().numpy()
    dec_o = O.decode(O.FORMATS[fmt], codes_o, scale_o)
    assert np.array_equal(dec_g, dec_o)


def test_f32_encode_rounding_edges():
    """The f32 encoder rounds FP64 -> FP32 to nearest even with integer operations on the
    normal range; check ties, neighbours of ties, the normal/subnormal boundary, the
    overflow boundary and special values against numpy's correctly rounded cast."""
    torch, cb = need_gpu()
    rng = np.random.default_rng(7)
    f = rng.standard_normal(2000).astype(np.float32) * np.float32(2.0) ** rng.integers(-120, 120, 2000)
    f = f[np.isfinite(f) & (f != 0)].astype(np.float64)
    ulp = np.abs(np.spacing(f.astype(np.float32)).astype(np.float64))
    ties = f + 0.5 * ulp
    above = np.nextafter(ties, np.inf)
    below = np.nextafter(ties, -np.inf)
    tiny = np.float64(np.finfo(np.float32).tiny)
    big = np.float64(np.finfo(np.float32).max)
    edges = np.array([0.0, -0.0, tiny, -tiny, np.nextafter(tiny, 0), tiny * 0.75, tiny * 1e-3, 1e-300,
                      big, -big, big + 0.49 * np.spacing(np.float32(big)), big * (1 + 2.0 ** -25), 1e300,
                      np.inf, -np.inf, 1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 - 2.0 ** -25])
    v = np.concatenate([f, ties, above, below, -ties, edges])
    ref = v.astype(np.float32)
    codes, scale = cb.encode("f32", torch.from_numpy(v).cuda(), 1.0)
    got = codes.cpu().numpy().view(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), np.count_nonzero(got.view(np.uint32) != ref.view(np.uint32))


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3", "i16"])
def test_decode_every_code(fmt):
    """All 2^16 (2^8) codes decode to the oracle's values (finite codes)."""
    torch, cb = need_gpu()
    ncode = 256 if fmt == "e4m3" else 65536
    codes = np.arange(ncode, dtype=np.int64)
    if fmt == "e4m3":
        c_np = codes.astype(np.uint8)
    elif fmt == "i16":
        c_np = codes.astype(np.uint16).view(np.int16)
        c_np = c_np[c_np != -32768]
    else:
        c_np = codes.astype(np.uint16)
    scale = 2.0 ** -3 if fmt in ("bf16", "e4m3") else (1.0 / 32767 if fmt == "i16" else 1.0)
    ref = O.decode(O.FORMATS[fmt], c_np, scale)
    fin = np.isfinite(ref)
    if fmt == "f16":
        fin &= np.abs(ref) <= 65504
    tdt = {"e4m3": torch.uint8, "i16": torch.int16, "f16": torch.int16, "bf16": torch.int16}[fmt]
    ct = torch.from_numpy(c_np.view(np.int16) if fmt in ("f16", "bf16") else c_np).to(tdt).cuda()
    got = cb.decode(fmt, ct, scale).cpu().numpy()
    assert np.array_equal(got[fin], ref[fin])


def _random_basis(fmt, n, ncols, ld, seed):
    """Encoded random unit columns (codes from the oracle), padded to ld rows."""
    rng = np.random.default_rng(seed)
    f = O.FORMATS[fmt]
    codes = np.zeros((ncols, ld), dtype=O.CODE_DTYPE[f])
    scales = np.zeros(ncols)
    dec = np.zeros((ncols, n))
    for k in range(ncols):
        w = rng.standard_normal(n)
        c, s, d = O.compress_roundtrip(f, w, np.linalg.norm(w))
        codes[k, :n] = c; scales[k] = s; dec[k] = d
    return codes, scales, dec


@pytest.mark.parametrize("arith", ["df32", "fp64"])
@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n,ncols", [(5000, 1), (12289, 13), (40000, 64), (8191, 101), (600000, 40),
                                    (20000, 200), (9000, 256), (12289, 301), (4096, 320)])
def test_basis_dot_and_axpy_parity(fmt, arith, n, ncols):
    torch, cb = need_gpu()
    ld = (n + cb.TILE_ROWS - 1) // cb.TILE_ROWS * cb.TILE_ROWS
    codes, scales, dec = _random_basis(fmt, n, ncols, ld, seed=n + ncols)
    rng = np.random.default_rng(3)
    w = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
    Vt = torch.from_numpy(codes.view(np.uint8).reshape(ncols, -1)).cuda()
    wd = to_dev(torch, w, ld)
    h_g = cb.basis_dot(fmt, arith, n, Vt, ld, scales, wd)
    h_o = np.array([O.dot(dec[k], w) for k in range(ncols)])
    # normwise bound: |h_k error| <= 1e-13 * ||v_k|| ||w||
    tol = 1e-13 * np.linalg.norm(w) * np.linalg.norm(dec, axis=1)
    assert np.all(np.abs(h_g - h_o) <= tol), np.max(np.abs(h_g - h_o) / tol)
    # axpy: w - V h
    hc = rng.standard_normal(ncols)
    cb.basis_axpy(fmt, arith, n, Vt, ld, scales, hc, wd)
    got = wd.cpu().numpy()
    ref = w.copy()
    for k in range(ncols):
        ref -= dec[k] * hc[k]
    scale_ref = np.abs(w) + np.abs(dec.T) @ np.abs(hc)
    # FP64: one rounding per operation.  DF32: w, v and c are carried to 47 bits
    # (split error <= 2^-47), products and sums to ~2^-48: <= 2^-45 per term.
    rel = 1.2e-16 * (ncols + 2) if arith == "fp64" else 2.0 ** -45 * (ncols + 2)
    assert np.all(np.abs(got[:n] - ref) <= rel * scale_ref + 1e-300)
    assert np.all(got[n:] == 0.0)


def test_decode_f32_special_values():
    """The integer FP32 -> FP64 widening of the decoders: zeros, subnormals (every leading
    bit position), the normal range ends, infinities and NaN, against numpy's exact
    conversion (scale 1: the decode is the widening itself)."""
    torch, cb = need_gpu()
    bits = [0x00000000, 0x80000000, 0x7F7FFFFF, 0xFF7FFFFF, 0x00800000, 0x80800000, 0x3F800000,
            0x7F800000, 0xFF800000, 0x7FC00000]
    bits += [1 << k for k in range(23)] + [0x80000000 | ((1 << k) | 1) for k in range(1, 23)]
    bits += [0x007FFFFF, 0x807FFFFF, 0x00400001, 0x00000003]
    b = np.array(bits, dtype=np.uint32)
    ref = b.view(np.float32).astype(np.float64)
    ct = torch.from_numpy(b.view(np.int32)).cuda()
    got = cb.decode("f32", ct, 1.0).cpu().numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))
