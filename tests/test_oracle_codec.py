"""Pins for the oracle's basis codec (Section 4.2 memory accessor; readings R3-R6).

Each check ties the oracle to something other than itself: the format definitions
(exact nearest-value search between representable neighbours), library conversions
(numpy float16, torch bfloat16 / float8_e4m3fn), a worked example of the paper's
sigma formula, and error bounds.
"""
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_finite_values(decode, ncodes, dtype):
    codes = np.arange(ncodes, dtype=np.int64).astype(dtype)
    vals = decode(codes)
    ok = np.isfinite(vals)
    return codes[ok], vals[ok]


def _nearest_even(x, codes, vals, sign_bit):
    """Round-to-nearest-even by definition: locate the representable neighbours of x
    and compare x with their midpoint (exact in FP64 for these formats).  A negative x
    that rounds to zero gives -0 (IEEE 754 keeps the sign)."""
    order = np.lexsort((codes.astype(np.int64), vals))
    v = vals[order]; c = codes[order]
    # drop the duplicate zero (-0 / +0): keep +0 (even code 0)
    keep = np.ones(v.size, bool)
    zs = np.nonzero(v == 0)[0]
    if zs.size > 1:
        keep[zs[c[zs] != 0]] = False
    v = v[keep]; c = c[keep]
    idx = np.searchsorted(v, x, side="right")
    out = np.empty(x.shape, dtype=np.int64)
    for k, (xi, i) in enumerate(zip(x, idx)):
        if i == 0:
            out[k] = c[0]; continue
        if i == v.size or v[i - 1] == xi:
            out[k] = c[i - 1]; continue
        lo, hi = v[i - 1], v[i]
        mid = (lo + hi) / 2
        if xi < mid:
            out[k] = c[i - 1]
        elif xi > mid:
            out[k] = c[i]
        else:
            cl, ch = int(c[i - 1]), int(c[i])
            # ties to the code with an even last mantissa bit
            out[k] = cl if (cl & 1) == 0 else ch
    zero_neg = (out == 0) & (x < 0)
    out[zero_neg] = sign_bit
    return out


def _sample_doubles(rng, n, emin, emax):
    e = rng.uniform(emin, emax, n)
    x = np.ldexp(rng.uniform(0.5, 1.0, n), np.floor(e).astype(int))
    return x * rng.choice([-1.0, 1.0], n)


# ------------------------------------------------------------------------------ f16
def test_f16_decode_matches_numpy_all_codes(oracle_lib):
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = codes.view(np.float16).astype(np.float64)
    got = O.f16_to_f64(codes)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(got[np.isinf(ref)], ref[np.isinf(ref)])


def test_f16_roundtrip_identity_all_codes(oracle_lib):
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    vals = O.f16_to_f64(codes)
    fin = np.isfinite(vals)
    back = O.f64_to_f16(vals[fin])
    assert np.array_equal(back, codes[fin])


def test_f16_encode_nearest_even_by_definition(oracle_lib):
    rng = np.random.default_rng(1)
    x = _sample_doubles(rng, 4000, -27, 16)
    codes, vals = _all_finite_values(O.f16_to_f64, 65536, np.uint16)
    # ties: exact midpoints of neighbouring values (including subnormal ones)
    v = np.sort(np.unique(np.abs(vals)))
    mids = (v[:-1] + v[1:]) / 2
    x = np.concatenate([x, rng.choice(mids, 500), -rng.choice(mids, 500)])
    x = x[np.abs(x) <= 65504.0]
    got = O.f64_to_f16(x).astype(np.int64)
    ref = _nearest_even(x, codes.astype(np.int64), vals, 0x8000)
    assert np.array_equal(got, ref)


def test_f16_encode_matches_numpy_cast(oracle_lib):
    rng = np.random.default_rng(2)
    x = np.concatenate([_sample_doubles(rng, 20000, -30, 17),
                        [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e6, -1e6, 2.0 ** -25,
                         2.0 ** -25 * 1.0000001, 2.0 ** -24, 3 * 2.0 ** -26]])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(O.f64_to_f16(x), ref)


# ----------------------------------------------------------------------------- bf16
def test_bf16_decode_matches_torch_all_codes(oracle_lib):
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = torch.from_numpy(codes.astype(np.int16)).view(torch.bfloat16).double().numpy()
    got = O.bf16_to_f64(codes)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))


def test_bf16_encode_matches_torch_and_definition(oracle_lib):
    rng = np.random.default_rng(3)
    x = _sample_doubles(rng, 20000, -140, 120).astype(np.float32)
    codes, vals = _all_finite_values(O.bf16_to_f64, 65536, np.uint16)
    v = np.sort(np.unique(np.abs(vals)))
    mids = ((v[:-1] + v[1:]) / 2)
    mids = mids[(mids < 3e38) & (mids.astype(np.float32).astype(np.float64) == mids)]
    x = np.concatenate([x, rng.choice(mids, 1000).astype(np.float32)])
    got = O.f32_to_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, ref)
    small = x[:2000].astype(np.float64)
    assert np.array_equal(O.f32_to_bf16(small.astype(np.float32)).astype(np.int64),
                          _nearest_even(small, codes.astype(np.int64), vals, 0x8000))


def test_bf16_roundtrip_identity_all_codes(oracle_lib):
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    vals = O.bf16_to_f64(codes)
    fin = np.isfinite(vals)
    assert np.array_equal(O.f32_to_bf16(vals[fin].astype(np.float32)), codes[fin])


# ----------------------------------------------------------------------------- e4m3
def test_e4m3_decode_matches_torch_all_codes(oracle_lib):
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
    got = O.e4m3_to_f64(codes)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.nanmax(got) == 448.0 and np.isnan(got[0x7F]) and np.isnan(got[0xFF])


def test_e4m3_encode_matches_torch_and_definition(oracle_lib):
    rng = np.random.default_rng(4)
    x = _sample_doubles(rng, 20000, -12, 9)
    x = x[np.abs(x) <= 448.0].astype(np.float32)
    codes, vals = _all_finite_values(O.e4m3_to_f64, 256, np.uint8)
    v = np.sort(np.unique(np.abs(vals)))
    mids = (v[:-1] + v[1:]) / 2
    x = np.concatenate([x, mids.astype(np.float32), -mids.astype(np.float32)])
    got = O.f32_to_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(got, ref)
    xd = x.astype(np.float64)
    assert np.array_equal(got.astype(np.int64), _nearest_even(xd, codes.astype(np.int64), vals, 0x80))


def test_e4m3_saturates(oracle_lib):
    x = np.array([448.0, 460.0, 470.0, 480.0, 1e4, np.inf, -1e4, -np.inf], np.float32)
    got = O.e4m3_to_f64(O.f32_to_e4m3(x))
    assert np.array_equal(got, [448, 448, 448, 448, 448, 448, -448, -448])


def test_e4m3_roundtrip_identity_all_codes(oracle_lib):
    codes = np.arange(256, dtype=np.uint8)
    vals = O.e4m3_to_f64(codes)
    fin = np.isfinite(vals)
    assert np.array_equal(O.f32_to_e4m3(vals[fin].astype(np.float32)), codes[fin])


# ------------------------------------------------------------- fixed point (Section 4.2)
def test_int_codec_worked_example(oracle_lib):
    with open(os.path.join(GOLDEN, "int16_worked_example.txt")) as f:
        rows = [l for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for line in rows:
        lhs, rhs = line.split("|")
        parts = lhs.split()
        fmt = O.FORMATS[parts[0]]
        w = np.array([float(t) for t in parts[1:]])
        want = np.array([int(t) for t in rhs.split()])
        codes, scale, dec = O.compress_roundtrip(fmt, w, np.linalg.norm(w))
        assert np.array_equal(codes.astype(np.int64), want)
        mx = 32767.0 if fmt == O.I16 else 2147483647.0
        sigma_paper = (np.max(np.abs(w)) / np.linalg.norm(w)) / mx
        assert scale == pytest.approx(sigma_paper, rel=1e-15)
        assert np.allclose(dec, want * scale, rtol=0, atol=0)


@pytest.mark.parametrize("fmt", ["i32", "i16"])
def test_int_codec_error_bound_and_range(oracle_lib, fmt):
    f = O.FORMATS[fmt]
    rng = np.random.default_rng(5)
    for n in (1, 7, 1000):
        w = rng.standard_normal(n) * 10.0 ** rng.uniform(-5, 5)
        codes, sigma, dec = O.compress_roundtrip(f, w, np.linalg.norm(w))
        v = w * (1.0 / np.linalg.norm(w))
        mx = 32767 if f == O.I16 else 2147483647
        assert np.abs(codes.astype(np.int64)).max() == mx      # full range used
        assert np.all(np.abs(v - dec) <= 0.5 * sigma * (1 + 1e-9) + 1e-300)


@pytest.mark.parametrize("fmt,fmax,rel", [("bf16", 1.0, 2.0 ** -8), ("e4m3", 448.0, 2.0 ** -4)])
def test_pow2_scale_formats(oracle_lib, fmt, fmax, rel):
    f = O.FORMATS[fmt]
    rng = np.random.default_rng(6)
    for n in (1, 5, 4096):
        w = rng.standard_normal(n)
        codes, s, dec = O.compress_roundtrip(f, w, np.linalg.norm(w))
        v = w * (1.0 / np.linalg.norm(w))
        vmax = np.abs(v).max()
        e = np.log2(s)
        assert e == np.round(e)                                 # power of two
        assert vmax <= fmax * s and vmax > fmax * s / 2         # smallest such power
        # decoded values are exact code * s; error within half an ulp of the format
        # (relative, for the normal range) plus the FP32 pre-rounding
        normal_min = (2.0 ** -126 if f == O.BF16 else 2.0 ** -6) * s
        big = np.abs(v) >= normal_min
        assert np.all(np.abs(v - dec)[big] <= (rel + 2.0 ** -24) * np.abs(v)[big])
        sub_q = (2.0 ** -133 if f == O.BF16 else 2.0 ** -9) * s
        assert np.all(np.abs(v - dec)[~big] <= 0.5 * sub_q * (1 + 1e-6) + 2.0 ** -24 * np.abs(v)[~big])


@pytest.mark.parametrize("fmt,rel", [("f32", 2.0 ** -24), ("f16", 2.0 ** -11)])
def test_plain_float_formats_error_bound(oracle_lib, fmt, rel):
    f = O.FORMATS[fmt]
    rng = np.random.default_rng(7)
    w = rng.standard_normal(5000)
    codes, s, dec = O.compress_roundtrip(f, w, np.linalg.norm(w))
    v = w * (1.0 / np.linalg.norm(w))
    assert s == 1.0
    sub = np.abs(v) < 2.0 ** -14 if f == O.F16 else np.zeros(v.size, bool)
    assert np.all(np.abs(v - dec)[~sub] <= rel * np.abs(v)[~sub])
    assert np.all(np.abs(v - dec)[sub] <= 2.0 ** -25)


def test_f32_codec_is_the_ieee_cast(oracle_lib):
    rng = np.random.default_rng(8)
    v = rng.standard_normal(1000) / 40.0
    codes, s = O.encode(O.F32, v)
    assert np.array_equal(codes, v.astype(np.float32)) and s == 1.0
