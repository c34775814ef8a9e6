"""The double-float (FP32 pair) arithmetic the kernels use for the basis products and the
per-step SpMV, restated step by step in exact rational arithmetic with one IEEE
round-to-nearest-even per operation, and checked against the error bounds the design
relies on:

* splitting an FP64 value into hi = RN32(x), lo = RN32(x - hi) reproduces x within
  2^-48 |x| (the batched solver's value planes);
* the FMA form of TwoProd gives the exact product v*wh as p + e;
* TwoSum gives the exact sum as s + e;
* a row of n multiply-accumulates v_i * (wh_i + wl_i) into (S, C), renormalised at the
  end, is within a few units of 2^-46 of the exact sum for the row lengths of the
  workloads (7 and 27 nonzeros) and for 16-term chunks of the basis products.
No GPU is needed; nothing here imports the CUDA path or the oracle."""
from fractions import Fraction

import numpy as np


def rn32(q):
    """Round an exact rational to the nearest FP32 value (ties to even).  Going through
    the nearest double can round twice, so the FP32 candidate and its two neighbours are
    compared exactly."""
    f = np.float32(float(q))
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - q),
                                     int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1))
    return np.float32(best)


def F(x):
    return Fraction(float(x))


def add(a, b):
    return rn32(F(a) + F(b))


def sub(a, b):
    return rn32(F(a) - F(b))


def mul(a, b):
    return rn32(F(a) * F(b))


def fma(a, b, c):
    return rn32(F(a) * F(b) + F(c))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    e = add(sub(a, sub(s, bb)), sub(b, bb))
    return s, e


def fast_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def df_mac(S, C, v, wh, wl):
    """(S, C) += v * (wh + wl) with v an exact FP32 value: TwoProd by FMA, then TwoSum."""
    p = mul(v, wh)
    pe = fma(v, wh, -p)
    pe = fma(v, wl, pe)
    s, e = two_sum(S, p)
    return s, add(C, add(e, pe))


def split(x):
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return hi, lo


def test_split_is_within_2_pow_minus_48():
    rng = np.random.default_rng(1)
    for x in np.concatenate([rng.standard_normal(3000), rng.uniform(-1, 1, 1000) * 2.0 ** 40,
                             rng.uniform(-1, 1, 1000) * 2.0 ** -60]):
        hi, lo = split(x)
        assert abs(F(hi) + F(lo) - F(x)) <= Fraction(2) ** -48 * abs(F(x))


def test_two_prod_and_two_sum_are_exact():
    rng = np.random.default_rng(2)
    for _ in range(1500):
        a = np.float32(rng.standard_normal() * 2.0 ** int(rng.integers(-20, 20)))
        b = np.float32(rng.standard_normal() * 2.0 ** int(rng.integers(-20, 20)))
        p = mul(a, b)
        e = fma(a, b, -p)
        assert F(p) + F(e) == F(a) * F(b)
        s, t = two_sum(a, b)
        assert F(s) + F(t) == F(a) + F(b)


def _row_error(n, rng, code_bits=None):
    v = rng.standard_normal(n) / np.sqrt(n)
    if code_bits is not None:          # f16-like codes: few significant bits
        v = np.round(v * 2.0 ** code_bits) / 2.0 ** code_bits
    v = v.astype(np.float32)
    w = rng.standard_normal(n)
    S = C = np.float32(0.0)
    exact = Fraction(0)
    for vi, wi in zip(v, w):
        wh, wl = split(wi)
        S, C = df_mac(S, C, vi, wh, wl)
        exact += F(vi) * F(wi)
    S, C = fast_two_sum(S, C)
    scale = sum(abs(F(vi) * F(wi)) for vi, wi in zip(v, w))
    return abs(F(S) + F(C) - exact) / scale


def test_row_accumulation_error_bound():
    """Relative to sum |v_i w_i| (the bound's natural scale): the split of w costs 2^-48
    per term, each TwoSum leaves an FP32 rounding of the correction term (about 2^-48
    relative to the running sum), so short rows stay below n * 2^-46."""
    rng = np.random.default_rng(3)
    for n in (7, 16, 27):
        worst = max(_row_error(n, rng) for _ in range(40))
        assert worst <= n * 2.0 ** -46, (n, worst)
        worst16 = max(_row_error(n, rng, code_bits=11) for _ in range(40))
        assert worst16 <= n * 2.0 ** -46, (n, worst16)
