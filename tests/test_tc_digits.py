"""The exactness argument of the tensor-core multi-RHS product (csrc/multi_tc.cu),
checked on the CPU by restating each arithmetic step with numpy rounding:

* every f16 code v with |v| <= 1 is cut, in FP16 arithmetic (one rounding per fused
  multiply-add, subnormals kept), into v = hi 2^-11 + lo 2^-12 exactly, with an integer
  |hi| <= 2048 and lo on the 2^-12 grid with |lo| <= 1;
* y = trunc(w 2^(54 - E)) computed from the bits of w equals the exact truncation, and its
  14 signed base-16 digits (nibbles of y + 8 * sum 16^b) reproduce y;
* the digits of two rows are packed pairwise with byte permutes into FP16 pairs holding
  exactly the digits;
* products and 512-row sums stay within 2^24 grid points, so FP32 accumulation is exact.
No GPU is needed; nothing here imports the CUDA path or the oracle."""
import struct
from fractions import Fraction

import numpy as np


def f16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def hfma(a, b, c):
    # a, b, c are FP16 values: a*b + c is exact in FP64 for these magnitudes, then one
    # rounding to FP16, as a fused multiply-add does
    return f16(a * b + c)


def test_v_cut_is_exact_for_every_code_up_to_one():
    bits = np.arange(0, 0x10000, dtype=np.uint32).astype(np.uint16)
    v = bits.view(np.float16).astype(np.float64)
    v = v[np.isfinite(v) & (np.abs(v) <= 1)]
    assert v.size == 30722
    magic = 1536.0
    c = f16(hfma(v, 4.0, magic) - magic)                    # rint(4 v)
    r = hfma(c, -0.25, v)
    assert np.array_equal(r, v - c / 4)                     # exact remainder
    f = f16(hfma(r, 2048.0, magic) - magic)                 # rint(2048 r)
    hi = hfma(c, 512.0, f)
    assert np.array_equal(hi, c * 512 + f)
    lo = f16(hfma(f, -(2.0 ** -11), r) * 4096.0)
    assert np.array_equal(v, hi * 2.0 ** -11 + lo * 2.0 ** -12)
    assert np.array_equal(hi, np.round(hi)) and np.abs(hi).max() == 2048
    assert np.array_equal(lo * 4096, np.round(lo * 4096)) and np.abs(lo).max() <= 1


def test_accumulation_budget():
    # |e| <= 8 for a signed base-16 digit; 512 rows per exact block
    assert 2048 * 8 * 512 <= 2 ** 24                        # hi slice, integer grid
    assert (1 * 4096) * 8 * 512 <= 2 ** 24                  # lo slice, 2^-12 grid


def _trunc_from_bits(w, E):
    u = struct.unpack("<Q", struct.pack("<d", w))[0]
    ex = (u >> 52) & 0x7FF
    m = (u & (2 ** 52 - 1)) | (1 << 52)
    sh = E + 1021 - ex
    q = (m << 1) if sh < 0 else (m >> min(sh, 63))
    if ex == 0 or sh > 63:
        q = 0
    return -q if u >> 63 else q


def test_w_scaling_and_digits():
    rng = np.random.default_rng(4)
    bias = int("88888888888888", 16)                        # 8 in each of 14 nibbles
    for _ in range(20000):
        E = int(rng.integers(-1000, 1000))
        w = float(rng.uniform(0.5, 1.0)) * 2.0 ** (E - int(rng.integers(0, 80)))
        w = -w if rng.random() < 0.5 else w
        if abs(w) >= 2.0 ** E or abs(w) < 2.0 ** -1022:
            continue
        y = _trunc_from_bits(w, E)
        assert y == int(Fraction(w) * Fraction(2) ** (54 - E))   # truncation toward zero
        z = y + bias
        assert 0 <= z < 16 ** 14
        digits = [((z >> (4 * b)) & 15) - 8 for b in range(14)]
        assert all(-8 <= t <= 7 for t in digits)
        assert sum(t * 16 ** b for b, t in enumerate(digits)) == y


def test_digit_pairs_from_byte_permutes():
    def byte_perm(x, y, s):
        b = list(x.to_bytes(4, "little")) + list(y.to_bytes(4, "little"))
        return int.from_bytes(bytes([b[(s >> (4 * k)) & 7] for k in range(4)]), "little")

    def half(bits):
        return float(np.frombuffer(struct.pack("<H", bits), dtype=np.float16)[0])

    rng = np.random.default_rng(5)
    bias = int("88888888888888", 16)
    for _ in range(3000):
        z0 = int(rng.integers(-2 ** 54, 2 ** 54)) + bias
        z1 = int(rng.integers(-2 ** 54, 2 ** 54)) + bias
        for p in (0, 1):                                    # low word: digits 0-7, high: 8-13
            wa, wb = (z0 >> (32 * p)) & 0xFFFFFFFF, (z1 >> (32 * p)) & 0xFFFFFFFF
            for i in range(4 if p == 0 else 3):
                u = byte_perm(wa, wb, i | (i << 4) | ((4 + i) << 8) | ((4 + i) << 12))
                ev = (u & 0x000F000F) | 0x64006400
                od = (u & 0x00F000F0) | 0x64006400
                b = 8 * p + 2 * i
                for word, k, dec in ((ev, b, lambda h: h - 1032), (od, b + 1, lambda h: h / 16 - 72)):
                    t0, t1 = ((z0 >> (4 * k)) & 15) - 8, ((z1 >> (4 * k)) & 15) - 8
                    assert dec(half(word & 0xFFFF)) == t0 and dec(half(word >> 16)) == t1
