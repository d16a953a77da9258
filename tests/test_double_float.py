"""The double-float arithmetic of the complex128 CUDA-core kernels, emulated
on the host: a double held as an unevaluated sum hi + lo of two floats.

- split: FP64 -> (hi, lo) by bit manipulation: hi keeps the top 24
  significand bits, lo the next 23.
- the multiply-add: an FMA-based TwoProduct of the heads, the cross terms by
  FMA, and a TwoSum into the running head.
- join: back to FP64.

These tests check the error claims the kernels are designed around, using
exact rational arithmetic for every fp32 operation (each one rounded once,
to nearest even, as the hardware does):
- the split loses under 2^-46 of |x| (the six dropped bits are worth less
  than 2^6 units of the 2^-52 place);
- a multiply-add is good to ~2^-46;
- a dot product of 32 complex terms stays below 2^-44, far inside the 1e-12
  tolerance of complex128.
No CUDA and no oracle are involved."""
from fractions import Fraction

import numpy as np
import pytest


def f32(v):
    """Round an exact rational (or float) to the nearest float32 (ties to
    even), through float64 only when that is exact."""
    if isinstance(v, Fraction):
        # float64 nearest first is exact enough when the value has <= 53 bits;
        # otherwise round the rational directly to 24 bits
        if v == 0:
            return np.float32(0.0)
        sign = -1 if v < 0 else 1
        a = abs(v)
        e = a.numerator.bit_length() - a.denominator.bit_length()
        if Fraction(2) ** e > a:
            e -= 1
        q = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
        n = q.numerator // q.denominator
        r = q - n
        if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
            n += 1
        return np.float32(sign * float(Fraction(n) * Fraction(2) ** (e - 23)))
    return np.float32(v)


def F(x):
    return Fraction(float(x))


def split(x):
    """FP64 -> (hi, lo) as the device does it: hi the top 24 significand
    bits, lo the next 23 (the 6 lowest dropped); |x| < 2^-100 -> 0."""
    b = np.float64(x).view(np.uint64)
    sign = np.uint32((int(b) >> 32) & 0x80000000)
    e = int((int(b) >> 52) & 0x7FF) - 1023
    if e < -100:
        return np.float32(0.0), np.float32(0.0)
    m = int(b) & ((1 << 52) - 1)
    hi = np.uint32(int(sign) | ((e + 127) << 23) | (m >> 29)).view(np.float32)
    te = e - 23 + 127
    t = np.uint32(int(sign) | (te << 23) | ((m >> 6) & 0x7FFFFF)).view(np.float32)
    p = np.uint32(int(sign) | (te << 23)).view(np.float32)
    return hi, f32(F(t) - F(p))


def mac(sh, sl, ah, al, bh, bl):
    """(sh, sl) += (ah, al) * (bh, bl), every fp32 operation rounded once."""
    p = f32(F(ah) * F(bh))
    e = f32(F(ah) * F(bh) - F(p))
    e = f32(F(ah) * F(bl) + F(e))
    e = f32(F(al) * F(bh) + F(e))
    s = f32(F(sh) + F(p))
    bb = f32(F(s) - F(sh))
    t = f32(F(f32(F(sh) - F(f32(F(s) - F(bb))))) + F(f32(F(p) - F(bb))))
    return s, f32(F(sl) + F(f32(F(t) + F(e))))


def value(h, l):
    return F(h) + F(l)


def test_split_keeps_46_bits():
    rng = np.random.default_rng(1)
    x = rng.normal(size=4000) * np.exp2(rng.integers(-90, 90, size=4000))
    worst = 0.0
    for v in x:
        h, l = split(v)
        assert np.float32(h) == np.float32(np.float32(h))  # a float32 value
        err = abs(value(h, l) - F(v)) / abs(F(v))
        worst = max(worst, float(err))
    assert 2.0 ** -47 < worst < 2.0 ** -46
    assert split(1e-31) == (0.0, 0.0)


def test_split_is_exact_for_values_of_47_bits():
    """A double whose significand ends in six zero bits splits exactly."""
    rng = np.random.default_rng(2)
    for _ in range(500):
        m = int(rng.integers(1 << 46, 1 << 47))  # 47 significant bits
        v = float(m) * 2.0 ** int(rng.integers(-80, 30))
        h, l = split(v)
        assert value(h, l) == F(v)


def test_multiply_add_error():
    """One df multiply-add of unit-scale operands: within ~2^-46 of the exact
    result of the split operands (measured 2^-46.1)."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(400):
        a, b, c = rng.normal(size=3)
        ah, al = split(a)
        bh, bl = split(b)
        sh, sl = split(c)
        rh, rl = mac(sh, sl, ah, al, bh, bl)
        exact = value(sh, sl) + value(ah, al) * value(bh, bl)
        scale = abs(value(sh, sl)) + abs(value(ah, al) * value(bh, bl))
        worst = max(worst, float(abs(value(rh, rl) - exact) / scale))
    assert 0.0 < worst < 2.0 ** -45


@pytest.mark.parametrize("length", [32])
def test_complex_dot_product_stays_near_2_to_minus_44(length):
    """A row of a dense 5-qubit gate (32 complex terms) applied to a slice in
    df arithmetic: the error against the exact product of the FP64 inputs,
    relative to sum |u x|, stays below 2^-44 (measured 2^-46.9, the split
    of the inputs included) -- at 30 qubits (|amplitude| ~ 3e-5) ~1e-18
    absolute, against the 1e-12 tolerance."""
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(6):
        u = (rng.normal(size=length) + 1j * rng.normal(size=length)) / np.sqrt(2 * length)
        x = (rng.normal(size=length) + 1j * rng.normal(size=length)) * 3e-5
        rh = rl = ih = il = np.float32(0.0)
        for c in range(length):
            urh, url = split(u[c].real)
            uih, uil = split(u[c].imag)
            xrh, xrl = split(x[c].real)
            xih, xil = split(x[c].imag)
            rh, rl = mac(rh, rl, urh, url, xrh, xrl)
            rh, rl = mac(rh, rl, -uih, -uil, xih, xil)
            ih, il = mac(ih, il, urh, url, xih, xil)
            ih, il = mac(ih, il, uih, uil, xrh, xrl)
        ex_re = sum(F(u[c].real) * F(x[c].real) - F(u[c].imag) * F(x[c].imag) for c in range(length))
        ex_im = sum(F(u[c].real) * F(x[c].imag) + F(u[c].imag) * F(x[c].real) for c in range(length))
        scale = sum(abs(F(u[c].real)) * abs(F(x[c].real)) + abs(F(u[c].imag)) * abs(F(x[c].imag))
                    for c in range(length))
        err = max(abs(value(rh, rl) - ex_re), abs(value(ih, il) - ex_im)) / scale
        worst = max(worst, float(err))
    assert worst < 2.0 ** -44
    assert float(worst * scale) < 1e-16


def test_a_dropped_cross_term_would_show():
    """Planted mistake: a multiply-add without the al * bh term is off by
    ~2^-24, far outside the bound above."""
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(100):
        a, b = rng.normal(size=2)
        ah, al = split(a)
        bh, bl = split(b)
        p = f32(F(ah) * F(bh))
        e = f32(F(ah) * F(bh) - F(p))
        e = f32(F(ah) * F(bl) + F(e))  # al * bh left out
        exact = value(ah, al) * value(bh, bl)
        worst = max(worst, float(abs(F(p) + F(e) - exact) / abs(exact)))
    assert worst > 2.0 ** -30
