"""The complex128 digit-product scheme of the tensor-core kernel for k = 3..5,
emulated exactly on the host.

A dense complex128 gate is applied as the real GEMM y = W x, with x a slice
row of 2D reals and W the 2D x 2D real form of U (Eq. 3). Both operands are
cut into seven signed 7-bit digits and multiplied digit by digit
(Ozaki-style). The kernel relies on several integer bounds:
- the fp32 accumulators of each digit weight d = i + j <= 7 hold exact
  integers (below 2^23);
- the weights d <= 3 fit the magic-number conversion (below 2^22);
- the pairs packed into 32-bit integers in the epilogue do not overflow.
These tests check those bounds at their worst case. They also check the
error of the assembled result against exact rational arithmetic.

No CUDA and no oracle are involved: these tests check the arithmetic that
the kernel is designed around. The GPU parity tests check the kernel
itself."""
from fractions import Fraction

import numpy as np
import pytest

DIGITS = 7


def row_exponent(v):
    """The smallest E with every |v| < 2^E (that of the largest entry)."""
    m = float(np.max(np.abs(v)))
    return int(np.frexp(m)[1]) if m > 0 else -1022


def split(v, E):
    """Seven signed 7-bit digits of v / 2^E rounded to 49 fractional bits:
    v ~ 2^E sum_i a_i 2^(-7(i+1)), every digit with the sign of v."""
    F = np.rint(np.ldexp(np.abs(v), 49 - E)).astype(np.int64)
    F = np.minimum(F, (1 << 49) - 1)
    s = np.where(v < 0, -1, 1).astype(np.int64)
    return [s * ((F >> (7 * (DIGITS - 1 - i))) & 127) for i in range(DIGITS)]


def accumulate(ax, bw):
    """acc[d] = sum over digit pairs i + j = d <= 7 of w_j . a_i (exact)."""
    acc = np.zeros((8, bw[0].shape[0]), dtype=np.int64)
    for i in range(DIGITS):
        for j in range(DIGITS):
            if i + j <= 7:
                acc[i + j] += bw[j] @ ax[i]
    return acc


def assemble(acc):
    """The epilogue at the common scale 2^-36 of the weight-0 products:
    the exact weights 0..3 paired in 32 bits; weight 4 exact; weights 5..7
    summed in fp32 (two roundings) and converted once.  Returns Y and the
    three 32-bit parts."""
    hi = acc[0] * 128 + acc[1]
    mid = acc[2] * 128 + acc[3]
    t = np.float32(2.0 * acc[5].astype(np.float64) + acc[6].astype(np.float64) * 2.0 ** -6)
    t = np.float32(t.astype(np.float64) + acc[7].astype(np.float64) * 2.0 ** -13)
    lo = acc[4] * 256 + np.rint(t.astype(np.float64)).astype(np.int64)
    Y = hi * (1 << 29) + mid * (1 << 15) + lo
    return Y, hi, mid, lo


def real_form(u):
    d = u.shape[0]
    W = np.zeros((2 * d, 2 * d))
    W[0::2, 0::2] = u.real
    W[0::2, 1::2] = -u.imag
    W[1::2, 0::2] = u.imag
    W[1::2, 1::2] = u.real
    return W


def apply_digits(u, x):
    """y = W x through the digit scheme; returns (y as exact Fractions, acc
    of every output row, the 32-bit parts, E_r, E_n)."""
    W = real_form(u)
    xr = np.empty(2 * x.size)
    xr[0::2], xr[1::2] = x.real, x.imag
    Er = row_exponent(xr)
    ax = split(xr, Er)
    En = np.array([row_exponent(W[n]) for n in range(W.shape[0])])
    bw = [np.zeros(W.shape, dtype=np.int64) for _ in range(DIGITS)]
    for n in range(W.shape[0]):
        for j, dj in enumerate(split(W[n], En[n])):
            bw[j][n] = dj
    acc = accumulate(ax, bw)
    Y, hi, mid, lo = assemble(acc)
    y = [Fraction(int(Y[n])) * Fraction(2) ** int(Er + En[n] - 50) for n in range(W.shape[0])]
    return y, acc, (hi, mid, lo), Er, En, W, xr


def haar(k, rng):
    d = 1 << k
    z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("k", [3, 4, 5])
def test_bounds_hold_with_every_digit_at_its_largest(k):
    """Every digit 127 with one sign: the largest sums the accumulators can
    hold (K = 2^(k+1) reals per row)."""
    K = 2 << k
    ax = [np.full(K, 127, dtype=np.int64) for _ in range(DIGITS)]
    bw = [np.full((K, K), 127, dtype=np.int64) for _ in range(DIGITS)]
    acc = accumulate(ax, bw)
    for d in range(8):
        pairs = min(d, 6) - max(0, d - 6) + 1
        assert np.all(acc[d] == pairs * K * 127 * 127)
    assert np.max(np.abs(acc)) < 2 ** 23          # exact in fp32 (24 bits)
    assert np.max(np.abs(acc[:4])) < 2 ** 22      # magic-number conversion range
    _, hi, mid, lo = assemble(acc)
    for part in (hi, mid, lo):
        assert np.max(np.abs(part)) < 2 ** 31     # 32-bit packing
    if k == 5:  # the bounds are tight: weight 3 sits just below 2^22
        assert acc[3].max() > 0.98 * 2 ** 22


def test_k6_would_break_the_bounds():
    """Where the one-pass epilogue stops: with K = 128 reals (k = 6) the
    weight-3 sum passes the 2^22 range of the magic-number conversion and
    the weight-4 term of the 32-bit low part passes 2^31 (the k = 6, 7 kernel
    also runs out of tensor memory for seven digit blocks of 64 columns, so
    it feeds K in chunks and keeps six accumulators with its own epilogue)."""
    K = 128
    ax = [np.full(K, 127, dtype=np.int64) for _ in range(DIGITS)]
    bw = [np.full((1, K), 127, dtype=np.int64) for _ in range(DIGITS)]
    acc = accumulate(ax, bw)
    assert acc[3].max() >= 2 ** 22
    assert acc[4].max() * 256 >= 2 ** 31
    assert acc.max() < 2 ** 24  # the fp32 sums themselves would still be exact


def max_error(k, seed, drop_from=8):
    """Largest |y - exact| over the outputs of twelve Haar gates on random
    slice rows (some with magnitudes spread over 40 binades, some far from
    unit scale), in units of 2^(E_r + E_n); the accumulators of weight
    drop_from and above are left out (a planted mistake)."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for trial in range(12):
        u = haar(k, rng)
        d = 1 << k
        x = rng.normal(size=d) + 1j * rng.normal(size=d)
        if trial % 3 == 1:
            x *= np.exp2(rng.integers(-40, 1, size=d))
        if trial % 3 == 2:
            x *= 2.0 ** -300
        _, acc, _, Er, En, W, xr = apply_digits(u, x)
        assert np.max(np.abs(acc)) < 2 ** 23
        acc = acc.copy()
        acc[drop_from:] = 0
        Y, *_ = assemble(acc)
        for n in range(2 * d):
            exact = sum(Fraction(float(W[n, c])) * Fraction(float(xr[c])) for c in range(2 * d))
            got = Fraction(int(Y[n])) * Fraction(2) ** int(Er + En[n] - 50)
            worst = max(worst, abs(float(got - exact)) / 2.0 ** (Er + En[n]))
    return worst


@pytest.mark.parametrize("k", [3, 4, 5])
def test_result_within_the_error_bound(k):
    """The assembled result agrees with the exact product of the FP64 inputs
    to ~2^-48 of 2^(E_r + E_n) (measured 2^-48.4 .. 2^-47.4 here): the
    rounding of both operands to 49 bits, the dropped pairs of weight 8 and
    above, and the two fp32 roundings of the low weights."""
    worst = max_error(k, 40 + k)
    assert 0.0 < worst < 2.0 ** -46


@pytest.mark.parametrize("k", [3, 4, 5])
def test_a_dropped_digit_weight_would_show(k):
    """Planted mistake: without the weight-7 pairs the error grows past the
    bound above (to ~2^-44), without weights 6 and 7 to ~2^-37."""
    assert max_error(k, 40 + k, drop_from=7) > 2.0 ** -46
    assert max_error(k, 40 + k, drop_from=6) > 2.0 ** -40
