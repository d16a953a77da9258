"""The operand splits of the complex64 tensor-core kernels, emulated on the
host with the same bit operations: 3xTF32 (a truncated tf32 head and a
rounded tf32 tail, three of the four products) and split-bf16 (two
truncated bf16 pieces and a rounded third, the six products of weight above
2^-24).

These tests check the claims the kernels are designed around:
- the tf32 pair represents an fp32 operand to 22 significant bits, and the
  bf16 triple represents it exactly (3 x 8 = 24 bits);
- the remainders are exact;
- the dropped products are below those sizes.
The tensor cores' own fp32 accumulation is not modelled here: the GPU
parity tests measure the kernels against the oracle. No CUDA and no oracle
are involved."""
import numpy as np
import pytest


def bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def from_bits(u):
    return np.asarray(u, dtype=np.uint32).view(np.float32)


def tf32_trunc(x):
    return from_bits(bits(x) & np.uint32(0xFFFFE000))


def tf32_round(x):  # nearest, ties away from zero
    return from_bits((bits(x) + np.uint32(0x1000)) & np.uint32(0xFFFFE000))


def bf16_trunc(x):
    return from_bits(bits(x) & np.uint32(0xFFFF0000))


def bf16_round(x):
    return from_bits((bits(x) + np.uint32(0x8000)) & np.uint32(0xFFFF0000))


def split_tf32(x):
    hi = tf32_trunc(x)
    r = (x - hi).astype(np.float32)  # exact: hi shares x's leading bits
    return hi, tf32_round(r), r


def split_bf16(x):
    p0 = bf16_trunc(x)
    r1 = (x - p0).astype(np.float32)
    p1 = bf16_trunc(r1)
    r2 = (r1 - p1).astype(np.float32)
    return p0, p1, bf16_round(r2), (r1, r2)


def sample(rng, n=200000):
    x = rng.normal(size=n) * np.exp2(rng.integers(-30, 30, size=n))
    return x.astype(np.float32)


def test_remainders_are_exact():
    x = sample(np.random.default_rng(1))
    x64 = x.astype(np.float64)
    hi, _, r = split_tf32(x)
    assert np.array_equal(hi.astype(np.float64) + r.astype(np.float64), x64)
    p0, p1, _, (r1, r2) = split_bf16(x)
    assert np.array_equal(p0.astype(np.float64) + r1.astype(np.float64), x64)
    assert np.array_equal(p1.astype(np.float64) + r2.astype(np.float64), r1.astype(np.float64))


def test_pieces_fit_their_formats():
    """tf32 pieces keep 10 stored significand bits, bf16 pieces 7."""
    x = sample(np.random.default_rng(2))
    hi, lo, _ = split_tf32(x)
    assert np.all(bits(hi) & np.uint32(0x1FFF) == 0) and np.all(bits(lo) & np.uint32(0x1FFF) == 0)
    p0, p1, p2, _ = split_bf16(x)
    for p in (p0, p1, p2):
        assert np.all(bits(p) & np.uint32(0xFFFF) == 0)


def test_representation_error_22_against_24_bits():
    """|x - sum of pieces| relative to |x|: at most 2^-22 for the tf32 pair
    (11 + 11 significant bits), zero for the bf16 triple (the last
    remainder has at most 8 significant bits, so its rounding is exact)."""
    x = sample(np.random.default_rng(3))
    x64 = x.astype(np.float64)
    hi, lo, _ = split_tf32(x)
    e_tf = np.max(np.abs(x64 - hi.astype(np.float64) - lo.astype(np.float64)) / np.abs(x64))
    p0, p1, p2, _ = split_bf16(x)
    e_bf = np.max(np.abs(x64 - p0.astype(np.float64) - p1.astype(np.float64) - p2.astype(np.float64)) / np.abs(x64))
    assert 2.0 ** -23 < e_tf <= 2.0 ** -22
    assert e_bf == 0.0


@pytest.mark.parametrize("k", [4, 5])
def test_kept_products_match_the_exact_product(k):
    """Dot products of length 2^(k+1) (the real form of a k-qubit gate's
    row) from the kept products only, summed exactly: the 3xTF32 result is
    within ~2^-23 of the row's scale sum |a w| (measured 2^-22.9 / 2^-23.2
    for k = 4 / 5), split-bf16 within ~2^-24 (2^-24.1 / 2^-24.8): the tf32
    operands' missing bits against the dropped bf16 products of weight
    2^-24 and below."""
    rng = np.random.default_rng(10 + k)
    K = 2 << k
    err_tf = err_bf = 0.0
    for _ in range(200):
        a = rng.normal(size=K).astype(np.float32)
        w = (rng.normal(size=K) / np.sqrt(K)).astype(np.float32)
        exact = float(np.dot(a.astype(np.float64), w.astype(np.float64)))
        scale = float(np.dot(np.abs(a.astype(np.float64)), np.abs(w.astype(np.float64))))
        ah, al, _ = split_tf32(a)
        wh, wl, _ = split_tf32(w)
        d = lambda u, v: float(np.dot(u.astype(np.float64), v.astype(np.float64)))
        tf = d(al, wh) + d(ah, wl) + d(ah, wh)
        pa, pw = split_bf16(a)[:3], split_bf16(w)[:3]
        bf = sum(d(pa[i], pw[j]) for i, j in ((2, 0), (1, 1), (0, 2), (1, 0), (0, 1), (0, 0)))
        err_tf = max(err_tf, abs(tf - exact) / scale)
        err_bf = max(err_bf, abs(bf - exact) / scale)
    assert err_tf < 2.0 ** -22
    assert err_bf < 2.0 ** -23.5
    assert err_bf < err_tf


def test_dropping_a_kept_product_would_show():
    """Planted mistake: 3xTF32 without its lo * hi term is no better than
    a single tf32 product (~2^-11)."""
    rng = np.random.default_rng(9)
    a = rng.normal(size=64).astype(np.float32)
    w = (rng.normal(size=64) / 8).astype(np.float32)
    exact = float(np.dot(a.astype(np.float64), w.astype(np.float64)))
    scale = float(np.dot(np.abs(a.astype(np.float64)), np.abs(w.astype(np.float64))))
    ah, al, _ = split_tf32(a)
    wh, wl, _ = split_tf32(w)
    d = lambda u, v: float(np.dot(u.astype(np.float64), v.astype(np.float64)))
    bad = d(ah, wl) + d(ah, wh)
    assert abs(bad - exact) / scale > 2.0 ** -16
