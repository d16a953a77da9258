// Double-float ("df") arithmetic for complex128 states on the FP32 pipe.
//
// GB300's FP64 units run at ~1/67 of the FP32 rate and FP64<->FP32
// conversions share that slow pipe, so complex128 gate arithmetic is done on
// unevaluated sums hi + lo of two floats (Dekker 1971; the error-free
// TwoSum of Knuth and the FMA-based TwoProduct), with the conversions to and
// from FP64 done by integer bit manipulation:
//   split  FP64 -> (hi, lo): hi keeps the top 24 significand bits; lo is the
//          next 23, formed as t - 2^(E-23) where t carries the same exponent
//          as the subtracted power of two (an exact FP32 subtraction).  The
//          six lowest bits are dropped: |x - hi - lo| < 2^-46 |x|.  Values
//          below 2^-100 in magnitude become 0 (an absolute error < 1e-30).
//   join   (hi, lo) -> FP64: the pair is renormalised (TwoSum) and both
//          significands are placed into one 53-bit integer significand.
//   mac    s += a * b in df: TwoProduct of the heads, the two cross terms by
//          FMA, TwoSum into the running head (~10 FP32 instructions).
// Relative error of a df product or sum is ~2^-46; a length-32 dot product
// stays near 2^-44, far inside the 1e-12 absolute tolerance of complex128.
// Magnitudes must stay below 2^120 (states and unitary matrices are <= 1).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace cast {
namespace df {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 split(double x) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
    const uint32_t sign = uint32_t(b >> 32) & 0x80000000u;
    const int e = int((b >> 52) & 0x7FF) - 1023;  // unbiased exponent
    F2 r;
    if (e < -100) {
        r.h = 0.f;
        r.l = 0.f;
        return r;
    }
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;  // 52 stored significand bits
    r.h = __uint_as_float(sign | (uint32_t(e + 127) << 23) | uint32_t(m >> 29));
    // t = +-1.m[28..6] * 2^(e-23); lo = t - (+-2^(e-23)) is exact
    const uint32_t te = uint32_t(e - 23 + 127);
    const float t = __uint_as_float(sign | (te << 23) | (uint32_t(m >> 6) & 0x7FFFFFu));
    const float p = __uint_as_float(sign | (te << 23));
    r.l = t - p;
    return r;
}

// hi + lo -> nearest-ish FP64 (truncating below 2^-53 relative).
__device__ __forceinline__ double join(float hi, float lo) {
    // renormalise (TwoSum) so that |l| <= ulp(s) / 2
    const float s = hi + lo;
    const float bb = s - hi;
    const float l = (hi - (s - bb)) + (lo - bb);
    const uint32_t hb = __float_as_uint(s);
    const int he = int((hb >> 23) & 0xFF);
    if (he == 0) return 0.0;  // |s| < 2^-126: negligible
    const uint64_t sign = uint64_t(hb & 0x80000000u) << 32;
    // significand of s as a 53-bit integer with the binary point after bit 52
    int64_t M = int64_t((hb & 0x7FFFFFu) | 0x800000u) << 29;
    const uint32_t lb = __float_as_uint(l);
    const int le = int((lb >> 23) & 0xFF);
    if (le != 0) {
        const int d = he - le;  // >= 23 after renormalisation
        int64_t ml = int64_t((lb & 0x7FFFFFu) | 0x800000u);
        ml = (d <= 29) ? (ml << (29 - d)) : (d - 29 < 63 ? (ml >> (d - 29)) : 0);
        M += ((lb ^ hb) & 0x80000000u) ? -ml : ml;
    }
    int E = he - 127 + 1023;
    // renormalise M into [2^52, 2^53)
    if (M >= (int64_t(1) << 53)) {
        M >>= 1;
        E += 1;
    } else {
        while (M < (int64_t(1) << 52) && M > 0) {
            M <<= 1;
            E -= 1;
        }
    }
    if (M <= 0) return 0.0;
    const uint64_t bits = sign | (uint64_t(E) << 52) | (uint64_t(M) & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double(static_cast<long long>(bits));
}

// s (head sh, tail sl) += a * b
__device__ __forceinline__ void mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float bb = s - sh;
    const float t = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += t + e;
}

// s -= a * b
__device__ __forceinline__ void msub(float &sh, float &sl, float ah, float al, float bh, float bl) {
    mac(sh, sl, -ah, -al, bh, bl);
}

// complex double-float: re = (rh, rl), im = (ih, il)
struct CF {
    float rh, rl, ih, il;
};

__device__ __forceinline__ CF split_c(double2 v) {
    const F2 a = split(v.x), b = split(v.y);
    CF c;
    c.rh = a.h;
    c.rl = a.l;
    c.ih = b.h;
    c.il = b.l;
    return c;
}

__device__ __forceinline__ double2 join_c(const CF &c) { return make_double2(join(c.rh, c.rl), join(c.ih, c.il)); }

// acc += u * x (complex)
__device__ __forceinline__ void cmac(CF &acc, const CF &u, const CF &x) {
    mac(acc.rh, acc.rl, u.rh, u.rl, x.rh, x.rl);
    msub(acc.rh, acc.rl, u.ih, u.il, x.ih, x.il);
    mac(acc.ih, acc.il, u.rh, u.rl, x.ih, x.il);
    mac(acc.ih, acc.il, u.ih, u.il, x.rh, x.rl);
}

}  // namespace df
}  // namespace cast
