// Host-side digit images of the complex128 digit-product kernels
// (apply_oz.cu): a gate's real form W split row by row into seven 7-bit
// digits, stored as bf16 in the 128-byte swizzled K-major shared-memory
// layout the tcgen05 B operand descriptors expect.  Host code only (no CUDA
// call), shared by the kernels' launchers and the host checks.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace cast {

constexpr int kOzImageDigits = 7;

// Seven 7-bit digits of |w| / 2^E (49 fractional bits, rounded to nearest,
// at most 2^49 - 1), E with every |w| of the row below 2^E.
inline void host_digits(double w, int E, int *dig) {
    const double f = std::nearbyint(std::ldexp(std::fabs(w), 49 - E));  // <= 2^49, exact
    uint64_t F = uint64_t(f);
    if (F >= (uint64_t(1) << 49)) F = (uint64_t(1) << 49) - 1;
    for (int j = kOzImageDigits - 1; j >= 0; j--) {
        dig[j] = int(F & 127u);
        F >>= 7;
    }
}

// digit a (0..127) of weight j as bf16, times 2^(-7j), with a sign
inline uint16_t host_bf16_digit(int a, int j, bool neg) {
    if (a == 0) return 0;
    const float f = std::ldexp(float(a), -7 * j);  // exact: 7 significant bits
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return uint16_t(u >> 16) | (neg ? 0x8000u : 0u);
}

// The digit image of a gate: W[n][c] (n output real, c input real = 2 member +
// part) is U's real form; row n gets exponent E_n (every |W[n][c]| < 2^E_n)
// and its entries' seven digits go to img at off(n, c, j) as bf16 with the
// sign of the entry (unit: the digit itself; else digit j times 2^(-7j));
// wexp[n] = E_n - 14.
template <class Off>
void build_digit_image(const PreparedGate &g, int k, std::vector<uint8_t> &img, int8_t *wexp, Off off, bool unit) {
    const int D = 1 << k, NR = 2 * D;
    std::vector<double> W(size_t(NR) * NR);
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++) {
            cplx u = g.m[size_t(r) * D + c];
            // parts below 2^-100 are dropped (they cannot reach an FP64 output
            // of a unit-scale row) so every row exponent fits the parameters
            if (std::fabs(u.real()) < 0x1p-100) u.real(0.0);
            if (std::fabs(u.imag()) < 0x1p-100) u.imag(0.0);
            W[size_t(2 * r) * NR + 2 * c] = u.real();
            W[size_t(2 * r) * NR + 2 * c + 1] = -u.imag();
            W[size_t(2 * r + 1) * NR + 2 * c] = u.imag();
            W[size_t(2 * r + 1) * NR + 2 * c + 1] = u.real();
        }
    for (int n = 0; n < NR; n++) {
        int E = -1022;
        for (int c = 0; c < NR; c++) {
            const double w = W[size_t(n) * NR + c];
            if (w != 0.0) {
                int e;
                std::frexp(w, &e);  // |w| in [2^(e-1), 2^e)
                E = std::max(E, e);
            }
        }
        wexp[n] = int8_t(std::max(-128, std::min(127, E - 14)));
        for (int c = 0; c < NR; c++) {
            const double w = W[size_t(n) * NR + c];
            int dig[kOzImageDigits];
            host_digits(w, E, dig);
            for (int j = 0; j < kOzImageDigits; j++) {
                const uint16_t b = host_bf16_digit(dig[j], unit ? 0 : j, w < 0);
                std::memcpy(img.data() + off(n, c, j), &b, 2);
            }
        }
    }
}

// 128-byte swizzled K-major image of rows of 64 bf16: row n (within its 8-row
// atoms), element c < 64: atom n/8, row n%8, 16-byte chunk (c/8) ^ (n%8)
inline size_t sw128_bf16(int n, int c) {
    return size_t(n >> 3) * 1024 + size_t(n & 7) * 128 + size_t(((c >> 3) ^ (n & 7)) << 4) + size_t(c & 7) * 2;
}

// k = 3..5: output half n / nhw, digit block j of nacc (the last stays zero),
// row n % nhw of the block
inline size_t oz_image_offset(int n, int c, int j, int nhw, int nacc) {
    return (size_t(n / nhw) * nacc + size_t(j)) * nhw * 128 + sw128_bf16(n % nhw, c);
}

// k = 6, 7: block (pass n / 64, K-block c / 64) of wblk bytes, digit j, row
// n % 64, element c % 64
inline size_t ozc_image_offset(int n, int c, int j, int nkb, size_t wblk) {
    return size_t((n >> 6) * nkb + (c >> 6)) * wblk + size_t(j) * 64 * 128 + sw128_bf16(n & 63, c & 63);
}

}  // namespace cast
