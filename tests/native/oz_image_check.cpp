// Host-logic check of the complex128 digit images (oz_image.h): for random
// complex matrices of k = 3..7 (entries spread over 40 binades, some purely
// real, some with parts below 2^-100), in the k = 3..5 layout (with integer
// and with pre-scaled digits) and the k = 6, 7 block layout:
//   - every (output real n, input real c, digit j) lands at its own offset
//     inside the image, and every other byte stays zero (the zero digit
//     block 7 of the k = 3..5 layout included);
//   - the seven bf16 digits of an entry, weighted 2^(E_n - 7(j+1)), give back
//     the entry of the real form to within 2^(E_n - 49), E_n = wexp[n] + 14
//     bounding the row (flushed parts below 2^-100 excepted);
//   - every digit is an integer 0..127 (times 2^(-7j) when pre-scaled) with
//     the sign of its entry.
// Prints the counts; exit status 1 on a mismatch.
#include <cstdint>
#include <cstdio>
#include <random>
#include <set>
#include <vector>
#include "oz_image.h"
using namespace cast;

static double bf16_value(const uint8_t *p) {
    uint16_t h;
    std::memcpy(&h, p, 2);
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int main() {
    std::mt19937_64 rng(23);
    std::normal_distribution<double> nd;
    long bad = 0, entries = 0, images = 0;
    for (int k = 3; k <= 7; k++)
        for (int trial = 0; trial < 12; trial++) {
            const int D = 1 << k, NR = 2 * D;
            PreparedGate g;
            g.k = k;
            g.m.resize(size_t(D) * D);
            for (auto &x : g.m) {
                const double s = std::ldexp(1.0, int(rng() % 40) - 30);
                x = cplx(nd(rng) * s, trial % 3 == 0 ? 0.0 : nd(rng) * s);
                if (trial % 4 == 1 && rng() % 8 == 0) x = cplx(1e-31, x.imag());  // flushed part
            }
            std::vector<double> W(size_t(NR) * NR);
            for (int r = 0; r < D; r++)
                for (int c = 0; c < D; c++) {
                    cplx u = g.m[size_t(r) * D + c];
                    if (std::fabs(u.real()) < 0x1p-100) u.real(0.0);
                    if (std::fabs(u.imag()) < 0x1p-100) u.imag(0.0);
                    W[size_t(2 * r) * NR + 2 * c] = u.real();
                    W[size_t(2 * r) * NR + 2 * c + 1] = -u.imag();
                    W[size_t(2 * r + 1) * NR + 2 * c] = u.imag();
                    W[size_t(2 * r + 1) * NR + 2 * c + 1] = u.real();
                }
            for (int form = 0; form < 3; form++) {  // 0, 1: k <= 5 layout, unit / scaled; 2: k = 6, 7 layout
                if ((form < 2) != (k <= 5)) continue;
                const bool unit = form == 0;
                const int nh = k >= 4 ? 2 : 1, nhw = NR / nh, nkb = NR / 64;
                const size_t wblk = size_t(kOzImageDigits) * 64 * 128;
                const size_t bytes = form < 2 ? size_t(nh) * 8 * nhw * 128 : size_t(NR / 64) * nkb * wblk;
                auto off = [&](int n, int c, int j) {
                    return form < 2 ? oz_image_offset(n, c, j, nhw, 8) : ozc_image_offset(n, c, j, nkb, wblk);
                };
                std::vector<uint8_t> img(bytes, 0);
                int8_t wexp[256];
                build_digit_image(g, k, img, wexp, off, unit);
                images++;
                std::vector<char> used(bytes, 0);
                for (int n = 0; n < NR; n++) {
                    const int E = wexp[n] + 14;
                    for (int c = 0; c < NR; c++) {
                        const double w = W[size_t(n) * NR + c];
                        if (std::fabs(w) >= std::ldexp(1.0, E)) bad++;  // E bounds the row
                        double recon = 0.0;
                        for (int j = 0; j < kOzImageDigits; j++) {
                            const size_t o = off(n, c, j);
                            if (o + 2 > bytes || used[o] || used[o + 1]) { bad++; continue; }
                            used[o] = used[o + 1] = 1;
                            const double v = bf16_value(&img[o]);
                            const double a = unit ? v : std::ldexp(v, 7 * j);  // the digit itself
                            if (a != std::trunc(a) || std::fabs(a) > 127 || (a != 0 && (a < 0) != (w < 0))) bad++;
                            recon += std::ldexp(a, E - 7 * (j + 1));
                        }
                        if (std::fabs(recon - w) > std::ldexp(1.0, E - 49)) bad++;
                        entries++;
                    }
                }
                for (size_t o = 0; o < bytes; o++)
                    if (!used[o] && img[o] != 0) bad++;
            }
        }
    printf("images=%ld entries=%ld bad=%ld\n", images, entries, bad);
    return bad ? 1 : 0;
}
