// Dense complex128 gates (k = 4, 5) on the tcgen05 tensor cores with an
// Ozaki-style split into exactly multiplied integer digits (Ozaki, Ogita and
// Oishi 2012; Ootomo, Ozaki and Yokota 2024 for the GPU form).
//
// Eq. 3's matvec for a tile of 128 slices is the real GEMM
//     Y (128 x 2D) = X (128 x 2D) * W^T,   D = 2^k,
// with X the slices' interleaved (re, im) parts and W the real form of U
// (2x2 blocks [[a, -b], [b, a]] for u = a + ib), as in the complex64 kernel.
//
// Splitting.  Each slice row r of X gets an exponent E_r with every |x| <
// 2^E_r; x / 2^E_r is rounded to 49 fractional bits (error at most
// 2^(E_r - 50), unbiased) and written as seven 7-bit digits, x = 2^E_r
// sum_i a_i 2^(-7(i+1)), a_i in [-127, 127] (all digits carry the sign of x).  Each
// output row n of W is split the same way with its own exponent E_n into
// digits w_j.  Digits are stored pre-scaled, a_i 2^(-7i) and w_j 2^(-7j),
// which bf16 represents exactly (7 significant bits times a power of two).
//
// Products.  For every pair (i, j) with i + j <= 7 one tcgen05.mma per
// K-step (kind::f16, bf16 operands, fp32 accumulation; A = digit i of X from
// tensor memory, B = digit j of W from shared memory) adds a_i w_j 2^(-7(i+j))
// into accumulator min(i + j, 5).  Accumulators d = 0..4 only ever hold
// integers times 2^(-7d) of magnitude below (d + 1) * 2D * 127^2 <= 5.2e6 <
// 2^24 (in units of 2^(-7d)), so they are exact in fp32 whatever the order
// of the additions or the rounding of the tensor cores; accumulator 5 gathers
// the products of weight 2^-35 and below, where the fp32 accumulation
// (it truncates, so its errors add up over the MMAs) costs about 2^-50 of
// the output.  The dropped pairs (i + j >= 8) are all of the sign of their
// product (every digit carries the sign of its value), so they shrink the
// outputs by ~2^-53; with i + j <= 6 only, that bias was 2^-46 and the norm
// of a state fell by 6.5e-12 over 200 gates.  Measured: a design that let
// weights 2^-21 and below share one inexact accumulator was 3.5e-12 off, one
// that let 2^-28 and below share it 1.8e-13 off (relative to the slice's
// scale), against 1.5e-13 for a 2^-28 common integer scale alone: both limits
// are gone here.
//
// Epilogue.  y = 2^(E_r + E_n - 14) (acc0 + ... + acc5): acc_d 2^(7d) for
// d <= 3 are converted to integers exactly (fp32 magic-number rounding of an
// exact integer below 2^22), acc4 * 2^28 (an exact integer below 2^24) and
// acc5 * 2^36 are converted with rounding, the six are summed in 64-bit
// integer arithmetic at the common scale 2^-36 and the result is written as
// an FP64 with integer operations (leading-zero count, shift, exponent), so no
// FP64 instruction runs on the device.
//
// Tensor memory holds the seven digits of A (D columns each, two bf16 per
// column) and six accumulators; for k = 4, 5 the outputs are produced in two
// halves of D columns (MMAs of half the N, then that half's epilogue) so that
// six accumulators fit beside the digits.
//
// Data path: four threads per slice row (TMEM lane),
// each with its share of the row's members.  A tile's 128 slice rows are
// loaded with 16-byte loads into shared memory ([member][row]); the parts'
// exponents meet in shared memory; each thread forms the digits of its members once per real
// and stores them to tensor memory with tcgen05.st; one thread issues the MMAs and
// commits them to an mbarrier; while they run, every thread loads the next
// tile into shared memory; the epilogue reads the four accumulators with
// tcgen05.ld and stores the outputs.  W's digits (host-built, already in the
// 128-byte-swizzled K-major shared-memory image) are copied in once per CTA.
// TMEM per CTA: 7 x D digit columns + 6 x 2D / NH accumulator columns (NH
// output halves): 152 / 208 / 416 for k = 3 / 4 / 5, so 2 / 2 / 1 CTAs per SM.
// Waits on the mbarrier are bounded (error flag, no trap).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "tc.cuh"

namespace cast {

int oz_error_flag_take();

namespace {

__device__ int g_oz_error;
std::atomic<int> g_c128_tc{CAST_C128_TC_OZAKI};
constexpr uint32_t kOzWait = 1u << 26;
constexpr int kDigits = 7;

template <int K>
struct OzShape {
    static constexpr int D = 1 << K;         // members per slice
    static constexpr int NR = 2 * D;         // reals per slice: GEMM K and N
    static constexpr int KS = NR / 16;       // MMA K-steps (16 bf16 each)
    static constexpr int DCOL = NR / 2;      // TMEM columns of one digit (two bf16 per column)
    static constexpr int NH = K >= 4 ? 2 : 1;  // output halves (MMA N >= 16)
    static constexpr int NHW = NR / NH;        // outputs per half = MMA N
    static constexpr int NACC = 6;
    static constexpr int ACOL0 = kDigits * DCOL;  // first accumulator column
    static constexpr int NCOL_USED = ACOL0 + NACC * NHW;
    static constexpr int NCOL = NCOL_USED <= 128 ? 128 : (NCOL_USED <= 256 ? 256 : 512);
    static constexpr int WBYTES = kDigits * NR * 128;  // W digits: N rows of 128 bytes per digit
    static constexpr int SBYTES = 128 * D * 16;        // staged tile: [member][row] double2
    // four threads per slice row: k = 4 two CTAs of 16 warps per SM (TMEM 2 x
    // 256 columns, 64 registers), k = 5 one CTA of 16 warps (416 columns)
    static constexpr int R = 4;
    static constexpr int NT = 128 * R;
    static constexpr int MIN_CTAS = K == 4 ? 2 : 1;
};

struct OzParams {
    int8_t wexp[64];  // E_n - 14 per output real n
};

// bf16 bit pattern of s * a * 2^(-7 i), a an integer in [0, 127]
__device__ __forceinline__ uint32_t digit_bf16(uint32_t a, int i, uint32_t sign) {
    const float f = (__uint_as_float(0x4B000000u | a) - 8388608.0f) * __uint_as_float(uint32_t(127 - 7 * i) << 23);
    return (__float_as_uint(f) >> 16) | (a ? (sign >> 16) : 0u);
}

// integer value of an fp32 holding an exact integer of magnitude < 2^22
__device__ __forceinline__ int32_t exact_int(float v) {
    return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// FP64 of Y * 2^e (Y an integer of magnitude < 2^62), by integer operations
__device__ __forceinline__ double i64_to_double(int64_t Y, int e) {
    if (Y == 0) return 0.0;
    const uint64_t sgn = Y < 0 ? (uint64_t(1) << 63) : 0;
    const uint64_t M = Y < 0 ? uint64_t(-Y) : uint64_t(Y);
    const int msb = 63 - __clzll((long long)M);
    const int ex = msb + e + 1023;
    if (ex <= 0) return 0.0;  // below 2^-1022: flushed
    const uint64_t frac = msb <= 52 ? (M << (52 - msb)) : (M >> (msb - 52));
    return __longlong_as_double((long long)(sgn | (uint64_t(ex) << 52) | (frac & 0xFFFFFFFFFFFFFull)));
}

template <int K>
__global__ void __launch_bounds__(OzShape<K>::NT, OzShape<K>::MIN_CTAS)
k_dense_oz(double2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg,
           const uint8_t *__restrict__ wimg, const __grid_constant__ OzParams P, uint32_t wait_limit) {
    using S = OzShape<K>;
    constexpr int D = S::D, NR = S::NR, NHW = S::NHW, NACC = S::NACC;
    constexpr int R = S::R, NT = S::NT;
    constexpr int DH = D / R;     // members of a row this thread handles
    constexpr int OH = NHW / R;   // outputs of an output half this thread finishes
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sW = base;                                              // W digits (1024-aligned)
    double2 *stg = reinterpret_cast<double2 *>(sW + S::WBYTES);      // [member][row]
    int *sE = reinterpret_cast<int *>(stg + 128 * D);                // [part][row] partial exponents
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sE + NT);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, half = tid >> 7;  // slice row = TMEM lane; members [half * DH, half * DH + DH)
                                                 // (half: this thread's part of the row, 0..R-1)

    for (int i = tid; i < S::WBYTES / 16; i += NT)
        reinterpret_cast<uint4 *>(sW)[i] = __ldg(reinterpret_cast<const uint4 *>(wimg) + i);
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, S::NCOL);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t lane_addr = taddr + (uint32_t(32 * (warp & 3)) << 16);

    uint64_t p[K];
#pragma unroll
    for (int i = 0; i < K; i++) p[i] = uint64_t(1) << tg.q[i];
    auto member_off = [&](int j) {
        uint64_t off = 0;
#pragma unroll
        for (int i = 0; i < K; i++)
            if ((j >> i) & 1) off += p[i];
        return off;
    };
    auto load_tile = [&](uint64_t t) {
        const uint64_t b = slice_base<K>(t * 128 + row, tg);
#pragma unroll
        for (int jj = 0; jj < DH; jj++) {
            const int j = half * DH + jj;
            stg[j * 128 + row] = __ldcs(sv + b + member_off(j));
        }
    };

    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NHW >> 3) << 17) | (uint32_t(128 >> 4) << 24);
    const uint32_t wbase = tc::smem_u32(sW);
    uint32_t phase = 0;
    bool failed = false;
    uint64_t tile = blockIdx.x;
    if (tile < ntiles) load_tile(tile);
    while (tile < ntiles) {
        // ---- row exponent: both halves' maxima
        int eh = -1022;
#pragma unroll
        for (int jj = 0; jj < DH; jj++) {
            const double2 v = stg[(half * DH + jj) * 128 + row];
            const int e0 = int((__double_as_longlong(v.x) >> 52) & 0x7FF), e1 = int((__double_as_longlong(v.y) >> 52) & 0x7FF);
            eh = max(eh, max(e0, e1) - 1022);
        }
        sE[half * 128 + row] = eh;
        __syncthreads();
        int er = sE[row];
#pragma unroll
        for (int r = 1; r < R; r++) er = max(er, sE[r * 128 + row]);
        // ---- digits of this thread's members, in chunks of (up to) 8 members
        constexpr int CH = DH < 8 ? DH : 8;
#pragma unroll
        for (int c0 = 0; c0 < DH; c0 += CH) {
            uint64_t F[2 * CH];  // fixed-point magnitudes, 49 fractional bits below 2^er
            uint32_t sg[2 * CH];
#pragma unroll
            for (int c = 0; c < CH; c++) {
                const double2 x = stg[(half * DH + c0 + c) * 128 + row];
#pragma unroll
                for (int part = 0; part < 2; part++) {
                    const uint64_t bits = uint64_t(__double_as_longlong(part ? x.y : x.x));
                    const int e = int((bits >> 52) & 0x7FF);
                    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (uint64_t(1) << 52);
                    const int sh = 4 + (er - (e - 1022));
                    // nearest 49-bit fraction (unbiased: truncation would shrink every
                    // product and the error would build up over a circuit); a value
                    // that rounds up to 2^er keeps the largest fraction below it
                    const uint64_t f = (e == 0 || sh >= 54) ? 0 : ((m >> (sh - 1)) + 1) >> 1;
                    F[2 * c + part] = f < (uint64_t(1) << 49) ? f : (uint64_t(1) << 49) - 1;
                    sg[2 * c + part] = uint32_t(bits >> 32) & 0x80000000u;
                }
            }
#pragma unroll
            for (int i = 0; i < kDigits; i++) {
                float v[CH];
                const int sh = 7 * (kDigits - 1 - i);
#pragma unroll
                for (int c = 0; c < CH; c++) {
                    const uint32_t a0 = uint32_t(F[2 * c] >> sh) & 127u, a1 = uint32_t(F[2 * c + 1] >> sh) & 127u;
                    v[c] = __uint_as_float(digit_bf16(a0, i, sg[2 * c]) | (digit_bf16(a1, i, sg[2 * c + 1]) << 16));
                }
                tc::tmem_st<CH>(lane_addr + uint32_t(i * S::DCOL + half * DH + c0), v);
            }
        }
        tc::tmem_wait_st();
        tc::fence_before_sync();
        if (__syncthreads_or(failed)) break;
        tc::fence_after_sync();
        const uint64_t next = tile + gridDim.x;
        const int er_cur = er;
        const uint64_t ob = slice_base<K>(tile * 128 + row, tg);
#pragma unroll
        for (int h = 0; h < S::NH; h++) {
            if (tid == 0) {
                bool first[NACC];
#pragma unroll
                for (int d = 0; d < NACC; d++) first[d] = true;
#pragma unroll
                for (int d = 0; d < NACC; d++) {
#pragma unroll
                    for (int i = 0; i < kDigits; i++) {
#pragma unroll
                        for (int j = 0; j < kDigits && i + j <= kDigits; j++) {
                            if ((i + j < NACC - 1 ? i + j : NACC - 1) != d) continue;
#pragma unroll
                            for (int ks = 0; ks < S::KS; ks++) {
                                const uint64_t bdesc =
                                    tc::smem_desc_sw128(wbase + uint32_t(j * NR * 128 + h * NHW * 128 + ks * 32));
                                const uint32_t a = taddr + uint32_t(i * S::DCOL + ks * 8);
                                const uint32_t dcol = taddr + uint32_t(S::ACOL0 + d * NHW);
                                const uint32_t acc = first[d] ? 0u : 1u;
                                asm volatile(
                                    "{\n\t.reg .pred pp;\n\tsetp.ne.b32 pp, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pp;\n\t}" ::"r"(dcol),
                                    "r"(a), "l"(bdesc), "r"(idesc), "r"(acc));
                                first[d] = false;
                            }
                        }
                    }
                }
                tc::mma_commit(mbar);
            }
            __syncwarp();
            if (h == 0) {
                // ---- the next tile's loads run while the MMAs execute
                __syncthreads();  // every thread has read the staged tile and the exponents
                if (next < ntiles) load_tile(next);
            }
            failed = __syncthreads_or(!tc::mbar_wait(mbar, phase, wait_limit));  // agreed by all threads
            if (failed) break;
            phase ^= 1u;
            tc::fence_after_sync();
            // ---- epilogue of outputs [h NHW + half OH, + OH): y = 2^(E_r + E_n - 14) (acc0 + ... + acc5)
            constexpr int EC = OH < 16 ? OH : 16;
#pragma unroll
            for (int n0 = 0; n0 < OH; n0 += EC) {
                const int col = half * OH + n0;  // within this output half
                float ac[NACC][EC];
#pragma unroll
                for (int d = 0; d < NACC; d++) tc::tmem_ld<EC>(lane_addr + uint32_t(S::ACOL0 + d * NHW + col), ac[d]);
#pragma unroll
                for (int m = 0; m < EC / 2; m++) {
                    double out[2];
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        const int c = 2 * m + hh;
                        // common scale 2^-36 (in units of the weight-0 products)
                        const int64_t Y = (int64_t(exact_int(ac[0][c])) << 36) +
                                          (int64_t(exact_int(ac[1][c] * 128.0f)) << 29) +
                                          (int64_t(exact_int(ac[2][c] * 16384.0f)) << 22) +
                                          (int64_t(exact_int(ac[3][c] * 2097152.0f)) << 15) +
                                          (int64_t(__float2int_rn(ac[4][c] * 268435456.0f)) << 8) +
                                          int64_t(__float2int_rn(ac[5][c] * 68719476736.0f));
                        out[hh] = i64_to_double(Y, er_cur + int(P.wexp[h * NHW + col + c]) - 36);
                    }
                    const int j = ((h * NHW + col) >> 1) + m;
                    __stcs(sv + ob + member_off(j), make_double2(out[0], out[1]));
                }
            }
            tc::fence_before_sync();
            __syncthreads();  // the accumulators are read before the next MMAs overwrite them
            tc::fence_after_sync();
        }
        if (failed) break;
        tc::fence_before_sync();
        tile = next;
    }
    failed = __syncthreads_or(failed);
    if (failed) {
        if (tid == 0) {
            atomicOr(&g_oz_error, 1);
            tc::mbar_wait(mbar, phase, wait_limit);  // an MMA in flight finishes before TMEM is freed
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, S::NCOL);
}

// ----------------------------------------------------------------- host side
// Seven 7-bit digits of |w| / 2^E (49 fractional bits, rounded to nearest,
// at most 2^49 - 1), E with every |w| of the row below 2^E.
void host_digits(double w, int E, int *dig) {
    const double f = std::nearbyint(std::ldexp(std::fabs(w), 49 - E));  // <= 2^49, exact
    uint64_t F = uint64_t(f);
    if (F >= (uint64_t(1) << 49)) F = (uint64_t(1) << 49) - 1;
    for (int j = kDigits - 1; j >= 0; j--) {
        dig[j] = int(F & 127u);
        F >>= 7;
    }
}

uint16_t host_bf16_digit(int a, int j, bool neg) {
    if (a == 0) return 0;
    const float f = std::ldexp(float(a), -7 * j);  // exact: 7 significant bits
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return uint16_t(u >> 16) | (neg ? 0x8000u : 0u);
}

template <int K>
cast_status run_oz(cast_sv *sv, const PreparedGate &g) {
    using S = OzShape<K>;
    constexpr int D = S::D, NR = S::NR;
    // real form W[n][c]: n output real, c input real (2 member + part)
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
    OzParams P{};
    std::vector<uint8_t> img(S::WBYTES, 0);
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
        P.wexp[n] = int8_t(std::max(-128, std::min(127, E - 14)));
        for (int c = 0; c < NR; c++) {
            const double w = W[size_t(n) * NR + c];
            int dig[kDigits];
            host_digits(w, E, dig);
            for (int j = 0; j < kDigits; j++) {
                const uint16_t b = host_bf16_digit(dig[j], j, w < 0);
                // 128-byte swizzled K-major: atom n/8, row n%8, 16-byte chunk (c/8) ^ (n%8)
                const size_t off = size_t(j) * NR * 128 + size_t(n >> 3) * 1024 + size_t(n & 7) * 128 +
                                   size_t(((c >> 3) ^ (n & 7)) << 4) + size_t(c & 7) * 2;
                std::memcpy(img.data() + off, &b, 2);
            }
        }
    }
    const void *dev = nullptr;
    cast_status st = upload_matrix(sv, img.data(), img.size(), &dev);
    if (st != CAST_OK) return st;
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const size_t smem = 1024 + S::WBYTES + S::SBYTES + S::NT * 4 + 64;
    CAST_CUDA(cudaFuncSetAttribute(k_dense_oz<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = 512 / S::NCOL;
    const uint64_t cap = uint64_t(sm_count_cached()) * per_sm;
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    const double N = double(uint64_t(1) << sv->n);
    ProfScope ps(sv->stream, "ozdense_k" + std::to_string(K) + "_c128", 32.0 * N, 8.0 * N * double(D));
    k_dense_oz<K><<<(unsigned)grid, S::NT, smem, sv->stream>>>(reinterpret_cast<double2 *>(sv->data), ntiles, tg,
                                                             static_cast<const uint8_t *>(dev), P, kOzWait);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool oz_eligible(const cast_sv *sv, const PreparedGate &g) {
    if (g_c128_tc.load() != CAST_C128_TC_OZAKI || f64_mode() != CAST_F64_EMULATED || sv->dt != CAST_C128 ||
        g.cls != CLS_DENSE || g.k < 4 || g.k > 5 || sv->n < g.k + 7)
        return false;
    // measured per 30-qubit gate: this kernel 22-23 ms (k = 4) and 32-38 ms
    // (k = 5) whatever the matrix; the sparse kernel 10-12 / 11-20 ms at 10-30%
    // density and 35 / 62-69 ms dense: the digit kernel takes the gates above
    // 60% of the dense operation count (k = 3 gates stay on the CUDA cores,
    // where the sparse and dense double-float kernels match it)
    return 5 * opcount(g.m.data(), g.k, 0.0) > 3 * dense_opcount(g.k);
}

cast_status launch_gate_oz(cast_sv *sv, const PreparedGate &g) {
    switch (g.k) {
        case 4: return run_oz<4>(sv, g);
        case 5: return run_oz<5>(sv, g);
        default: return fail(CAST_ERR_UNSUPPORTED, "tensor-core complex128 path covers k = 4, 5");
    }
}

int oz_error_flag_take() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_oz_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_oz_error, &zero, sizeof(int));
    }
    return v;
}

}  // namespace cast

extern "C" {

cast_status cast_set_c128_tensor_mode(int mode) {
    if (mode != CAST_C128_TC_OFF && mode != CAST_C128_TC_OZAKI)
        return cast::fail(CAST_ERR_ARG, "unknown complex128 tensor-core mode");
    cast::g_c128_tc = mode;
    return CAST_OK;
}

int cast_get_c128_tensor_mode(void) { return cast::g_c128_tc.load(); }

}  // extern "C"
