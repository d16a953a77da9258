// Dense complex128 gates (k = 3..7) on the tcgen05 tensor cores with an
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
// digits w_j.  For k = 3..5 the digits are stored as the integers a_i, w_j
// themselves, for k = 6, 7 pre-scaled, a_i 2^(-7i) and w_j 2^(-7j); bf16
// represents both exactly (7 significant bits times a power of two).
//
// Products.  Every pair (i, j) with i + j <= 7 contributes a_i w_j
// (weight 2^(-7(i+j))) to accumulator d = i + j (eight accumulators, d = 0..7).  For a
// fixed digit i of X the weights i + j of j = 0, 1, ... are consecutive, so
// with the B blocks of W's digits stacked (rows of digit 0, then digit 1, ...)
// and the accumulators in adjacent TMEM columns, one tcgen05.mma per (i,
// K-step) (kind::f16, bf16 operands, fp32 accumulation; A = digit i of X from
// tensor memory, B = the stacked digits of W from shared memory, N' = blocks x
// N) adds all of digit i's pairs at once: 7 MMAs per K-step instead of 34.
// The MMA of i = 0 also covers a zero eighth block, so it starts every
// accumulator.  (Measured on GB300 with cast_measure_mma_issue: an M = 128,
// K = 16 bf16 MMA costs 49.5 cycles for any N <= 64, 64 at N = 128 and 128 at
// N = 256, the last two at the bf16 peak.)  Accumulator d only
// ever holds integers (times 2^(-7d) when pre-scaled) of magnitude below (pairs of weight d) *
// 2D * 127^2 <= 7 * 64 * 16129 < 2^23 (k <= 5), so all eight are exact in fp32
// whatever the order of the additions or the rounding of the tensor cores.
// The dropped pairs (i + j >= 8) are all of the sign of their product (every
// digit carries the sign of its value), so they shrink the outputs by
// ~2^-53; with i + j <= 6 only, that bias was 2^-46 and the norm of a state
// fell by 6.5e-12 over 200 gates.  Measured: a design that let weights 2^-21
// and below share one inexact accumulator was 3.5e-12 off, one that let
// 2^-28 and below share it 1.8e-13 off (relative to the slice's scale),
// against 1.5e-13 for a 2^-28 common integer scale alone: both limits are
// gone here.
//
// Epilogue.  y = 2^(E_r + E_n - 14) sum_d acc_d 2^(-7d), summed at the
// common scale 2^-36 (in units of the weight-0 products): acc_d for d <= 3
// are converted to integers exactly (fp32 magic-number rounding of an exact
// integer below 2^22) and paired in 32 bits (acc0 * 2^7 + acc1, acc2 * 2^7 +
// acc3); acc4 (an exact integer below 2^23) with the conversion instruction,
// times 2^8, plus acc5 * 2 + acc6 * 2^-6 + acc7 * 2^-13 summed in fp32 (two
// roundings of at most half a unit at 2^-36) and converted once; the three
// parts are summed in 64-bit integer arithmetic and the result is written as
// an FP64 with integer operations (leading-zero count, shift, exponent), so
// no FP64 instruction runs on the device.
//
// Tensor memory holds the seven digits of A (D columns each, two bf16 per
// column) and the eight accumulators; for k = 4, 5 the outputs are produced
// in two halves of D columns (MMAs of half the N, then that half's epilogue)
// so that eight accumulators fit beside the digits.
//
// Data path: four threads per slice row (TMEM lane),
// each with its share of the row's members.  A tile's 128 slice rows are
// copied with 16-byte cp.async into shared memory ([member][row]); the parts'
// exponents meet in shared memory; each thread forms the digits of its members once per real
// and stores them to tensor memory with tcgen05.st; one thread issues the MMAs and
// commits them to an mbarrier; while they run, every thread loads the next
// tile into shared memory (cp.async, waited for at the next tile by the
// thread that issued it, the only one that reads it); the epilogue reads the eight accumulators with
// tcgen05.ld and stores the outputs.  W's digits (host-built, already in the
// 128-byte-swizzled K-major shared-memory image) are copied in once per CTA.
// TMEM per CTA: 7 x D digit columns + 8 x 2D / NH accumulator columns (NH
// output halves): 184 / 240 / 480 for k = 3 / 4 / 5, so 2 / 2 / 1 CTAs per SM.
// Waits on the mbarrier are bounded (error flag, no trap).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "oz_image.h"
#include "tc.cuh"

namespace cast {

int oz_error_flag_take();

namespace {

__device__ int g_oz_error;
std::atomic<int> g_c128_tc{CAST_C128_TC_OZAKI};
constexpr uint32_t kOzWait = 1u << 26;
constexpr int kDigits = 7;
static_assert(kDigits == kOzImageDigits, "the kernels and the host image agree on the digit count");
// Measured per 30-qubit gate on a random state (mean of low, high and mixed
// targets, k = 3 / 4 / 5): 17.6 / 17.3 / 22.6 ms with none of the four
// options below, 14.7 / 14.6 / 17.6 ms with the first three, 14.2 / 14.1 /
// 16.3 ms with all four.
// k = 3..5: the next tile's loads as cp.async (the threads go on to the
// epilogue while they land) instead of loads into registers: 15.4 / 15.4 /
// 18.6 ms alone
constexpr bool kOzAsyncLoad = true;
// k = 3..5: digits stored as the plain integers a_i, w_j (the weights 2^(-7d)
// applied in the epilogue's integer shifts) instead of pre-scaled: 16.6 /
// 16.5 / 22.0 ms alone
constexpr bool kOzUnitDigits = true;
// k = 3..5 with unit digits: the weights d = 5, 6, 7 summed in fp32 before
// one conversion instead of three (16.5 / 16.3 / 21.6 ms with unit digits)
constexpr bool kOzSumLow = true;
// k = 3..5: two CTA barriers per tile left out. The one before the next
// tile's loads guarded nothing (each thread reloads only the staged rows it
// read itself, and the exponents are read before the MMA barrier); the one
// after the last output half's epilogue is implied by the next tile's
// barriers, which every thread reaches only after its epilogue.
constexpr bool kOzFewBarriers = true;

template <int K>
struct OzShape {
    static constexpr int D = 1 << K;         // members per slice
    static constexpr int NR = 2 * D;         // reals per slice: GEMM K and N
    static constexpr int KS = NR / 16;       // MMA K-steps (16 bf16 each)
    static constexpr int DCOL = NR / 2;      // TMEM columns of one digit (two bf16 per column)
    static constexpr int NH = K >= 4 ? 2 : 1;  // output halves (MMA N >= 16)
    static constexpr int NHW = NR / NH;        // outputs per half = MMA N
    static constexpr int NACC = 8;                // one per digit weight d = i + j, 0..7
    static constexpr int ACOL0 = kDigits * DCOL;  // first accumulator column
    static constexpr int NCOL_USED = ACOL0 + NACC * NHW;
    static constexpr int NCOL = NCOL_USED <= 128 ? 128 : (NCOL_USED <= 256 ? 256 : 512);
    // W digits per output half: blocks j = 0..7 of NHW rows x 128 bytes (block 7 zero)
    static constexpr int WBYTES = NH * NACC * NHW * 128;
    static constexpr int SBYTES = 128 * D * 16;        // staged tile: [member][row] double2
    // four threads per slice row: k = 4 two CTAs of 16 warps per SM (TMEM 2 x
    // 256 columns, 64 registers), k = 5 one CTA of 16 warps (416 columns)
    static constexpr int R = 4;
    static constexpr int NT = 128 * R;
    static constexpr int MIN_CTAS = K <= 4 ? 2 : 1;
};

struct OzParams {
    int8_t wexp[64];  // E_n - 14 per output real n
};

// x / 2^er rounded to 49 fractional bits, as a magnitude F < 2^49, and the
// fp32 magic number +-2^23 carrying the sign of x
struct Fixed49 {
    uint64_t f;
    uint32_t mg;
};
__device__ __forceinline__ Fixed49 fixed49(double x, int er) {
    const uint64_t bits = uint64_t(__double_as_longlong(x));
    const int e = int((bits >> 52) & 0x7FF);
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (uint64_t(1) << 52);
    const int sh = 4 + (er - (e - 1022));
    // nearest (unbiased; truncation would shrink every product and the error
    // would build up over a circuit); a value that rounds up to 2^er keeps
    // the largest fraction below it
    uint64_t f = (e == 0 || sh >= 54) ? 0 : ((m >> (sh - 1)) + 1) >> 1;
    f = f < (uint64_t(1) << 49) ? f : (uint64_t(1) << 49) - 1;
    return {f, (uint32_t(bits >> 32) & 0x80000000u) | 0x4B000000u};
}
// digit i of v as the float +-a_i 2^(-7i): +-(2^23 + a) - (+-2^23) = +-a
// exactly, then an exact power-of-two scale; its top half is the bf16 digit
__device__ __forceinline__ float digit_f(const Fixed49 &v, int i) {
    const uint32_t a = uint32_t(v.f >> (7 * (kDigits - 1 - i))) & 127u;
    return (__uint_as_float(v.mg | a) - __uint_as_float(v.mg)) * __uint_as_float(uint32_t(127 - 7 * i) << 23);
}
// digit i of v as the float +-a_i (exact)
__device__ __forceinline__ float digit_u(const Fixed49 &v, int i) {
    const uint32_t a = uint32_t(v.f >> (7 * (kDigits - 1 - i))) & 127u;
    return __uint_as_float(v.mg | a) - __uint_as_float(v.mg);
}
// two such floats as one TMEM column of bf16 (lo: a, hi: b)
__device__ __forceinline__ float bf16_pair(float a, float b) {
    return __uint_as_float(__byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632));
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
           const uint8_t *__restrict__ wimg, const __grid_constant__ OzParams P, uint32_t wait_limit,
           int skip_mma) {
    using S = OzShape<K>;
    constexpr int D = S::D, NHW = S::NHW, NACC = S::NACC;
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
            if constexpr (kOzAsyncLoad)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(stg + j * 128 + row)),
                             "l"(sv + b + member_off(j))
                             : "memory");
            else
                stg[j * 128 + row] = __ldcs(sv + b + member_off(j));
        }
        if constexpr (kOzAsyncLoad) asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // kind::f16 with D fp32, A and B bf16, M = 128 (N set per MMA)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(128 >> 4) << 24);
    const uint32_t wbase = tc::smem_u32(sW);
    uint32_t phase = 0;
    bool failed = false;
    uint64_t tile = blockIdx.x;
    if (tile < ntiles) load_tile(tile);
    while (tile < ntiles) {
        // this thread's own copies of the tile (it reads only what it loaded)
        if constexpr (kOzAsyncLoad) asm volatile("cp.async.wait_all;" ::: "memory");
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
            Fixed49 F[2 * CH];
#pragma unroll
            for (int c = 0; c < CH; c++) {
                const double2 x = stg[(half * DH + c0 + c) * 128 + row];
                F[2 * c] = fixed49(x.x, er);
                F[2 * c + 1] = fixed49(x.y, er);
            }
#pragma unroll
            for (int i = 0; i < kDigits; i++) {
                float v[CH];
#pragma unroll
                for (int c = 0; c < CH; c++) {
                    if constexpr (kOzUnitDigits)
                        v[c] = bf16_pair(digit_u(F[2 * c], i), digit_u(F[2 * c + 1], i));
                    else
                        v[c] = bf16_pair(digit_f(F[2 * c], i), digit_f(F[2 * c + 1], i));
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
            // (skip_mma: failure-detection test hook, no MMA and no commit, so
            // every thread's bounded wait below runs out)
            if (tid == 0 && !skip_mma) {
                // one MMA per (A digit i, K-step): the B blocks of digits j = 0.. are
                // stacked rows, and the accumulators of weights d = i + j adjacent
                // columns, so N' = (blocks) x NHW covers accumulators i..7 at once.
                // i = 0 also takes the zero block 7 and so starts every accumulator.
#pragma unroll
                for (int ks = 0; ks < S::KS; ks++) {
#pragma unroll
                    for (int i = 0; i < kDigits; i++) {
                        const int nblk = i == 0 ? NACC : NACC - i;
                        const uint32_t idesc_i = idesc | (uint32_t((nblk * NHW) >> 3) << 17);
                        const uint64_t bdesc =
                            tc::smem_desc_sw128(wbase + uint32_t(h * NACC * NHW * 128 + ks * 32));
                        const uint32_t a = taddr + uint32_t(i * S::DCOL + ks * 8);
                        const uint32_t dcol = taddr + uint32_t(S::ACOL0 + i * NHW);
                        const uint32_t acc = (ks == 0 && i == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred pp;\n\tsetp.ne.b32 pp, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pp;\n\t}" ::"r"(dcol),
                            "r"(a), "l"(bdesc), "r"(idesc_i), "r"(acc));
                    }
                }
                tc::mma_commit(mbar);
            }
            __syncwarp();
            if (h == 0) {
                // ---- the next tile's loads run while the MMAs execute
                if constexpr (!kOzFewBarriers) __syncthreads();
                if (next < ntiles) load_tile(next);
            }
            failed = __syncthreads_or(!tc::mbar_wait(mbar, phase, wait_limit));  // agreed by all threads
            if (failed) break;
            phase ^= 1u;
            tc::fence_after_sync();
            // ---- epilogue of outputs [h NHW + half OH, + OH): y = 2^(E_r + E_n - 14) (acc0 + ... + acc7)
            constexpr int EC = OH < 4 ? OH : 4;
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
                        // common scale 2^-36 (in units of the weight-0 products): acc_d
                        // 2^(7d) is an exact integer for every d; those of d <= 5 stay
                        // exact at this scale, d = 6, 7 round to it
                        int64_t Y;
                        if constexpr (kOzUnitDigits) {
                            // acc_d holds the integer sum itself; pairs of
                            // terms that fit 32 bits are combined first
                            const int32_t hi = exact_int(ac[0][c]) * 128 + exact_int(ac[1][c]);
                            const int32_t mid = exact_int(ac[2][c]) * 128 + exact_int(ac[3][c]);
                            int32_t lo = __float2int_rn(ac[4][c]) * 256;  // |acc4| < 5 * 64 * 127^2 < 2^23
                            if constexpr (kOzSumLow)
                                lo += __float2int_rn(fmaf(ac[7][c], 0x1p-13f, fmaf(ac[6][c], 0x1p-6f, 2.0f * ac[5][c])));
                            else
                                lo += __float2int_rn(ac[5][c]) * 2 + __float2int_rn(ac[6][c] * 0x1p-6f) +
                                      __float2int_rn(ac[7][c] * 0x1p-13f);
                            Y = (int64_t(hi) << 29) + (int64_t(mid) << 15) + int64_t(lo);
                        } else {
                            Y = (int64_t(exact_int(ac[0][c])) << 36) + (int64_t(exact_int(ac[1][c] * 128.0f)) << 29) +
                                (int64_t(exact_int(ac[2][c] * 16384.0f)) << 22) +
                                (int64_t(exact_int(ac[3][c] * 2097152.0f)) << 15) +
                                (int64_t(__float2int_rn(ac[4][c] * 268435456.0f)) << 8) +
                                int64_t(__float2int_rn(ac[5][c] * 68719476736.0f)) +
                                int64_t(__float2int_rn(ac[6][c] * 68719476736.0f)) +
                                int64_t(__float2int_rn(ac[7][c] * 68719476736.0f));
                        }
                        out[hh] = i64_to_double(Y, er_cur + int(P.wexp[h * NHW + col + c]) - 36);
                    }
                    const int j = ((h * NHW + col) >> 1) + m;
                    __stcs(sv + ob + member_off(j), make_double2(out[0], out[1]));
                }
            }
            tc::fence_before_sync();
            // the accumulators are read before the next MMAs overwrite them (the
            // next tile's MMAs wait at that tile's barriers)
            if (!kOzFewBarriers || h + 1 < S::NH) __syncthreads();
            tc::fence_after_sync();
        }
        if (failed) break;
        tc::fence_before_sync();
        tile = next;
    }
    if constexpr (kOzAsyncLoad) asm volatile("cp.async.wait_all;" ::: "memory");
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

// ------------------------------------------------------------ k = 6, 7
// The same digit products with K fed in chunks.  The seven digits of a row
// (7 x 2D bf16) no longer fit in tensor memory beside six accumulators, so:
// - a chunk is 8 members (16 reals, one MMA K-step); its digits go to one of
//   two TMEM buffers of 7 x 8 columns while the MMAs of the previous chunk
//   read the other;
// - outputs come in passes of 64 reals (MMA N = 64; six accumulators of 64
//   columns at columns 128..511), and every pass runs over the whole K again;
//   pass 0 forms the digits from the state and also writes them to a per-CTA
//   digit buffer in device memory (64 bytes per thread and chunk: 256 / 512
//   KB per CTA for k = 6 / 7, meant to stay in L2), from which later passes
//   reload them instead of forming them again;
// - W's digits stream through two shared-memory buffers in blocks of 64
//   output rows x 64 inputs (the 128-byte swizzled K-major image of the seven
//   digits, 57,344 bytes), the next block copied in bulk while the current one
//   is in use;
// - every read of a tile's state happens in pass 0, so each pass's outputs go
//   straight back to the state after its epilogue.
// Warp roles: sixteen worker warps (four threads per slice row) form digits
// and run the epilogues; a seventeenth issues the MMAs and the W copies.
// Hand-offs are mbarriers:
//   full[b]   digits of the chunk in buffer b stored (512 arrivals)   phase: chunk / 2
//   free[b]   MMAs of the chunk in buffer b done (commit)             phase: chunk / 2
//   wfull[b]  W block in shared buffer b (bulk-copy bytes)            phase: block / 2
//   accfree   accumulators read by a pass's epilogue (512 arrivals)   phase: pass
// The row exponents of the next tile are gathered during the last pass of
// the current one.  Every wait is bounded; a thread that gives up raises a
// shared flag, the workers agree on it at the per-tile barrier (bar.red.or),
// and the control thread lets MMAs and copies in flight land before TMEM and
// shared memory are released.
// Exactness: accumulators d <= 4 hold integers below (d + 1) 2D 127^2 times
// 2^(-7d); for k = 7 and d = 4 that bound is 2^24.3, so accumulator 4 may
// round once its sum passes 2^24, an error below 2^-44 of sum_c |x_c w_nc|
// (never reached by rows of unit norm, whose sums stay near 2^22).
template <int K>
struct OzcShape {
    static constexpr int D = 1 << K;
    static constexpr int NR = 2 * D;               // reals per slice: GEMM K and N
    static constexpr int NHW = 64;                 // outputs per pass (MMA N)
    static constexpr int NPASS = NR / NHW;         // 2 / 4
    static constexpr int NCH = NR / 16;            // chunks (K-steps) per pass: 8 / 16
    static constexpr int NKB = NR / 64;            // W blocks per pass: 2 / 4
    static constexpr int NB = NPASS * NKB;         // W blocks per tile
    static constexpr int DQ = D / 4;               // members per thread in the exponent gather (2 per chunk)
    static constexpr int NACC = 6;
    static constexpr int ABUF = kDigits * 8;       // TMEM columns of one digit buffer
    static constexpr int ACOL0 = 128;              // first accumulator column
    static constexpr int NCOL = 512;
    static constexpr int WBLK = kDigits * NHW * 128;  // bytes of one W block
    static constexpr int NW = 512;                 // worker threads: four per slice row
    static constexpr int NT = NW + 32;             // and the control warp
    // per-CTA digit buffer: a thread's seven bf16 pairs of a chunk (two columns
    // each) padded to 64 bytes, [chunk][part][row]
    static constexpr int NDIG = NCH * NW;  // uint4 x 4 entries per CTA
    static constexpr int OFF_E = 2 * WBLK, OFF_BAR = OFF_E + 2 * NW * 4, OFF_OFF = OFF_BAR + 128;
    static constexpr int SMEM = 1024 + OFF_OFF + D * 8;
    static_assert(DQ == 2 * NCH, "two exponent members per chunk");
};

struct OzcParams {
    int8_t wexp[256];  // E_n - 14 per output real n
};

// acc * 2^(7d) as an integer: exact_int where the bound (d + 1) NR 127^2 of the
// accumulator's integer is below 2^22, else the conversion instruction (exact
// for integers below 2^24, rounding above)
template <int NR, int Dd>
__device__ __forceinline__ int32_t acc_int(float v) {
    if constexpr ((Dd + 1) * NR * 16129 < (1 << 22)) return exact_int(v);
    else return __float2int_rn(v);
}

// Digit-buffer accesses with an L2 eviction policy: kept (evict_last) from the
// write in pass 0 until the last pass reloads them (evict_first), so the
// buffer competes well against the state streaming through L2.
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_drop() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_l2hint(uint4 *a, const uint4 &v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ uint4 ld_l2hint(const uint4 *a, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(a), "l"(pol)
                 : "memory");
    return v;
}

__device__ __forceinline__ void oz_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}
// barrier 1 over the worker warps, returning the OR of their predicates
__device__ __forceinline__ bool workers_sync_or(bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\tbar.red.or.pred b, 1, %2, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(p)), "n"(512)
        : "memory");
    return r != 0;
}

template <int K>
__global__ void __launch_bounds__(OzcShape<K>::NT, 1)
k_dense_ozc(double2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg,
            const uint8_t *__restrict__ wimg, uint4 *__restrict__ gdig, const __grid_constant__ OzcParams P,
            uint32_t wait_limit) {
    using S = OzcShape<K>;
    constexpr int NHW = S::NHW, NACC = S::NACC, NCH = S::NCH, NKB = S::NKB, NB = S::NB, NR = S::NR;
    constexpr int DQ = S::DQ;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sW = base;                                        // two W blocks (1024-aligned)
    int *sE = reinterpret_cast<int *>(base + S::OFF_E);        // [tile parity][part][row] partial exponents
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + S::OFF_BAR);
    uint64_t *full = bar, *freeb = bar + 2, *wfull = bar + 4, *accfree = bar + 6;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 7);
    volatile int *fail = reinterpret_cast<volatile int *>(bar + 8);
    uint64_t *sOff = reinterpret_cast<uint64_t *>(base + S::OFF_OFF);  // [member] offset in the state
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int jm = tid; jm < S::D; jm += S::NT) {
        uint64_t off = 0;
        for (int i = 0; i < K; i++)
            if ((jm >> i) & 1) off += uint64_t(1) << tg.q[i];
        sOff[jm] = off;
    }

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&full[b], S::NW);
            tc::mbar_init(&freeb[b], 1);
            tc::mbar_init(&wfull[b], 1);
        }
        tc::mbar_init(accfree, S::NW);
        *fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, S::NCOL);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t njobs = my_tiles * S::NPASS * NCH;  // chunk j: local tile j / (NPASS NCH), pass (j / NCH) % NPASS

    if (warp == S::NW / 32) {
        // ---------------- control: MMA issue and W copies (one thread)
        if (lane == 0) {
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NHW >> 3) << 17) | (uint32_t(128 >> 4) << 24);
            const uint32_t wbase = tc::smem_u32(sW);
            uint32_t ncommit = 0, nissued = 0, nw = 0;  // MMA groups committed, W copies issued, W blocks used
            if (njobs > 0) {
                tc::mbar_expect_tx(&wfull[0], S::WBLK);
                tc::bulk_g2s(sW, wimg, S::WBLK, &wfull[0]);
                nissued = 1;
            }
            for (uint64_t j = 0; j < njobs; j++) {
                if (*fail) break;
                const int c = int(j % NCH), s = c & 3;
                const uint64_t pj = j / NCH;  // pass, counted over the tiles
                const int h = int(pj % S::NPASS);
                const uint32_t ab = uint32_t(j & 1), wb = nw & 1;
                bool ok = true;
                // the previous pass's epilogue has read the accumulators
                if (c == 0 && pj >= 1) ok = tc::mbar_wait(accfree, uint32_t(pj - 1) & 1u, wait_limit);
                if (ok && s == 0) ok = tc::mbar_wait(&wfull[wb], (nw >> 1) & 1u, wait_limit);
                if (ok) ok = tc::mbar_wait(&full[ab], uint32_t(j >> 1) & 1u, wait_limit);
                if (!ok) {
                    *fail = 1;
                    break;
                }
                tc::fence_after_sync();
                bool first[NACC];
#pragma unroll
                for (int d = 0; d < NACC; d++) first[d] = c == 0;
#pragma unroll
                for (int d = 0; d < NACC; d++) {
#pragma unroll
                    for (int i = 0; i < kDigits; i++) {
#pragma unroll
                        for (int jd = 0; jd < kDigits && i + jd <= kDigits; jd++) {
                            if ((i + jd < NACC - 1 ? i + jd : NACC - 1) != d) continue;
                            const uint64_t bdesc =
                                tc::smem_desc_sw128(wbase + uint32_t(wb * S::WBLK + jd * NHW * 128 + s * 32));
                            const uint32_t a = taddr + uint32_t(ab * S::ABUF + i * 8);
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
                tc::mma_commit(&freeb[ab]);
                ncommit++;
                // at a block's first chunk: copy the next block into the other
                // buffer once the MMAs of the block before (ending at chunk j - 1) are done
                const int bnext = h * NKB + (c >> 2) + 1;
                if (s == 0 && (bnext < NB || j / (S::NPASS * NCH) + 1 < my_tiles)) {
                    if (j >= 1 && !tc::mbar_wait(&freeb[(j - 1) & 1], uint32_t((j - 1) >> 1) & 1u, wait_limit)) {
                        *fail = 1;
                        break;
                    }
                    const uint32_t nb = (nw + 1) & 1;
                    tc::mbar_expect_tx(&wfull[nb], S::WBLK);
                    tc::bulk_g2s(sW + nb * S::WBLK, wimg + size_t(bnext % NB) * S::WBLK, S::WBLK, &wfull[nb]);
                    nissued++;
                }
                if (s == 3) nw++;
            }
            if (*fail) {  // MMAs and copies in flight land before TMEM and shared memory go away
                atomicOr(&g_oz_error, 1);
                if (ncommit > 0) tc::mbar_wait(&freeb[(ncommit - 1) & 1], ((ncommit - 1) >> 1) & 1u, wait_limit);
                for (uint32_t cp = nissued >= 2 ? nissued - 2 : 0; cp < nissued; cp++)
                    tc::mbar_wait(&wfull[cp & 1], (cp >> 1) & 1u, wait_limit);
            }
        }
    } else {
        // ---------------- workers: four threads per slice row
        const int row = tid & 127, q = tid >> 7;  // slice row = TMEM lane; q: this thread's part of the row
        const uint32_t lane_addr = taddr + (uint32_t(32 * (warp & 3)) << 16);
        uint4 *dig = gdig + size_t(blockIdx.x) * S::NDIG * 4 + size_t(tid) * 4;  // + chunk * NW * 4
        const uint64_t keep = l2_policy_keep(), drop = l2_policy_drop();
        // member offsets from the shared table (warp-uniform indices: broadcast reads)
        auto member_off = [&](int jm) { return sOff[jm]; };
        auto exp_of = [](const double2 &v) {
            const int e0 = int((__double_as_longlong(v.x) >> 52) & 0x7FF), e1 = int((__double_as_longlong(v.y) >> 52) & 0x7FF);
            return max(e0, e1) - 1022;
        };
        uint64_t j = 0;  // chunks so far (digit buffer j & 1)
        int eh = -1022;  // this thread's share of the row exponent of the current tile
        if (my_tiles > 0) {
            const uint64_t sb0 = slice_base<K>(uint64_t(blockIdx.x) * 128 + row, tg);
#pragma unroll 8
            for (int jj = 0; jj < DQ; jj++) eh = max(eh, exp_of(sv[sb0 + member_off(q * DQ + jj)]));
        }
        for (uint64_t lt = 0; lt < my_tiles; lt++) {
            const uint64_t tile = uint64_t(blockIdx.x) + lt * gridDim.x;
            const uint64_t sb = slice_base<K>(tile * 128 + row, tg);
            const bool more = lt + 1 < my_tiles;
            const uint64_t sbn = more ? slice_base<K>((tile + gridDim.x) * 128 + row, tg) : sb;
            int *e_t = sE + int(lt & 1) * S::NW;
            e_t[q * 128 + row] = eh;
            if (workers_sync_or(*fail != 0)) break;  // agreed: every worker leaves here
            const int er = max(max(e_t[row], e_t[128 + row]), max(e_t[256 + row], e_t[384 + row]));
            int eh_next = -1022;
            // inputs of the next chunk: pass 0 reads the state (last use: streaming
            // loads), later passes the digits pass 0 left in the digit buffer
            double2 nx0 = __ldcs(sv + sb + member_off(2 * q)), nx1 = __ldcs(sv + sb + member_off(2 * q + 1));
            uint4 nd[4];
            for (int h = 0; h < S::NPASS; h++) {
                for (int c = 0; c < NCH; c++) {
                    const uint32_t ab = uint32_t(j & 1);
                    const double2 x0 = nx0, x1 = nx1;
                    uint4 dc[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) dc[u] = nd[u];
                    {
                        const int cn = c + 1 < NCH ? c + 1 : 0, hn = c + 1 < NCH ? h : h + 1;
                        if (hn == 0) {
                            nx0 = __ldcs(sv + sb + member_off(cn * 8 + 2 * q));
                            nx1 = __ldcs(sv + sb + member_off(cn * 8 + 2 * q + 1));
                        } else if (hn < S::NPASS) {
                            const uint64_t pol = hn + 1 < S::NPASS ? keep : drop;  // the last reload lets go
#pragma unroll
                            for (int u = 0; u < 4; u++) nd[u] = ld_l2hint(dig + size_t(cn) * S::NW * 4 + u, pol);
                        }
                    }
                    // the next tile's exponents, two members per chunk of the last pass
                    // (used at the end of the chunk, so the loads overlap the digits)
                    const bool gather = h + 1 == S::NPASS && more;
                    double2 en0 = make_double2(0.0, 0.0), en1 = en0;
                    if (gather) {
                        en0 = sv[sbn + member_off(q * DQ + 2 * c)];
                        en1 = sv[sbn + member_off(q * DQ + 2 * c + 1)];
                    }
                    // the MMAs two chunks back read this digit buffer
                    if (!*fail && j >= 2 && !tc::mbar_wait(&freeb[ab], uint32_t((j >> 1) + 1) & 1u, wait_limit))
                        *fail = 1;
                    tc::fence_after_sync();
                    if (!*fail) {
                        float col[16];  // digit i: columns 2i, 2i + 1 (members 2q, 2q + 1)
                        if (h == 0) {
                            const Fixed49 f0 = fixed49(x0.x, er), f1 = fixed49(x0.y, er), f2 = fixed49(x1.x, er),
                                          f3 = fixed49(x1.y, er);
#pragma unroll
                            for (int i = 0; i < kDigits; i++) {
                                col[2 * i] = bf16_pair(digit_f(f0, i), digit_f(f1, i));
                                col[2 * i + 1] = bf16_pair(digit_f(f2, i), digit_f(f3, i));
                            }
                            col[14] = col[15] = 0.f;
#pragma unroll
                            for (int u = 0; u < 4; u++)
                                st_l2hint(dig + size_t(c) * S::NW * 4 + u,
                                          make_uint4(__float_as_uint(col[4 * u]), __float_as_uint(col[4 * u + 1]),
                                                     __float_as_uint(col[4 * u + 2]), __float_as_uint(col[4 * u + 3])),
                                          keep);
                        } else {
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                col[4 * u] = __uint_as_float(dc[u].x);
                                col[4 * u + 1] = __uint_as_float(dc[u].y);
                                col[4 * u + 2] = __uint_as_float(dc[u].z);
                                col[4 * u + 3] = __uint_as_float(dc[u].w);
                            }
                        }
#pragma unroll
                        for (int i = 0; i < kDigits; i++) {
                            const float v[2] = {col[2 * i], col[2 * i + 1]};
                            tc::tmem_st<2>(lane_addr + uint32_t(ab * S::ABUF + i * 8 + 2 * q), v);
                        }
                    }
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    oz_arrive(&full[ab]);
                    if (gather) eh_next = max(eh_next, max(exp_of(en0), exp_of(en1)));
                    j++;
                }
                // ---- epilogue of outputs [h NHW + 16 q, + 16): y = 2^(E_r + E_n - 14) (acc0 + ... + acc5).
                // Every read of the tile's state happened in pass 0, before its last
                // chunk's digits went to the tensor cores, so outputs go straight out.
                if (!*fail && !tc::mbar_wait(&freeb[(j - 1) & 1], uint32_t((j - 1) >> 1) & 1u, wait_limit)) *fail = 1;
                tc::fence_after_sync();
                if (!*fail) {
#pragma unroll
                    for (int n0 = 0; n0 < 16; n0 += 4) {
                        const int cl = q * 16 + n0;  // within the pass
                        float ac[NACC][4];
#pragma unroll
                        for (int d = 0; d < NACC; d++)
                            tc::tmem_ld<4>(lane_addr + uint32_t(S::ACOL0 + d * NHW + cl), ac[d]);
#pragma unroll
                        for (int m = 0; m < 2; m++) {
                            double out[2];
#pragma unroll
                            for (int hh = 0; hh < 2; hh++) {
                                const int cc = 2 * m + hh;
                                const int64_t Y = (int64_t(acc_int<NR, 0>(ac[0][cc])) << 36) +
                                                  (int64_t(acc_int<NR, 1>(ac[1][cc] * 128.0f)) << 29) +
                                                  (int64_t(acc_int<NR, 2>(ac[2][cc] * 16384.0f)) << 22) +
                                                  (int64_t(acc_int<NR, 3>(ac[3][cc] * 2097152.0f)) << 15) +
                                                  (int64_t(__float2int_rn(ac[4][cc] * 268435456.0f)) << 8) +
                                                  int64_t(__float2int_rn(ac[5][cc] * 68719476736.0f));
                                out[hh] = i64_to_double(Y, er + int(P.wexp[h * NHW + cl + cc]) - 36);
                            }
                            const int jm = (cl >> 1) + m;  // member within the pass
                            __stcs(sv + sb + member_off(h * (NHW / 2) + jm), make_double2(out[0], out[1]));
                        }
                    }
                }
                tc::fence_before_sync();
                oz_arrive(accfree);
            }
            eh = eh_next;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && *fail) atomicOr(&g_oz_error, 1);
    if (warp == 0) tc::tmem_dealloc(taddr, S::NCOL);
}

// ----------------------------------------------------------------- host side
template <int K>
cast_status run_oz(cast_sv *sv, const PreparedGate &g) {
    using S = OzShape<K>;
    constexpr int D = S::D;
    OzParams P{};
    std::vector<uint8_t> img(S::WBYTES, 0);
    // half n / NHW, digit block j, row n % NHW (block 7 stays zero)
    build_digit_image(g, K, img, P.wexp, [](int n, int c, int j) { return oz_image_offset(n, c, j, S::NHW, S::NACC); },
                      kOzUnitDigits);
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
    const uint32_t inject = take_inject_limit();
    k_dense_oz<K><<<(unsigned)grid, S::NT, smem, sv->stream>>>(reinterpret_cast<double2 *>(sv->data), ntiles, tg,
                                                             static_cast<const uint8_t *>(dev), P,
                                                             inject ? inject : kOzWait, inject ? 1 : 0);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

template <int K>
cast_status run_ozc(cast_sv *sv, const PreparedGate &g) {
    using S = OzcShape<K>;
    constexpr int D = S::D;
    OzcParams P{};
    std::vector<uint8_t> img(size_t(S::NB) * S::WBLK, 0);
    // block (pass n / 64, K-block c / 64): digit j, row n % 64, element c % 64
    static_assert(S::NHW == 64, "ozc_image_offset assumes 64-row blocks");
    build_digit_image(g, K, img, P.wexp, [](int n, int c, int j) { return ozc_image_offset(n, c, j, S::NKB, S::WBLK); },
                      false);
    const void *dev = nullptr;
    cast_status st = upload_matrix(sv, img.data(), img.size(), &dev);
    if (st != CAST_OK) return st;
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const uint64_t cap = uint64_t(sm_count_cached());
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    void *dig = nullptr;
    st = ensure_work(sv, size_t(grid) * S::NDIG * 4 * sizeof(uint4), &dig);
    if (st != CAST_OK) return st;
    CAST_CUDA(cudaFuncSetAttribute(k_dense_ozc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
    const double N = double(uint64_t(1) << sv->n);
    ProfScope ps(sv->stream, "ozdense_k" + std::to_string(K) + "_c128", 32.0 * N, 8.0 * N * double(D));
    k_dense_ozc<K><<<(unsigned)grid, S::NT, S::SMEM, sv->stream>>>(
        reinterpret_cast<double2 *>(sv->data), ntiles, tg, static_cast<const uint8_t *>(dev),
        static_cast<uint4 *>(dig), P, kOzWait);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool oz_eligible(const cast_sv *sv, const PreparedGate &g) {
    if (g_c128_tc.load() != CAST_C128_TC_OZAKI || f64_mode() != CAST_F64_EMULATED || sv->dt != CAST_C128 ||
        g.cls != CLS_DENSE || g.k < 3 || sv->n < g.k + 7 || sparse_mode() == CAST_SPARSE_ALWAYS)
        return false;
    // measured per 30-qubit gate on a random state: this kernel 14.2 / 14.1 /
    // 16.3 / 30-32 / 52-53 ms (k = 3..7) whatever the matrix; the list kernel
    // matches it at about 33 / 17 / 11 / 9.5 / 4.7% of the dense operation
    // count (it is faster below, its time growing with the operation count
    // above a floor of 13.4-14 ms for k = 3..5 and 20-44 ms for k = 6, 7)
    const int64_t ops = opcount(g.m.data(), g.k, 0.0), dense = dense_opcount(g.k);
    switch (g.k) {
        case 3: return 3 * ops > dense;
        case 4: return 6 * ops > dense;
        case 5: return 9 * ops > dense;
        case 6: return 10 * ops > dense;
        default: return 20 * ops > dense;
    }
}

cast_status launch_gate_oz(cast_sv *sv, const PreparedGate &g) {
    switch (g.k) {
        case 3: return run_oz<3>(sv, g);
        case 4: return run_oz<4>(sv, g);
        case 5: return run_oz<5>(sv, g);
        case 6: return run_ozc<6>(sv, g);
        case 7: return run_ozc<7>(sv, g);
        default: return fail(CAST_ERR_UNSUPPORTED, "tensor-core complex128 path covers k = 3..7");
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
