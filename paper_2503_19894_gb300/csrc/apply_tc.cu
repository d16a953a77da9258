// Dense k-qubit gates on complex64 states with the tcgen05 tensor cores
// (k = 4, 5, 6).
//
// The 2^(n-k) matrix-vector products of Eq. 3 are batched into GEMMs.  With an
// interleaved (re, im) slice written as a real vector of 2^(k+1) entries, the
// gate is the real matrix W of 2x2 blocks [[a, -b], [b, a]] (U = a + ib), and
// a tile of 128 consecutive slices is the product
//     Y^T (128 x 2^(k+1)) = X^T (128 x 2^(k+1)) * W^T,
// one tcgen05.mma chain with M = 128 (TMEM lane = slice), N = K = 2^(k+1).
//
// Precision: 3xTF32.  Each state operand x is split into hi = x with its 13
// low significand bits cleared (exactly representable in tf32) and lo =
// tf32(x - hi) rounded to nearest (the subtraction is exact); the gate is
// split as W_hi = tf32(W), W_lo = tf32(W - W_hi), both rounded.  The three
// products lo*W_hi + hi*W_lo + hi*W_hi are accumulated in fp32 in TMEM, giving
// fp32-class accuracy (the dropped lo*lo term and the rounding of lo are
// ~2^-21 relative).  Rounding lo (rather than letting the tensor cores
// truncate it) removes one bias.  The tensor cores' fp32 accumulation itself
// truncates toward zero, which shrinks every output slightly (measured:
// ~2^-23 of the norm per gate, growing with k).  A unitary gate preserves the
// norm of every slice exactly, so each slice's outputs are rescaled by
// |x| / |y|.  Both norms are plain fp32 sums: their rounding errors are
// unbiased and average out over slices and gates, while the truncation they
// correct is systematic; what remains is unbiased rounding noise.  The
// correction is applied as y + y * delta with delta formed as a small number,
// so it is not quantised to the fp32 spacing near 1.  Only gates that are
// unitary to 1e-9 take this path.
//
// Data path per tile: thread (warp w, lane i) owns slice 32*(w%4) + i, i.e.
// TMEM lane 32*(w%4) + i, and 16 of its members (warp group w/4).  A warp's
// 32 slices x 16 members form a cube of 9 index bits (the 5 lowest non-target
// bits and the targets q0..q3); bits 0..3 are always among them, so the cube
// is made of runs of at least 16 contiguous amplitudes (128 bytes).  The warp
// reads it with coalesced 16-byte loads in address order, parks it in its own
// 4 KB of shared memory and every thread then reads its slice row from there;
// outputs go back the same way.  For k <= 5 the loads are cp.async copies
// into a ring of two such buffers per warp, so two tiles are in flight while
// one is computed; k = 6 prefetches one tile into registers.  The buffer is
// XOR-swizzled per gate (host-built tables): a cube element c sits in slot
// c ^ X(c >> 4), with X mapping the row bits that land above bit 3 onto free
// slot bits 1..3, so that the 16-byte chunk accesses (8 lanes per phase) are
// conflict-free and the 8-byte row accesses (16 lanes per phase) are too,
// except for a 2-way conflict when qubit 0 is a target.  Rows are split hi/lo in registers and written into TMEM with
// tcgen05.st.  The MMAs read A from TMEM and W_hi / W_lo from shared memory
// (128-byte swizzled K-major, built once per CTA from the hi/lo split of U
// carried in the launch parameters).
// Pipeline: two accumulators alternate between tiles.  While the MMAs of tile
// t run, the threads drain tile t-1's accumulator (norm fix, stores), and the
// loads of tile t+1 are already in flight (issued right after tile t's
// operands went into TMEM).
// TMEM per CTA: two accumulators, A_hi, A_lo = 4 x 2^(k+1) columns (128, 256,
// 512 for k = 4, 5, 6); registers and padding of the shared-memory request
// keep the number of resident CTAs per SM within the 512 TMEM columns.
//
// Waits on the mbarrier are bounded; a CTA that gives up sets an error bit in
// g_tc_error (read by the host at its next synchronisation point), stops its
// tile loop, waits once more (bounded) for its MMAs and frees its TMEM.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "tc.cuh"

namespace cast {

namespace {

__device__ int g_tc_error;
std::atomic<int> g_tensor_mode{CAST_TC_TF32X3};

constexpr uint32_t kWaitLimit = 1u << 26;  // polls of the MMA barrier (~1 s)
// test hook (cast_debug_inject_timeout): the issuing thread skips its MMAs
// and commit, so every wait of the next launch runs out
std::atomic<uint32_t> g_inject_limit{0};

// The hi/lo split of U: by value in the launch parameters for k <= 5 (at most
// 16 KB), through a device buffer for k = 6 (64 KB, beyond the 32 KB limit).
template <int K, bool BYVAL = (K <= 5)>
struct TcMat;
template <int K>
struct TcMat<K, true> {
    float2 hi[1 << K][1 << K];
    float2 lo[1 << K][1 << K];
    __device__ __forceinline__ float2 h(int r, int c) const { return hi[r][c]; }
    __device__ __forceinline__ float2 l(int r, int c) const { return lo[r][c]; }
};
template <int K>
struct TcMat<K, false> {
    const float2 *hi;  // D x D, then lo (D x D) right after
    __device__ __forceinline__ float2 h(int r, int c) const { return hi[r * (1 << K) + c]; }
    __device__ __forceinline__ float2 l(int r, int c) const { return hi[(1 << (2 * K)) + r * (1 << K) + c]; }
};

// The three bf16 pieces of U (each a float holding a bf16-exact value), by
// value in the launch parameters (24 KB for k = 5).
template <int K>
struct TcMatB {
    float2 p[3][1 << K][1 << K];
};

// k = 4 with two warps per TMEM lane quarter (eight members each, eight
// warps per CTA, four CTAs per SM, 56 registers) instead of one (sixteen
// members, four warps): twice the warps and loads in flight per SM, measured
// no faster (2.88-2.93 against 2.88-2.90 ms per 30-qubit gate with 3xTF32;
// 3.08-3.14 against 2.85-2.88 ms with split bf16), so it stays off
constexpr bool kTc4Split = false;

template <int K>
struct TcShape {
    static constexpr int D = 1 << K;           // slice members
    static constexpr int NK = 2 * D;           // GEMM N = K (reals)
    static constexpr int MPT = (K == 4 && kTc4Split) ? 8 : (D < 16 ? D : 16);  // members per thread
    static constexpr int MB = MPT == 8 ? 3 : 4;  // member bits of a warp's cube
    static constexpr int CUBE = 32 * MPT;      // amplitudes of a warp's cube
    static constexpr int ROUNDS = CUBE / 64;   // 16-byte chunks per lane
    static constexpr int GROUPS = D / MPT;     // warps per TMEM lane quarter
    static constexpr int NT = 128 * GROUPS;    // threads per CTA
    static constexpr int NCOL = 4 * NK;        // two accumulators, A_hi, A_lo
    static constexpr int CTAS_PER_SM = 512 / NCOL;
    // staging cubes per warp: k <= 5 keeps a ring of two filled by cp.async
    // (two tiles in flight); k = 6 (128 KB of W in shared memory) keeps one
    // and prefetches the next tile into registers
    static constexpr int STAGES = K <= 5 ? 2 : 1;
    static_assert(NCOL >= 128 && NCOL <= 512, "TMEM columns");
};

// tf32 parts of an fp32 value with integer operations: the value with its 13
// low significand bits cleared (exact in tf32), and the nearest tf32 value
// (ties away from zero, as cvt.rna; the carry into the exponent is the
// correct rounding).
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}


// bf16 pieces of an fp32 value: the top 16 bits (8 significant bits), exact
// remainders, and the nearest bf16 for the last piece (ties away from zero)
__device__ __forceinline__ float bf16_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFF0000u); }
__device__ __forceinline__ float bf16_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x8000u) & 0xFFFF0000u);
}
// two bf16-exact floats as one TMEM column (lo half: a, hi half: b)
__device__ __forceinline__ float bf16x2(float a, float b) {
    return __uint_as_float(__byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632));
}
// 128-byte swizzled K-major image of rows of 64 bf16: row r, element c < 64
__host__ __device__ __forceinline__ uint32_t sw128_b16(int r, int c) {
    return uint32_t((r >> 3) * 1024 + (r & 7) * 128 + (((c >> 3) ^ (r & 7)) << 4) + (c & 7) * 2);
}

// W region of shared memory: 3xTF32 W_hi, W_lo (NK x NK fp32 each); split
// bf16 three pieces of NK rows x 128 bytes (k <= 5: NK <= 64 bf16 per row)
template <int K, bool BF>
__host__ __device__ constexpr int tc_w_bytes() { return BF ? 3 * (2 << K) * 128 : 2 * (2 << K) * (2 << K) * 4; }

template <int K, bool BF>
__global__ void __launch_bounds__(TcShape<K>::NT, TcShape<K>::CTAS_PER_SM)
k_dense_tc(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg,
           const __grid_constant__ std::conditional_t<BF, TcMatB<K>, TcMat<K>> U,
           const __grid_constant__ CubeTables st, uint32_t wait_limit, int skip_mma) {
    using S = TcShape<K>;
    constexpr int NK = S::NK, MPT = S::MPT;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, NK);
    // kind::f16: D fp32, A and B bf16, N = NK, M = 128
    constexpr uint32_t IDESC_BF = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NK >> 3) << 17) | (uint32_t(128 >> 4) << 24);
    constexpr int G = S::GROUPS;
    // 3xTF32: accumulator 0 at column 0, A_hi, A_lo, accumulator 1;
    // bf16: accumulators 0, 1, then the three A pieces of NK / 2 columns
    constexpr uint32_t COL_AH = NK, COL_AL = 2 * NK, COL_ACC1 = BF ? NK : 3 * NK, COL_AB = 2 * NK;
    static_assert(!BF || K <= 5, "the bf16 pieces of W fill 128-byte rows for k <= 5");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sWhi = base;                      // bf16: piece 0
    uint8_t *sWlo = sWhi + (BF ? NK * 128 : NK * NK * 4);  // bf16: piece 1 (piece 2 after it)
    uint64_t *mbar = reinterpret_cast<uint64_t *>(base + tc_w_bytes<K, BF>());
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    float *xnorm = reinterpret_cast<float *>(tslot + 2);  // [2][GROUPS][128] |x|^2 parts of a row
    float *ynorm = xnorm + 2 * G * 128;                   // [GROUPS][128] |y|^2 parts

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, group = warp >> 2, j0 = group * MPT;
    const int row = 32 * quarter + lane;

    // ---- prologue: W_hi / W_lo (SW128 K-major), barrier, TMEM
    for (int idx = tid; idx < NK * NK; idx += S::NT) {
        const int r = idx / NK, c = idx % NK;
        if constexpr (BF) {
#pragma unroll
            for (int pc = 0; pc < 3; pc++) {
                const float2 h = U.p[pc][r >> 1][c >> 1];
                const float v = (r & 1) == (c & 1) ? h.x : ((r & 1) ? h.y : -h.y);
                *reinterpret_cast<uint16_t *>(sWhi + pc * NK * 128 + sw128_b16(r, c)) =
                    uint16_t(__float_as_uint(v) >> 16);
            }
        } else {
            const float2 h = U.h(r >> 1, c >> 1), l = U.l(r >> 1, c >> 1);
            float vh, vl;
            if ((r & 1) == (c & 1)) { vh = h.x; vl = l.x; }   // a on the 2x2 diagonal
            else if (r & 1) { vh = h.y; vl = l.y; }           // b (row im, col re)
            else { vh = -h.y; vl = -l.y; }                    // -b (row re, col im)
            *reinterpret_cast<float *>(sWhi + tc::sw128_offset(r, c, NK)) = vh;
            *reinterpret_cast<float *>(sWlo + tc::sw128_offset(r, c, NK)) = vl;
        }
    }
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, S::NCOL);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t lane_addr = taddr + (uint32_t(32 * quarter) << 16);

    // this warp's staging cubes (STAGES x 512 amplitudes), after the norm arrays
    constexpr int NS = S::STAGES;
    float2 *stages = reinterpret_cast<float2 *>(ynorm + G * 128 + 4) + warp * (S::CUBE * NS);
    // member offset of this warp group's first member j0 (targets q4, q5 only)
    uint64_t off0 = 0;
#pragma unroll
    for (int i = S::MB; i < K; i++)
        if ((j0 >> i) & 1) off0 += uint64_t(1) << tg.q[i];
    const uint64_t g_lane = st.g_lane[lane];
    const uint32_t s_lane = st.s_lane[lane], s_row = st.s_row[lane];
    auto cube_base = [&](uint64_t t) { return slice_base<K>(t * 128 + uint64_t(32 * quarter), tg) + off0 + g_lane; };
    // the warp's cube of tile t, 8 chunks of 16 bytes per lane, coalesced
    auto copy_async = [&](uint64_t t, float2 *stage) {
        const float2 *b = sv + cube_base(t);
        const uint32_t d = tc::smem_u32(stage);
#pragma unroll
        for (int j = 0; j < S::ROUNDS; j++)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + ((s_lane ^ st.s_j[j]) >> 1) * 16u),
                         "l"(b + st.g_j[j])
                         : "memory");
    };
    auto load_regs = [&](uint64_t t, float4 (&c)[S::ROUNDS]) {
        const float2 *b = sv + cube_base(t);
#pragma unroll
        for (int j = 0; j < S::ROUNDS; j++) c[j] = __ldcs(reinterpret_cast<const float4 *>(b + st.g_j[j]));
    };
    auto regs_to_stage = [&](const float4 (&c)[S::ROUNDS], float2 *stage) {
        float4 *s4 = reinterpret_cast<float4 *>(stage);
#pragma unroll
        for (int j = 0; j < S::ROUNDS; j++) s4[(s_lane ^ st.s_j[j]) >> 1] = c[j];
    };

    // drain one tile's accumulator: restore each slice's norm, store to HBM
    // through the staging cube `stage` (free: its input is already in TMEM).
    // xh, xl: this thread's compensated |x|^2 of the tile (GROUPS == 1), else
    // the parts every warp group left in xnorm[xb]
    auto epilogue = [&](uint64_t t, uint32_t acc_col, int xb, float xrow, float2 *stage) {
        float Y = 0.f, Y2 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; h++) {  // pass 1: |y|^2 of the row
            float v[MPT];
            tc::tmem_ld<MPT>(lane_addr + acc_col + 2 * j0 + MPT * h, v);
#pragma unroll
            for (int m = 0; m < MPT / 2; m++) {
                Y = fmaf(v[2 * m], v[2 * m], Y);
                Y2 = fmaf(v[2 * m + 1], v[2 * m + 1], Y2);
            }
        }
        Y += Y2;
        float X = xrow;
        if constexpr (G > 1) {
            // the row's members are spread over the G warps of this lane quarter
            ynorm[group * 128 + row] = Y;
            asm volatile("bar.sync %0, %1;" ::"r"(1 + quarter), "r"(32 * G) : "memory");
            X = 0.f;
            Y = 0.f;
#pragma unroll
            for (int gq = 0; gq < G; gq++) {
                X += xnorm[(xb * G + gq) * 128 + row];
                Y += ynorm[gq * 128 + row];
            }
        }
        // y <- y * sqrt(X / Y) = y + y * delta with delta = (X - Y) / (2 Y) to
        // first order (|delta| ~ 1e-7; the second-order term is ~1e-14).
        // delta is formed as a small number (X - Y is exact when the two are
        // close) so the correction is not quantised to multiples of 2^-23 as
        // a scale factor near 1 would be.
        float delta = 0.0f;
        if (Y > 0.0f && X > 0.0f) delta = 0.5f * (X - Y) / Y;
        // pass 2: corrected row -> staging cube -> coalesced 16-byte stores
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float v[MPT];
            tc::tmem_ld<MPT>(lane_addr + acc_col + 2 * j0 + MPT * h, v);
            if (st.pair) {
#pragma unroll
                for (int m = 0; m < MPT / 2; m += 2)
                    reinterpret_cast<float4 *>(stage)[(s_row ^ st.s_mem[h * (MPT / 2) + m]) >> 1] =
                        make_float4(fmaf(v[2 * m], delta, v[2 * m]), fmaf(v[2 * m + 1], delta, v[2 * m + 1]),
                                    fmaf(v[2 * m + 2], delta, v[2 * m + 2]), fmaf(v[2 * m + 3], delta, v[2 * m + 3]));
            } else {
#pragma unroll
                for (int m = 0; m < MPT / 2; m++)
                    stage[s_row ^ st.s_mem[h * (MPT / 2) + m]] =
                        make_float2(fmaf(v[2 * m], delta, v[2 * m]), fmaf(v[2 * m + 1], delta, v[2 * m + 1]));
            }
        }
        __syncwarp();
        float2 *b = sv + cube_base(t);
        const float4 *s4 = reinterpret_cast<const float4 *>(stage);
#pragma unroll
        for (int j = 0; j < S::ROUNDS; j++)
            __stcs(reinterpret_cast<float4 *>(b + st.g_j[j]), s4[(s_lane ^ st.s_j[j]) >> 1]);
        __syncwarp();
    };

    float4 nxt[S::ROUNDS];  // register prefetch (one stage only)
    const uint64_t step = gridDim.x;
    uint64_t tile = blockIdx.x, prev = ~uint64_t(0);
    uint32_t phase = 0;
    int buf = 0;  // accumulator (and xnorm half) of the current tile
    float x_prev = 0.f;
    bool failed = false;
    if constexpr (NS > 1) {
#pragma unroll
        for (int si = 0; si < NS; si++) {
            if (tile + si * step < ntiles) copy_async(tile + si * step, stages + si * S::CUBE);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
    } else {
        if (tile < ntiles) load_regs(tile, nxt);
    }
    int si = 0;  // stage of the current tile
    while (tile < ntiles) {
        float2 *stage = stages + si * S::CUBE;
        // ---- this thread's slice row from the staged cube
        if constexpr (NS > 1) {
            asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
        } else {
            regs_to_stage(nxt, stage);
        }
        __syncwarp();
        // ---- split in two halves of 8 members, TMEM stores of A_hi and A_lo
        // (the previous MMAs are done)
        float xs = 0.f, xs2 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float2 x[MPT / 2];
            if (st.pair) {  // members 2m, 2m+1 in one 16-byte chunk
#pragma unroll
                for (int m = 0; m < MPT / 2; m += 2) {
                    const float4 c = reinterpret_cast<const float4 *>(stage)[(s_row ^ st.s_mem[h * (MPT / 2) + m]) >> 1];
                    x[m] = make_float2(c.x, c.y);
                    x[m + 1] = make_float2(c.z, c.w);
                }
            } else {
#pragma unroll
                for (int m = 0; m < MPT / 2; m++) x[m] = stage[s_row ^ st.s_mem[h * (MPT / 2) + m]];
            }
            if constexpr (BF) {
                // three bf16 pieces per real: truncated, truncated remainder,
                // rounded last remainder (each subtraction exact in fp32); one
                // column per member holds its (re, im) pair of a piece
                float p0[MPT / 2], p1[MPT / 2], p2[MPT / 2];
#pragma unroll
                for (int m = 0; m < MPT / 2; m++) {
                    const float a0 = bf16_trunc(x[m].x), b0 = bf16_trunc(x[m].y);
                    const float ar = x[m].x - a0, br = x[m].y - b0;
                    const float a1 = bf16_trunc(ar), b1 = bf16_trunc(br);
                    p0[m] = bf16x2(a0, b0);
                    p1[m] = bf16x2(a1, b1);
                    p2[m] = bf16x2(bf16_round(ar - a1), bf16_round(br - b1));
                }
                tc::tmem_st<MPT / 2>(lane_addr + COL_AB + j0 + (MPT / 2) * h, p0);
                tc::tmem_st<MPT / 2>(lane_addr + COL_AB + NK / 2 + j0 + (MPT / 2) * h, p1);
                tc::tmem_st<MPT / 2>(lane_addr + COL_AB + NK + j0 + (MPT / 2) * h, p2);
            } else {
                float v[MPT];
#pragma unroll
                for (int m = 0; m < MPT / 2; m++) {
                    v[2 * m] = tf32_trunc(x[m].x);
                    v[2 * m + 1] = tf32_trunc(x[m].y);
                }
                tc::tmem_st<MPT>(lane_addr + COL_AH + 2 * j0 + MPT * h, v);
                // the remainder is rounded to tf32 as well: the tensor cores would
                // otherwise truncate it, a bias that shrinks the norm gate after gate
#pragma unroll
                for (int m = 0; m < MPT / 2; m++) {
                    v[2 * m] = tf32_round(x[m].x - v[2 * m]);
                    v[2 * m + 1] = tf32_round(x[m].y - v[2 * m + 1]);
                }
                tc::tmem_st<MPT>(lane_addr + COL_AL + 2 * j0 + MPT * h, v);
            }
#pragma unroll
            for (int m = 0; m < MPT / 2; m++) {
                xs = fmaf(x[m].x, x[m].x, xs);
                xs2 = fmaf(x[m].y, x[m].y, xs2);
            }
        }
        xs += xs2;
        if constexpr (G > 1) xnorm[(buf * G + group) * 128 + row] = xs;
        tc::tmem_wait_st();
        const uint64_t next = tile + step;
        if constexpr (NS == 1) {  // prefetch the next tile; in flight meanwhile
            if (next < ntiles) load_regs(next, nxt);
        }
        tc::fence_before_sync();
        // every row is in TMEM; a failed wait of the previous tile ends the
        // loop here, agreed by all threads
        if (__syncthreads_or(failed)) break;
        tc::fence_after_sync();
        if (tid == 0 && !skip_mma) {
            const uint32_t wH = tc::smem_u32(sWhi);
            const uint32_t dacc = taddr + (buf ? COL_ACC1 : 0u);
            uint32_t acc = 0;
            if constexpr (BF) {
                // six products (piece of x, piece of W), smallest weight first
                constexpr int PA[6] = {2, 1, 0, 1, 0, 0}, PW[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
                for (int pr = 0; pr < 6; pr++) {
#pragma unroll
                    for (int s = 0; s < NK / 16; s++) {
                        const uint32_t a = taddr + COL_AB + uint32_t(PA[pr] * (NK / 2) + 8 * s);
                        const uint64_t b = tc::smem_desc_sw128(wH + uint32_t(PW[pr] * NK * 128 + 32 * s));
                        asm volatile(
                            "{\n\t.reg .pred pp;\n\tsetp.ne.b32 pp, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, pp;\n\t}" ::"r"(dacc),
                            "r"(a), "l"(b), "r"(IDESC_BF), "r"(acc));
                        acc = 1;
                    }
                }
            } else {
                const uint32_t wL = tc::smem_u32(sWlo);
#pragma unroll
                for (int pr = 0; pr < 3; pr++) {
                    const uint32_t acol = pr == 0 ? COL_AL : COL_AH;  // lo*W_hi, hi*W_lo, hi*W_hi
                    const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                    for (int s = 0; s < NK / 8; s++) {
                        const uint32_t kw = uint32_t((s >> 2) * (NK / 8) * 1024 + (s & 3) * 32);
                        tc::mma_tf32_ts(dacc, taddr + acol + 8 * s, tc::smem_desc_sw128(w + kw), IDESC, acc);
                        acc = 1;
                    }
                }
            }
            tc::mma_commit(mbar);
        }
        __syncwarp();  // warp 0 reconverges before its .sync.aligned TMEM loads
        // ---- the previous tile's epilogue runs while these MMAs execute; it
        // stores through this tile's staging cube, which is then refilled
        if (prev != ~uint64_t(0)) epilogue(prev, buf ? 0u : COL_ACC1, buf ^ 1, x_prev, stage);
        if constexpr (NS > 1) {
            __syncwarp();
            if (tile + NS * step < ntiles) copy_async(tile + NS * step, stage);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        x_prev = xs;
        failed = !tc::mbar_wait(mbar, phase, wait_limit);
        phase ^= 1u;
        tc::fence_after_sync();
        prev = tile;
        tile = next;
        buf ^= 1;
        si = (si + 1) % NS;
    }
    if constexpr (NS > 1) asm volatile("cp.async.wait_group 0;" ::: "memory");
    failed = __syncthreads_or(failed);
    if (failed) phase ^= 1u;  // the wait that ran out is retried below
    if (!failed && prev != ~uint64_t(0)) epilogue(prev, buf ? 0u : COL_ACC1, buf ^ 1, x_prev, stages + si * S::CUBE);
    if (failed) {
        if (tid == 0) atomicOr(&g_tc_error, 1);
        tc::mbar_wait(mbar, phase, wait_limit);  // let an MMA in flight finish before freeing TMEM
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, S::NCOL);
}

// host-side tf32 rounding matching cvt.rna (nearest, ties away from zero)
float host_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

template <int K, bool BF>
size_t tc_smem_bytes() {
    using S = TcShape<K>;
    const size_t need = 1024 + size_t(tc_w_bytes<K, BF>()) + 64 + 3 * 4 * 128 * S::GROUPS + 16 +
                        size_t(S::NT / 32) * S::CUBE * 8 * S::STAGES;
    // at most CTAS_PER_SM resident CTAs per SM (228 KB of shared memory each)
    const size_t floor = (228 * 1024) / (S::CTAS_PER_SM + 1) + 1024;
    return need > floor ? need : floor;
}

// bf16 pieces of a double, on the host: the top 8 significant bits
// (truncated) of the float nearest w, and the nearest bf16 of w
float host_bf16_trunc(double w) {
    const float f = (float)w;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u &= 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}
float host_bf16_round(double w) {
    const float f = (float)w;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x8000u) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

template <int K, bool BF>
cast_status run_tc(cast_sv *sv, const PreparedGate &g) {
    constexpr int D = 1 << K;
    using S = TcShape<K>;
    std::conditional_t<BF, TcMatB<K>, TcMat<K>> U;
    if constexpr (BF) {
        // w = p0 + p1 + p2: p0, p1 truncated (the remainders are exact in
        // double), p2 the nearest bf16 of what is left
        for (int r = 0; r < D; r++)
            for (int c = 0; c < D; c++) {
                const cplx u = g.m[size_t(r) * D + c];
                float pr[3], pi[3];
                double wr = u.real(), wi = u.imag();
                pr[0] = host_bf16_trunc(wr), pi[0] = host_bf16_trunc(wi);
                wr -= pr[0], wi -= pi[0];
                pr[1] = host_bf16_trunc(wr), pi[1] = host_bf16_trunc(wi);
                wr -= pr[1], wi -= pi[1];
                pr[2] = host_bf16_round(wr), pi[2] = host_bf16_round(wi);
                for (int pc = 0; pc < 3; pc++) U.p[pc][r][c] = make_float2(pr[pc], pi[pc]);
            }
    } else {
        std::vector<float2> hl(size_t(2) << (2 * K));
        for (int r = 0; r < D; r++)
            for (int c = 0; c < D; c++) {
                const cplx u = g.m[size_t(r) * D + c];
                const float hr = host_tf32((float)u.real()), hi = host_tf32((float)u.imag());
                hl[size_t(r) * D + c] = make_float2(hr, hi);
                hl[(size_t(1) << (2 * K)) + size_t(r) * D + c] =
                    make_float2(host_tf32((float)(u.real() - (double)hr)), host_tf32((float)(u.imag() - (double)hi)));
            }
        if constexpr (K <= 5) {
            std::memcpy(U.hi, hl.data(), sizeof(U.hi));
            std::memcpy(U.lo, hl.data() + (size_t(1) << (2 * K)), sizeof(U.lo));
        } else {
            const void *dev = nullptr;
            cast_status st = upload_matrix(sv, hl.data(), hl.size() * sizeof(float2), &dev);
            if (st != CAST_OK) return st;
            U.hi = static_cast<const float2 *>(dev);
        }
    }
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const size_t smem = tc_smem_bytes<K, BF>();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tc<K, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t cap = uint64_t(sm_count_cached()) * S::CTAS_PER_SM;
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    ProfScope ps(sv->stream, std::string(BF ? "tcbf_k" : "tc_k") + std::to_string(K) + "_c64",
                 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    const uint32_t inject = take_inject_limit();
    const CubeTables st = make_cube_tables(g.q, K, S::MB);
    k_dense_tc<K, BF><<<(unsigned)grid, S::NT, smem, sv->stream>>>(reinterpret_cast<float2 *>(sv->data), ntiles, tg, U, st,
                                                               inject ? inject : kWaitLimit, inject ? 1 : 0);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool tensor_cores_on() { return g_tensor_mode.load() != CAST_TC_OFF; }

uint32_t take_inject_limit() { return g_inject_limit.exchange(0); }

bool tc_eligible(const cast_sv *sv, const PreparedGate &g) {
    const int mode = g_tensor_mode.load();
    return mode != CAST_TC_OFF && sv->dt == CAST_C64 && g.cls == CLS_DENSE && g.unitary && g.k >= 4 &&
           g.k <= (mode == CAST_TC_BF16X6 ? 5 : 6) && sv->n >= g.k + 7;
}

cast_status launch_gate_tc(cast_sv *sv, const PreparedGate &g) {
    const bool bf = g_tensor_mode.load() == CAST_TC_BF16X6;
    if (g.k == 4) return bf ? run_tc<4, true>(sv, g) : run_tc<4, false>(sv, g);
    if (g.k == 5) return bf ? run_tc<5, true>(sv, g) : run_tc<5, false>(sv, g);
    if (g.k == 6) return run_tc<6, false>(sv, g);
    return fail(CAST_ERR_UNSUPPORTED, "tensor-core path covers k = 4, 5, 6");
}

cast_status take_device_error() {
    int v = 0;
    CAST_CUDA(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)));
    if (tcc_error_flag_take()) v = 1;
    if (oz_error_flag_take()) v = 1;
    if (v) {
        const int zero = 0;
        CAST_CUDA(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int)));
        return fail(CAST_ERR_TIMEOUT, "a tensor-core kernel gave up waiting for its MMAs (bounded wait)");
    }
    return CAST_OK;
}

}  // namespace cast

extern "C" {

cast_status cast_set_tensor_mode(int mode) {
    if (mode != CAST_TC_OFF && mode != CAST_TC_TF32X3 && mode != CAST_TC_BF16X6)
        return cast::fail(CAST_ERR_ARG, "unknown tensor mode");
    cast::g_tensor_mode = mode;
    return CAST_OK;
}

int cast_get_tensor_mode(void) { return cast::g_tensor_mode.load(); }

cast_status cast_debug_inject_timeout(uint32_t wait_limit) {
    if (wait_limit == 0) return cast::fail(CAST_ERR_ARG, "wait limit must be positive");
    cast::g_inject_limit = wait_limit;
    return CAST_OK;
}

}  // extern "C"
