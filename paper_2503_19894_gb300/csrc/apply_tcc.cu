// Dense 6- and 7-qubit gates on complex64 states with the tcgen05 tensor
// cores, with the K dimension fed in chunks.
//
// Same GEMM as apply_tc.cu (Eq. 3 batched: a tile of 128 slices times the
// real 2^(k+1) x 2^(k+1) form W of the gate, 3xTF32, fp32 accumulation in
// TMEM, per-slice norm restoration).  The K dimension is cut into chunks of
// 16 members (32 reals): 8 for k = 7, 4 for k = 6.
//   - A (the slice rows) of chunk c is the staged cube of member group c
//     (csrc/cube.cpp: 32 slices x 16 members per warp, coalesced 16-byte
//     cp.async copies, two in flight per warp), split hi/lo in registers and
//     written into one of two TMEM chunk buffers (64 columns each);
//   - B = W^T restricted to the chunk's 32 K columns, hi and lo, laid out on
//     the host as the exact 128-byte-swizzled shared-memory image.  For k = 7
//     (256 KB for each of W_hi and W_lo) a chunk (64 KB) arrives with two bulk
//     copies (TMA, non-tensor) onto an mbarrier, one chunk ahead of the MMAs
//     that read it (two shared buffers); for k = 6 all of W (128 KB) is copied
//     once and stays resident;
//   - the three products of a chunk are 3 x 4 MMAs of M = 128, N = 2^(k+1),
//     K = 8 into a 2^(k+1)-column accumulator.
// Eight worker warps in two groups take alternate chunks; a ninth warp issues
// the MMAs and the W copies (details at the kernel).  After a tile's last
// chunk both groups drain its accumulator: the row's |y|^2, the norm
// correction against |x|^2 summed over the chunks, and the outputs go back to
// HBM through per-warp output cubes.  TMEM: k = 7 one 256-column accumulator
// and two A buffers (384 of 512 columns); k = 6 two 128-column accumulators
// that alternate between tiles (the epilogue of one overlaps the next tile's
// MMAs) and the two A buffers (384).  Shared memory 226 KB; one CTA per SM.
//
// Measured per 30-qubit gate: k = 6 3.6 ms (4.5 ms for apply_tc.cu's kernel,
// whose single A buffer serialises the A writes with the MMAs; that kernel
// stays selectable with kTcc6); k = 7 6.6-7.0 ms.  A four-warp form (every
// warp on every chunk) ran 10% slower for k = 7.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "tc.cuh"

namespace cast {

int tcc_error_flag_take();

namespace {

__device__ int g_tcc_error;

// k = 6 streams W (64 KB of buffers) instead of keeping it resident (128 KB),
// for four cube stages per worker warp instead of two: measured 4.26-4.31
// against 3.58-3.62 ms per 30-qubit gate (W re-read from L2 every tile), so off
constexpr bool kTcc6Stream = false;

template <int K>
struct TccShape {
    static constexpr int D = 1 << K;            // slice members
    static constexpr int N = 2 * D;             // output reals = accumulator columns (MMA N)
    static constexpr int CHUNKS = D / 16;       // K chunks of 16 members (32 reals)
    // k = 6: two accumulators alternate between tiles, so a tile's epilogue
    // overlaps the next tile's MMAs; W (128 KB) resident, or streamed (kTcc6Stream)
    // to make room for four cube stages per warp instead of two.  k = 7: W is
    // streamed one chunk ahead and the one 256-column accumulator is all TMEM allows
    static constexpr bool RESIDENT_W = K == 6 && !kTcc6Stream;
    static constexpr int NACC = K == 6 ? 2 : 1;
    static constexpr int COL_A = NACC * N;      // TMEM: accumulators, then 2 A buffers of 64 columns
    static constexpr uint32_t CHUNK_BYTES = uint32_t(N) * 128u;  // W^T chunk, hi or lo
    static constexpr uint32_t W_BYTES = RESIDENT_W ? 2u * CHUNKS * CHUNK_BYTES : 4u * CHUNK_BYTES;  // W region
    static constexpr int NS = (K == 6 && !RESIDENT_W) ? 4 : 2;  // cube stages per worker warp
    static constexpr int COLS = 512;
    static_assert(COL_A + 128 <= COLS, "TMEM columns");
};
constexpr uint32_t kTccWaitLimit = 1u << 26;
// dense 6-qubit gates take this kernel rather than apply_tc.cu's resident-W one
constexpr bool kTcc6 = true;

struct TccMat {
    const uint8_t *hi;  // CHUNKS chunk images of CHUNK_BYTES
    const uint8_t *lo;
};

__device__ __forceinline__ float tcc_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ float tcc_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Warp-specialised form: the same chunks, but eight worker warps in two
// groups of four take alternate chunks (group g owns TMEM A buffer g), so one
// group prepares a chunk while the MMAs of the other group's chunk run, and a
// ninth warp only waits on mbarriers, issues the MMAs and brings in W (k = 7:
// chunk by chunk into two buffers; k = 6: once, resident).  Both groups drain
// an accumulator (alternate 32-column blocks, norms exchanged per lane quarter
// through an mbarrier).  A group drains tile t after it has prepared its first
// chunk of tile t + 1: with two accumulators (k = 6) those MMAs run during the
// epilogue; with one (k = 7) they can start as soon as it ends.  Barriers
// (a = accumulator of the tile, NACC of them):
//   bar_a[g]  A chunk of group g in TMEM (128 arrivals)     phase: job / 2
//   bar_b[b]  W chunk in shared buffer b (bulk-copy bytes)   phase: job / 2 (k = 6: all of W, once)
//   bar_m[b]  MMAs of the chunk in buffer b done (commit)    phase: job / 2
//   bar_f[a]  MMAs of a tile's last chunk done (commit)      phase: tile / NACC
//   bar_e[a]  accumulator drained (256 arrivals)            phase: tile / NACC
//   bar_q[q]  norm halves of lane quarter q written (64)    phase: tile
// A parity wait only tells phases apart within one phase of the barrier, so
// each waiter follows a barrier whose every phase it waits for (the groups
// learn that the accumulator is complete from bar_f, not from bar_m[1], which
// group 0 does not follow).  Every wait is bounded; a thread that gives up
// raises a shared flag that all loops check, and the control thread lets MMAs
// and copies in flight land.
constexpr int kWsWorkers = 8;
constexpr int kWsThreads = 32 * (kWsWorkers + 1);

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

template <int K>
__global__ void __launch_bounds__(kWsThreads, 1)
k_dense_tcc_ws(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg, TccMat W,
               const __grid_constant__ CubeTables st, uint32_t wait_limit, int skip_mma) {
    using S = TccShape<K>;
    constexpr int N = S::N, CHUNKS = S::CHUNKS, NACC = S::NACC;
    constexpr uint32_t CB = S::CHUNK_BYTES;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, N);
    extern __shared__ __align__(1024) uint8_t ws_smem[];
    if (tc::smem_u32(ws_smem) & 1023u) {  // the W images need 1024-byte alignment
        if (threadIdx.x == 0) atomicOr(&g_tcc_error, 2);
        return;
    }
    // W: k = 7 [2 buffers][hi, lo] x CB; k = 6 [hi chunks 0..3][lo chunks 0..3] x CB
    uint8_t *sB = ws_smem;
    float2 *cubes = reinterpret_cast<float2 *>(ws_smem + S::W_BYTES);   // [8 warps][NS stages][512]
    float2 *outc = cubes + kWsWorkers * S::NS * 512;                     // [8 warps][512]
    float *xnorm = reinterpret_cast<float *>(outc + kWsWorkers * 512);  // [2 groups][128]
    float *ynorm = xnorm + 256;                                          // [2 groups][128]
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(ynorm + 256);
    uint64_t *bar_b = bar_a + 2, *bar_m = bar_a + 4, *bar_e = bar_a + 6, *bar_f = bar_a + 8, *bar_q = bar_a + 10;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_a + 14);
    volatile int *fail = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&bar_a[i], 128);
            tc::mbar_init(&bar_b[i], 1);
            tc::mbar_init(&bar_m[i], 1);
            tc::mbar_init(&bar_e[i], 256);
            tc::mbar_init(&bar_f[i], 1);
        }
        for (int q = 0; q < 4; q++) tc::mbar_init(&bar_q[q], 64);
        *fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, S::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t njobs = my_tiles * CHUNKS;  // job j: local tile j / CHUNKS, chunk j % CHUNKS
    auto job_tile = [&](uint64_t j) { return uint64_t(blockIdx.x) + (j / CHUNKS) * gridDim.x; };

    if (warp == kWsWorkers) {
        // ---------------- control: MMA issue and W copies (one thread)
        if (lane == 0) {
            uint32_t m_done0 = 0, m_done1 = 0, b_armed0 = 0, b_armed1 = 0, f_done0 = 0, f_done1 = 0;
            auto load_w = [&](uint64_t j) {  // k = 7: chunk of job j into buffer j & 1
                const int b = int(j & 1), c = int(j % CHUNKS);
                tc::mbar_expect_tx(&bar_b[b], 2 * CB);
                tc::bulk_g2s(sB + (2 * b) * CB, W.hi + size_t(c) * CB, CB, &bar_b[b]);
                tc::bulk_g2s(sB + (2 * b + 1) * CB, W.lo + size_t(c) * CB, CB, &bar_b[b]);
                if (b) b_armed1++;
                else b_armed0++;
            };
            if (njobs > 0) {
                if constexpr (S::RESIDENT_W) {  // all of W once: hi chunks, then lo chunks
                    tc::mbar_expect_tx(&bar_b[0], 2 * CHUNKS * CB);
                    tc::bulk_g2s(sB, W.hi, CHUNKS * CB, &bar_b[0]);
                    tc::bulk_g2s(sB + CHUNKS * CB, W.lo, CHUNKS * CB, &bar_b[0]);
                    b_armed0 = 1;
                } else {
                    load_w(0);
                }
            }
            for (uint64_t j = 0; j < njobs; j++) {
                if (*fail) break;
                const int b = int(j & 1), c = int(j % CHUNKS);
                const uint64_t t = j / CHUNKS;
                const int a = int(t % NACC);  // accumulator of this tile
                const uint32_t ph = uint32_t(j >> 1) & 1u;
                bool ok = true;
                // the accumulator was drained by the epilogue of tile t - NACC
                if (c == 0 && t >= NACC) ok = tc::mbar_wait(&bar_e[a], uint32_t((t - NACC) / NACC) & 1u, wait_limit);
                if constexpr (S::RESIDENT_W) {
                    if (j == 0) ok = ok && tc::mbar_wait(&bar_b[0], 0u, wait_limit);
                } else {
                    ok = ok && tc::mbar_wait(&bar_b[b], ph, wait_limit);
                }
                ok = ok && tc::mbar_wait(&bar_a[b], ph, wait_limit);
                if (!ok) {
                    *fail = 1;
                    break;
                }
                tc::fence_after_sync();
                if (!skip_mma) {
                    const uint8_t *wh = S::RESIDENT_W ? sB + c * CB : sB + (2 * b) * CB;
                    const uint8_t *wl = S::RESIDENT_W ? sB + (CHUNKS + c) * CB : sB + (2 * b + 1) * CB;
                    const uint32_t wH = tc::smem_u32(wh), wL = tc::smem_u32(wl);
                    const uint32_t dacc = taddr + uint32_t(a * N);
#pragma unroll
                    for (int pr = 0; pr < 3; pr++) {
                        const uint32_t acol = uint32_t(S::COL_A + 64 * b) + (pr == 0 ? 32u : 0u);  // lo*W_hi, hi*W_lo, hi*W_hi
                        const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                        for (int s4 = 0; s4 < 4; s4++)
                            tc::mma_tf32_ts(dacc, taddr + acol + 8 * s4, tc::smem_desc_sw128(w + 32 * s4), IDESC,
                                            (c > 0 || pr > 0 || s4 > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&bar_m[b]);
                    if (b) m_done1++;
                    else m_done0++;
                    if (c == CHUNKS - 1) {
                        tc::mma_commit(&bar_f[a]);
                        if (a) f_done1++;
                        else f_done0++;
                    }
                }
                if constexpr (!S::RESIDENT_W) {
                    // the next W chunk goes into buffer b ^ 1, read by the MMAs of job j - 1
                    if (j + 1 < njobs) {
                        if (j >= 1 && !tc::mbar_wait(&bar_m[b ^ 1], uint32_t((j - 1) >> 1) & 1u, wait_limit)) {
                            *fail = 1;
                            break;
                        }
                        load_w(j + 1);
                    }
                }
            }
            if (*fail) {  // let MMAs and copies in flight land before TMEM and shared memory go away
                atomicOr(&g_tcc_error, 1);
                if (m_done0) tc::mbar_wait(&bar_m[0], (m_done0 - 1) & 1u, wait_limit);
                if (m_done1) tc::mbar_wait(&bar_m[1], (m_done1 - 1) & 1u, wait_limit);
                if (f_done0) tc::mbar_wait(&bar_f[0], (f_done0 - 1) & 1u, wait_limit);
                if (f_done1) tc::mbar_wait(&bar_f[1], (f_done1 - 1) & 1u, wait_limit);
                if (b_armed0) tc::mbar_wait(&bar_b[0], (b_armed0 - 1) & 1u, wait_limit);
                if (b_armed1) tc::mbar_wait(&bar_b[1], (b_armed1 - 1) & 1u, wait_limit);
            }
        }
    } else {
        // ---------------- workers: group g takes the chunks c = g (mod 2)
        const int g = warp >> 2, quarter = warp & 3, row = 32 * quarter + lane;
        const uint32_t lane_addr = taddr + (uint32_t(32 * quarter) << 16);
        const uint64_t g_lane = st.g_lane[lane];
        const uint32_t s_lane = st.s_lane[lane], s_row = st.s_row[lane];
        auto group_off = [&](int c) {
            uint64_t o = 0;
#pragma unroll
            for (int i = 4; i < K; i++)
                if ((c >> (i - 4)) & 1) o += uint64_t(1) << tg.q[i];
            return o;
        };
        auto cube_base = [&](uint64_t tile, int c) {
            return slice_base<K>(tile * 128 + uint64_t(32 * quarter), tg) + group_off(c) + g_lane;
        };
        float2 *my_cubes = cubes + warp * (S::NS * 512);
        float2 *my_out = outc + warp * 512;
        auto copy_async = [&](uint64_t j) {  // job j into stage (j / 2) % NS of this warp's ring
            const float2 *b = sv + cube_base(job_tile(j), int(j % CHUNKS));
            const uint32_t d = tc::smem_u32(my_cubes + ((j >> 1) % S::NS) * 512);
#pragma unroll
            for (int jj = 0; jj < 8; jj++)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + ((s_lane ^ st.s_j[jj]) >> 1) * 16u),
                             "l"(b + st.g_j[jj])
                             : "memory");
        };
        // drain the accumulator of local tile t (this group's 32-column blocks):
        // |y|^2, the norm correction against |x|^2 of the tile's chunks (xt, this
        // group's share), outputs through the warp's output cube
        auto epilogue = [&](uint64_t t, float xt) -> bool {
            const int a = int(t % NACC);
            const uint32_t acc = uint32_t(a * N);
            if (!tc::mbar_wait(&bar_f[a], uint32_t(t / NACC) & 1u, wait_limit)) return false;
            tc::fence_after_sync();
            float ya = 0.f, yb = 0.f;
#pragma unroll 1
            for (int gg = g; gg < CHUNKS; gg += 2) {
                float v[32];
                tc::tmem_ld<32>(lane_addr + acc + 32 * gg, v);
#pragma unroll
                for (int m = 0; m < 16; m++) {
                    ya = fmaf(v[2 * m], v[2 * m], ya);
                    yb = fmaf(v[2 * m + 1], v[2 * m + 1], yb);
                }
            }
            xnorm[g * 128 + row] = xt;
            ynorm[g * 128 + row] = ya + yb;
            mbar_arrive(&bar_q[quarter]);
            if (!tc::mbar_wait(&bar_q[quarter], uint32_t(t) & 1u, wait_limit)) return false;
            const float X = xnorm[row] + xnorm[128 + row], Y = ynorm[row] + ynorm[128 + row];
            float delta = 0.0f;
            if (Y > 0.0f && X > 0.0f) delta = 0.5f * (X - Y) / Y;
            const uint64_t tile = uint64_t(blockIdx.x) + t * gridDim.x;
#pragma unroll 1
            for (int gg = g; gg < CHUNKS; gg += 2) {
                float v[32];
                tc::tmem_ld<32>(lane_addr + acc + 32 * gg, v);
                if (st.pair) {
#pragma unroll
                    for (int m = 0; m < 16; m += 2)
                        reinterpret_cast<float4 *>(my_out)[(s_row ^ st.s_mem[m]) >> 1] =
                            make_float4(fmaf(v[2 * m], delta, v[2 * m]), fmaf(v[2 * m + 1], delta, v[2 * m + 1]),
                                        fmaf(v[2 * m + 2], delta, v[2 * m + 2]),
                                        fmaf(v[2 * m + 3], delta, v[2 * m + 3]));
                } else {
#pragma unroll
                    for (int m = 0; m < 16; m++)
                        my_out[s_row ^ st.s_mem[m]] =
                            make_float2(fmaf(v[2 * m], delta, v[2 * m]), fmaf(v[2 * m + 1], delta, v[2 * m + 1]));
                }
                __syncwarp();
                float2 *gb = sv + cube_base(tile, gg);
                const float4 *s4 = reinterpret_cast<const float4 *>(my_out);
#pragma unroll
                for (int jj = 0; jj < 8; jj++)
                    __stcs(reinterpret_cast<float4 *>(gb + st.g_j[jj]), s4[(s_lane ^ st.s_j[jj]) >> 1]);
                __syncwarp();
            }
            tc::fence_before_sync();
            mbar_arrive(&bar_e[a]);
            return true;
        };
        for (int p = 0; p < S::NS; p++) {
            const uint64_t jp = uint64_t(g) + 2 * uint64_t(p);
            if (jp < njobs) copy_async(jp);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        float xs = 0.f;  // |x|^2 of this group's chunks of the current tile
        for (uint64_t j = uint64_t(g); j < njobs; j += 2) {
            if (*fail) break;
            const int c = int(j % CHUNKS);
            const uint64_t t = j / CHUNKS;
            // A buffer g is free once the MMAs of job j - 2 are done
            if (j >= 2 && !tc::mbar_wait(&bar_m[g], uint32_t((j - 2) >> 1) & 1u, wait_limit)) {
                *fail = 1;
                break;
            }
            tc::fence_after_sync();
            asm volatile("cp.async.wait_group %0;" ::"n"(S::NS - 1) : "memory");
            __syncwarp();
            const float2 *stage = my_cubes + ((j >> 1) % S::NS) * 512;
            float xa = 0.f, xb = 0.f;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float2 x[8];
                if (st.pair) {
#pragma unroll
                    for (int m = 0; m < 8; m += 2) {
                        const float4 v = reinterpret_cast<const float4 *>(stage)[(s_row ^ st.s_mem[h * 8 + m]) >> 1];
                        x[m] = make_float2(v.x, v.y);
                        x[m + 1] = make_float2(v.z, v.w);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 8; m++) x[m] = stage[s_row ^ st.s_mem[h * 8 + m]];
                }
                float v[16];
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    v[2 * m] = tcc_trunc(x[m].x);
                    v[2 * m + 1] = tcc_trunc(x[m].y);
                }
                tc::tmem_st<16>(lane_addr + S::COL_A + 64 * g + 16 * h, v);
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    v[2 * m] = tcc_round(x[m].x - v[2 * m]);
                    v[2 * m + 1] = tcc_round(x[m].y - v[2 * m + 1]);
                }
                tc::tmem_st<16>(lane_addr + S::COL_A + 64 * g + 32 + 16 * h, v);
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    xa = fmaf(x[m].x, x[m].x, xa);
                    xb = fmaf(x[m].y, x[m].y, xb);
                }
            }
            tc::tmem_wait_st();
            tc::fence_before_sync();
            mbar_arrive(&bar_a[g]);
            // the stage of job j is in TMEM now: refill it with this warp's job j + 2 NS
            __syncwarp();
            if (j + 2 * S::NS < njobs) copy_async(j + 2 * S::NS);
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (c == g && t >= 1) {  // first chunk of tile t queued: drain tile t - 1
                const float xt = xs;
                xs = 0.f;
                if (!epilogue(t - 1, xt)) {
                    *fail = 1;
                    break;
                }
            }
            xs += xa + xb;
        }
        if (!*fail && my_tiles > 0 && !epilogue(my_tiles - 1, xs)) *fail = 1;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (*fail && tid == 0) atomicOr(&g_tcc_error, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, S::COLS);
}

// W, staging and output cubes, norms, 14 barriers, TMEM slot and fail flag
template <int K>
size_t tcc_ws_smem_bytes() {
    using S = TccShape<K>;
    return S::W_BYTES + size_t(kWsWorkers) * (S::NS + 1) * 512 * 8 + 2 * 256 * 4 + 14 * 8 + 8;
}

// host-side tf32 rounding (nearest, ties away from zero, as cvt.rna)
float host_tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

template <int K>
cast_status run_tcc(cast_sv *sv, const PreparedGate &g) {
    using S = TccShape<K>;
    constexpr int D = S::D, N = S::N;
    // W^T chunk images: chunk c, row n (output real), column k (input real 32 c + k), in the
    // 128-byte-swizzled K-major layout the MMA reads; W = [[a, -b], [b, a]] blocks of U = a + ib
    std::vector<uint8_t> hi(size_t(S::CHUNKS) * S::CHUNK_BYTES), lo(size_t(S::CHUNKS) * S::CHUNK_BYTES);
    for (int n = 0; n < N; n++)
        for (int col = 0; col < N; col++) {
            const cplx u = g.m[size_t(n >> 1) * D + (col >> 1)];
            double w;
            if ((n & 1) == (col & 1)) w = u.real();
            else if (n & 1) w = u.imag();
            else w = -u.imag();
            const float wh = host_tf32_rna(float(w));
            const float wl = host_tf32_rna(float(w - double(wh)));
            const size_t off = size_t(col >> 5) * S::CHUNK_BYTES + tc::sw128_offset(n, col & 31, N);
            std::memcpy(&hi[off], &wh, 4);
            std::memcpy(&lo[off], &wl, 4);
        }
    const void *dhi = nullptr, *dlo = nullptr;
    cast_status s1 = upload_matrix(sv, hi.data(), hi.size(), &dhi);
    if (s1 != CAST_OK) return s1;
    s1 = upload_matrix(sv, lo.data(), lo.size(), &dlo);
    if (s1 != CAST_OK) return s1;
    TccMat W;
    W.hi = static_cast<const uint8_t *>(dhi);
    W.lo = static_cast<const uint8_t *>(dlo);
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const CubeTables ct = make_cube_tables(g.q, K);
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const uint64_t cap = uint64_t(sm_count_cached());
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    ProfScope ps(sv->stream, "tc_k" + std::to_string(K) + "_c64", 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    const uint32_t inject = take_inject_limit();
    static_assert(K == 6 || K == 7, "the chunked kernel is built for k = 6, 7");
    const size_t smem = tcc_ws_smem_bytes<K>();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tcc_ws<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_dense_tcc_ws<K><<<(unsigned)grid, kWsThreads, smem, sv->stream>>>(
        reinterpret_cast<float2 *>(sv->data), ntiles, tg, W, ct, inject ? inject : kTccWaitLimit, inject ? 1 : 0);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

int tcc_error_flag_take() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tcc_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tcc_error, &zero, sizeof(int));
    }
    return v;
}

bool tcc_eligible(const cast_sv *sv, const PreparedGate &g) {
    return tensor_cores_on() && sv->dt == CAST_C64 && g.cls == CLS_DENSE && g.unitary &&
           (g.k == 7 || (g.k == 6 && kTcc6)) && sv->n >= g.k + 7;
}

cast_status launch_gate_tcc(cast_sv *sv, const PreparedGate &g) {
    if (g.k == 7) return run_tcc<7>(sv, g);
    if (g.k == 6) return run_tcc<6>(sv, g);
    return fail(CAST_ERR_UNSUPPORTED, "the chunked tensor-core path covers k = 6, 7");
}

}  // namespace cast
