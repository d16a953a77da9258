// Dense 7-qubit gates on complex64 states with the tcgen05 tensor cores, with
// the K dimension streamed in chunks.
//
// Same GEMM as apply_tc.cu (Eq. 3 batched: a tile of 128 slices times the
// real 2^(k+1) x 2^(k+1) form W of the gate, 3xTF32, fp32 accumulation in
// TMEM, per-slice norm restoration), but W does not fit in shared memory: for
// k = 7 it is 256 x 256 fp32 (256 KB for each of W_hi and W_lo).  The K
// dimension is cut into 8 chunks of 16 members (32 reals):
//   - A (the slice rows) of chunk c is the staged cube of member group c
//     (csrc/cube.cpp: 32 slices x 16 members per warp, coalesced 16-byte
//     cp.async copies, two in flight per warp), split hi/lo in registers and
//     written into one of two TMEM chunk buffers (64 columns each);
//   - B (W^T restricted to the chunk's 32 K columns, hi and lo: 64 KB) was laid
//     out on the host as the exact 128-byte-swizzled shared-memory image and
//     arrives with two bulk copies (TMA, non-tensor) onto an mbarrier, one
//     chunk ahead of the MMAs that read it (two shared buffers);
//   - the three products of a chunk are 3 x 4 MMAs of M = 128, N = 256, K = 8
//     into one 256-column accumulator.
// Eight worker warps in two groups take alternate chunks; a ninth warp issues
// the MMAs and the W copies (details at the kernel).  After the last chunk
// both groups drain the accumulator: the row's |y|^2, the norm correction
// against |x|^2 summed over the chunks, and the outputs go back to HBM through
// per-warp output cubes.  TMEM: accumulator 256 + two A buffers 2 x 64 = 384
// of 512 columns; shared memory 226 KB; one CTA per SM.
//
// A four-warp form of this kernel (every warp on every chunk) ran 10% slower;
// a two-tile form for k = 6 ran 6% slower than apply_tc.cu's resident-W kernel.
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

template <int K>
struct TccShape {
    static constexpr int D = 1 << K;            // slice members
    static constexpr int N = 2 * D;             // output reals = accumulator columns (MMA N)
    static constexpr int CHUNKS = D / 16;       // K chunks of 16 members (32 reals)
    static constexpr int TPC = 1;               // tiles per CTA
    static constexpr int SLOT = N + 128;        // TMEM columns of a tile: accumulator, 2 A buffers
    static constexpr uint32_t CHUNK_BYTES = uint32_t(N) * 128u;  // W^T chunk, hi or lo
    static constexpr int COLS = 512;
    static_assert(TPC * SLOT <= COLS, "TMEM columns");
};
constexpr uint32_t kTccWaitLimit = 1u << 26;

struct TccMat {
    const uint8_t *hi;  // CHUNKS chunk images of CHUNK_BYTES
    const uint8_t *lo;
};

__device__ __forceinline__ float tcc_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ float tcc_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Warp-specialised form for k = 7: the same chunks, but eight worker warps in
// two groups of four take alternate chunks (group g owns TMEM A buffer g), so
// one group prepares a chunk while the MMAs of the other group's chunk run, and
// a ninth warp only waits on mbarriers, issues the MMAs and streams the W
// chunks.  Both groups drain the accumulator (alternate 32-column blocks,
// norms exchanged per lane quarter through an mbarrier).  Barriers:
//   bar_a[g]  A chunk of group g in TMEM (128 arrivals)     phase: job / 2
//   bar_b[b]  W chunk in shared buffer b (bulk-copy bytes)   phase: job / 2
//   bar_m[b]  MMAs of the chunk in buffer b done (commit)    phase: job / 2
//   bar_f     MMAs of a tile's last chunk done (commit)      phase: tile
//   bar_e     accumulator drained (256 arrivals)            phase: tile
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

__global__ void __launch_bounds__(kWsThreads, 1)
k_dense_tcc_ws(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg, TccMat W,
               const __grid_constant__ CubeTables st, uint32_t wait_limit, int skip_mma) {
    using S = TccShape<7>;
    constexpr int N = S::N, CHUNKS = S::CHUNKS;
    constexpr uint32_t CB = S::CHUNK_BYTES;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, N);
    extern __shared__ __align__(1024) uint8_t ws_smem[];
    if (tc::smem_u32(ws_smem) & 1023u) {  // the W images need 1024-byte alignment
        if (threadIdx.x == 0) atomicOr(&g_tcc_error, 2);
        return;
    }
    uint8_t *sB = ws_smem;                                               // [2 buffers][hi, lo] x 32 KB
    float2 *cubes = reinterpret_cast<float2 *>(ws_smem + 4 * CB);       // [8 warps][2 stages][512]
    float2 *outc = cubes + kWsWorkers * 2 * 512;                         // [8 warps][512]
    float *xnorm = reinterpret_cast<float *>(outc + kWsWorkers * 512);  // [2 groups][128]
    float *ynorm = xnorm + 256;                                          // [2 groups][128]
    uint64_t *bar_a = reinterpret_cast<uint64_t *>(ynorm + 256);
    uint64_t *bar_b = bar_a + 2, *bar_m = bar_a + 4, *bar_e = bar_a + 6, *bar_q = bar_a + 7, *bar_f = bar_a + 11;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_a + 12);
    volatile int *fail = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&bar_a[i], 128);
            tc::mbar_init(&bar_b[i], 1);
            tc::mbar_init(&bar_m[i], 1);
        }
        tc::mbar_init(bar_e, 256);
        tc::mbar_init(bar_f, 1);
        for (int q = 0; q < 4; q++) tc::mbar_init(&bar_q[q], 64);
        *fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, S::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t njobs = my_tiles * CHUNKS;  // job j: tile blockIdx.x + (j / 8) gridDim.x, chunk j % 8
    auto job_tile = [&](uint64_t j) { return uint64_t(blockIdx.x) + (j / CHUNKS) * gridDim.x; };

    if (warp == kWsWorkers) {
        // ---------------- control: MMA issue and W chunk copies (one thread)
        if (lane == 0) {
            uint32_t m_done0 = 0, m_done1 = 0, b_armed0 = 0, b_armed1 = 0, f_done = 0;
            auto load_w = [&](uint64_t j) {
                const int b = int(j & 1), c = int(j % CHUNKS);
                tc::mbar_expect_tx(&bar_b[b], 2 * CB);
                tc::bulk_g2s(sB + (2 * b) * CB, W.hi + size_t(c) * CB, CB, &bar_b[b]);
                tc::bulk_g2s(sB + (2 * b + 1) * CB, W.lo + size_t(c) * CB, CB, &bar_b[b]);
                if (b) b_armed1++;
                else b_armed0++;
            };
            if (njobs > 0) load_w(0);
            for (uint64_t j = 0; j < njobs; j++) {
                if (*fail) break;
                const int b = int(j & 1), c = int(j % CHUNKS);
                const uint32_t ph = uint32_t(j >> 1) & 1u;
                bool ok = true;
                if (c == 0 && j >= CHUNKS) ok = tc::mbar_wait(bar_e, uint32_t(j / CHUNKS - 1) & 1u, wait_limit);
                ok = ok && tc::mbar_wait(&bar_b[b], ph, wait_limit);
                ok = ok && tc::mbar_wait(&bar_a[b], ph, wait_limit);
                if (!ok) {
                    *fail = 1;
                    break;
                }
                tc::fence_after_sync();
                if (!skip_mma) {
                    const uint32_t wH = tc::smem_u32(sB + (2 * b) * CB), wL = tc::smem_u32(sB + (2 * b + 1) * CB);
#pragma unroll
                    for (int pr = 0; pr < 3; pr++) {
                        const uint32_t acol = uint32_t(N + 64 * b) + (pr == 0 ? 32u : 0u);  // lo*W_hi, hi*W_lo, hi*W_hi
                        const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                        for (int s4 = 0; s4 < 4; s4++)
                            tc::mma_tf32_ts(taddr, taddr + acol + 8 * s4, tc::smem_desc_sw128(w + 32 * s4), IDESC,
                                            (c > 0 || pr > 0 || s4 > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&bar_m[b]);
                    if (b) m_done1++;
                    else m_done0++;
                    if (c == CHUNKS - 1) {
                        tc::mma_commit(bar_f);
                        f_done++;
                    }
                }
                // the next W chunk goes into buffer b ^ 1, read by the MMAs of job j - 1
                if (j + 1 < njobs) {
                    if (j >= 1 && !tc::mbar_wait(&bar_m[b ^ 1], uint32_t((j - 1) >> 1) & 1u, wait_limit)) {
                        *fail = 1;
                        break;
                    }
                    load_w(j + 1);
                }
            }
            if (*fail) {  // let MMAs and copies in flight land before TMEM and shared memory go away
                atomicOr(&g_tcc_error, 1);
                if (m_done0) tc::mbar_wait(&bar_m[0], (m_done0 - 1) & 1u, wait_limit);
                if (m_done1) tc::mbar_wait(&bar_m[1], (m_done1 - 1) & 1u, wait_limit);
                if (f_done) tc::mbar_wait(bar_f, (f_done - 1) & 1u, wait_limit);
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
            for (int i = 4; i < 7; i++)
                if ((c >> (i - 4)) & 1) o += uint64_t(1) << tg.q[i];
            return o;
        };
        auto cube_base = [&](uint64_t tile, int c) {
            return slice_base<7>(tile * 128 + uint64_t(32 * quarter), tg) + group_off(c) + g_lane;
        };
        float2 *my_cubes = cubes + warp * (2 * 512);
        float2 *my_out = outc + warp * 512;
        auto copy_async = [&](uint64_t j) {  // job j into stage (j / 2) & 1 of this warp's ring
            const float2 *b = sv + cube_base(job_tile(j), int(j % CHUNKS));
            const uint32_t d = tc::smem_u32(my_cubes + ((j >> 1) & 1) * 512);
#pragma unroll
            for (int jj = 0; jj < 8; jj++)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + ((s_lane ^ st.s_j[jj]) >> 1) * 16u),
                             "l"(b + st.g_j[jj])
                             : "memory");
        };
        for (int p = 0; p < 2; p++) {
            const uint64_t jp = uint64_t(g) + 2 * uint64_t(p);
            if (jp < njobs) copy_async(jp);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        float xs = 0.f;
        for (uint64_t j = uint64_t(g); j < njobs; j += 2) {
            if (*fail) break;
            const int c = int(j % CHUNKS);
            // A buffer g is free once the MMAs of job j - 2 are done
            if (j >= 2 && !tc::mbar_wait(&bar_m[g], uint32_t((j - 2) >> 1) & 1u, wait_limit)) {
                *fail = 1;
                break;
            }
            tc::fence_after_sync();
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
            const float2 *stage = my_cubes + ((j >> 1) & 1) * 512;
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
                tc::tmem_st<16>(lane_addr + N + 64 * g + 16 * h, v);
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    v[2 * m] = tcc_round(x[m].x - v[2 * m]);
                    v[2 * m + 1] = tcc_round(x[m].y - v[2 * m + 1]);
                }
                tc::tmem_st<16>(lane_addr + N + 64 * g + 32 + 16 * h, v);
#pragma unroll
                for (int m = 0; m < 8; m++) {
                    xa = fmaf(x[m].x, x[m].x, xa);
                    xb = fmaf(x[m].y, x[m].y, xb);
                }
            }
            xs += xa + xb;
            tc::tmem_wait_st();
            tc::fence_before_sync();
            mbar_arrive(&bar_a[g]);
            // the stage of job j is in TMEM now: refill it with this warp's job j + 4
            __syncwarp();
            if (j + 4 < njobs) copy_async(j + 4);
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (c == CHUNKS - 2 + g) {
                // ---- epilogue of the tile, shared by the two groups
                const uint32_t tph = uint32_t(j / CHUNKS) & 1u;
                if (!tc::mbar_wait(bar_f, tph, wait_limit)) {
                    *fail = 1;
                    break;
                }
                tc::fence_after_sync();
                float ya = 0.f, yb = 0.f;
#pragma unroll 1
                for (int gg = g; gg < CHUNKS; gg += 2) {
                    float v[32];
                    tc::tmem_ld<32>(lane_addr + 32 * gg, v);
#pragma unroll
                    for (int m = 0; m < 16; m++) {
                        ya = fmaf(v[2 * m], v[2 * m], ya);
                        yb = fmaf(v[2 * m + 1], v[2 * m + 1], yb);
                    }
                }
                xnorm[g * 128 + row] = xs;
                ynorm[g * 128 + row] = ya + yb;
                mbar_arrive(&bar_q[quarter]);
                if (!tc::mbar_wait(&bar_q[quarter], tph, wait_limit)) {
                    *fail = 1;
                    break;
                }
                const float X = xnorm[row] + xnorm[128 + row], Y = ynorm[row] + ynorm[128 + row];
                float delta = 0.0f;
                if (Y > 0.0f && X > 0.0f) delta = 0.5f * (X - Y) / Y;
                const uint64_t tile = job_tile(j);
#pragma unroll 1
                for (int gg = g; gg < CHUNKS; gg += 2) {
                    float v[32];
                    tc::tmem_ld<32>(lane_addr + 32 * gg, v);
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
                xs = 0.f;
                tc::fence_before_sync();
                mbar_arrive(bar_e);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (*fail && tid == 0) atomicOr(&g_tcc_error, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, S::COLS);
}

size_t tcc_ws_smem_bytes() {
    using S = TccShape<7>;
    return 4 * size_t(S::CHUNK_BYTES) + size_t(kWsWorkers) * 3 * 512 * 8 + 2 * 256 * 4 + 12 * 8 + 8;
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
    const uint64_t cap = uint64_t(sm_count_cached()), groups = ntiles / S::TPC;
    const uint64_t grid = groups < cap ? groups : cap;
    ProfScope ps(sv->stream, "tc_k" + std::to_string(K) + "_c64", 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    const uint32_t inject = take_inject_limit();
    static_assert(K == 7, "the chunked kernel is built for k = 7");
    const size_t smem = tcc_ws_smem_bytes();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tcc_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_dense_tcc_ws<<<(unsigned)grid, kWsThreads, smem, sv->stream>>>(
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
    return tensor_mode_tf32x3() && sv->dt == CAST_C64 && g.cls == CLS_DENSE && g.unitary && g.k == 7 &&
           sv->n >= 14;
}

cast_status launch_gate_tcc(cast_sv *sv, const PreparedGate &g) {
    if (g.k == 7) return run_tcc<7>(sv, g);
    return fail(CAST_ERR_UNSUPPORTED, "the chunked tensor-core path covers k = 7");
}

}  // namespace cast
