// Dense 7-qubit gates on complex64 states with the tcgen05 tensor cores, with
// the K dimension streamed in chunks.
//
// Same GEMM as apply_tc.cu (Eq. 3 batched: a tile of 128 slices times the
// real 2^(k+1) x 2^(k+1) form W of the gate, 3xTF32, fp32 accumulation in
// TMEM, per-slice norm restoration), but W does not fit in shared memory: for
// k = 7 it is 256 x 256 fp32 (256 KB for each of W_hi and W_lo).  The K
// dimension is cut into 8 chunks of 16 members (32 reals):
//   - A (the slice rows) of chunk c is the warp's staged cube for member group
//     c (csrc/cube.cpp: 32 slices x 16 members, coalesced 16-byte cp.async
//     copies, two in flight per warp), split hi/lo in registers and written
//     into one of two TMEM chunk buffers (64 columns each);
//   - B (W^T restricted to the chunk's 32 K columns, hi and lo: 2 x N x 128
//     bytes, N = 2^(k+1) output reals) was laid out on the host as the exact
//     128-byte-swizzled shared-memory image and arrives with two bulk copies
//     (TMA, non-tensor) onto an mbarrier, one chunk ahead of the MMAs that read
//     it (two shared buffers);
//   - the three products of a chunk are 3 x 4 MMAs of M = 128, N, K = 8.
// The template also runs TPC tiles per CTA side by side, sharing every W
// chunk (TPC tile slots of accumulator + A buffers in TMEM); measured for
// k = 6 with two tiles it ran 6% slower than apply_tc.cu's resident-W kernel,
// so only k = 7 (one tile) uses it.
// After the last chunk each accumulator is drained: the row's |y|^2, the norm
// correction against |x|^2 summed over the chunks, and the outputs go back to
// HBM through a per-warp output cube, group by group.
// TMEM per tile slot: accumulator N + two A chunk buffers 2 x 64 columns
// (k = 7: 384 of 512).  One CTA per SM.
//
// Waits on mbarriers are bounded; a CTA that gives up sets the error flag
// (read by the host at its next synchronisation point), waits once more
// (bounded) for its MMAs and bulk copies in flight and frees its TMEM.
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
    static constexpr int TPC = 1;               // tiles per CTA, sharing every W chunk
    static constexpr int NW = 4 * TPC;          // warps: one per TMEM lane quarter per tile
    static constexpr int NT = 32 * NW;
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

template <int K>
__global__ void __launch_bounds__(TccShape<K>::NT, 1)
k_dense_tcc(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg, TccMat W,
            const __grid_constant__ CubeTables st, uint32_t wait_limit, int skip_mma) {
    using S = TccShape<K>;
    constexpr int N = S::N, CHUNKS = S::CHUNKS, TPC = S::TPC, NW = S::NW;
    constexpr uint32_t CB = S::CHUNK_BYTES;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, N);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = base;                                             // [2 buffers][hi, lo] x CB
    float2 *cubes = reinterpret_cast<float2 *>(base + 4 * CB);     // [NW warps][2 stages][512]
    float2 *outc = cubes + NW * 2 * 512;                            // [NW warps][512]
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(outc + NW * 512);  // [2] W chunk landed
    uint64_t *bar_m = bar_b + 2;                                               // [2] MMAs of a chunk done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&bar_b[0], 1);
        tc::mbar_init(&bar_b[1], 1);
        tc::mbar_init(&bar_m[0], 1);
        tc::mbar_init(&bar_m[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, S::COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const int slot = warp >> 2, quarter = warp & 3;  // tile slot of this warp, its TMEM lane quarter
    const uint32_t tcol = uint32_t(slot * S::SLOT);   // accumulator of the slot; A buffers at + N
    const uint32_t lane_addr = taddr + (uint32_t(32 * quarter) << 16) + tcol;

    // tile groups (TPC tiles each) of this CTA; job j = (group j / CHUNKS, chunk j % CHUNKS)
    const uint64_t ngroups = ntiles / TPC;
    const uint64_t my_groups = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t njobs = my_groups * CHUNKS;
    const uint64_t g_lane = st.g_lane[lane];
    const uint32_t s_lane = st.s_lane[lane], s_row = st.s_row[lane];
    auto job_tile = [&](uint64_t j) { return (uint64_t(blockIdx.x) + (j / CHUNKS) * gridDim.x) * TPC + slot; };
    // member offset of member group c (targets q4 .. q_{K-1})
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
    float2 *my_cubes = cubes + warp * (2 * 512);
    float2 *my_out = outc + warp * 512;
    auto copy_async = [&](uint64_t j) {
        const float2 *b = sv + cube_base(job_tile(j), int(j % CHUNKS));
        const uint32_t d = tc::smem_u32(my_cubes + (j & 1) * 512);
#pragma unroll
        for (int jj = 0; jj < 8; jj++)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + ((s_lane ^ st.s_j[jj]) >> 1) * 16u),
                         "l"(b + st.g_j[jj])
                         : "memory");
    };
    // thread 0: W chunk of job j into shared buffer j & 1
    uint32_t b_armed0 = 0, b_armed1 = 0, m_done0 = 0, m_done1 = 0;  // phases started (thread 0)
    auto load_w = [&](uint64_t j) {
        const int b = int(j & 1), c = int(j % CHUNKS);
        tc::mbar_expect_tx(&bar_b[b], 2 * CB);
        tc::bulk_g2s(sB + (2 * b) * CB, W.hi + size_t(c) * CB, CB, &bar_b[b]);
        tc::bulk_g2s(sB + (2 * b + 1) * CB, W.lo + size_t(c) * CB, CB, &bar_b[b]);
        if (b) b_armed1++;
        else b_armed0++;
    };

    for (uint64_t jp = 0; jp < 2; jp++) {  // two cube stages in flight (empty groups keep the count)
        if (jp < njobs) copy_async(jp);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if (tid == 0 && njobs > 0) load_w(0);

    bool failed = false;
    float xs = 0.f;
    uint64_t j = 0;
    for (; j < njobs; j++) {
        const int b = int(j & 1), c = int(j % CHUNKS);
        // A chunk buffer b is free once the MMAs of job j - 2 are done
        if (j >= 2 && !tc::mbar_wait(&bar_m[b], uint32_t((j - 2) >> 1) & 1u, wait_limit)) failed = true;
        tc::fence_after_sync();
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncwarp();
        const float2 *stage = my_cubes + b * 512;
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
            tc::tmem_st<16>(lane_addr + N + 64 * b + 16 * h, v);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                v[2 * m] = tcc_round(x[m].x - v[2 * m]);
                v[2 * m + 1] = tcc_round(x[m].y - v[2 * m + 1]);
            }
            tc::tmem_st<16>(lane_addr + N + 64 * b + 32 + 16 * h, v);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                xa = fmaf(x[m].x, x[m].x, xa);
                xb = fmaf(x[m].y, x[m].y, xb);
            }
        }
        xs += xa + xb;
        tc::tmem_wait_st();
        tc::fence_before_sync();
        if (__syncthreads_or(failed)) break;
        tc::fence_after_sync();
        // the cube stage of job j is in TMEM now: refill it with job j + 2
        __syncwarp();
        if (j + 2 < njobs) copy_async(j + 2);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (tid == 0) {
            if (!tc::mbar_wait(&bar_b[b], uint32_t(j >> 1) & 1u, wait_limit)) failed = true;
            if (!failed && !skip_mma) {
                tc::fence_after_sync();
                const uint32_t wH = tc::smem_u32(sB + (2 * b) * CB);
                const uint32_t wL = tc::smem_u32(sB + (2 * b + 1) * CB);
#pragma unroll
                for (int t = 0; t < TPC; t++) {
                    const uint32_t acc_t = taddr + uint32_t(t * S::SLOT);
#pragma unroll
                    for (int pr = 0; pr < 3; pr++) {
                        const uint32_t acol = uint32_t(N + 64 * b) + (pr == 0 ? 32u : 0u);  // lo*W_hi, hi*W_lo, hi*W_hi
                        const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                        for (int s4 = 0; s4 < 4; s4++)
                            tc::mma_tf32_ts(acc_t, acc_t + acol + 8 * s4, tc::smem_desc_sw128(w + 32 * s4), IDESC,
                                            (c > 0 || pr > 0 || s4 > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&bar_m[b]);
                if (b) m_done1++;
                else m_done0++;
            }
            // the W chunk of job j + 1 goes into buffer b ^ 1, read by the MMAs of job j - 1
            if (!failed && j + 1 < njobs) {
                if (j >= 1 && !tc::mbar_wait(&bar_m[b ^ 1], uint32_t((j - 1) >> 1) & 1u, wait_limit)) failed = true;
                if (!failed) load_w(j + 1);
            }
        }
        __syncwarp();
        if (c == CHUNKS - 1) {
            // ---- epilogue of the tile: the accumulator holds all 256 outputs of each row
            if (!tc::mbar_wait(&bar_m[b], uint32_t(j >> 1) & 1u, wait_limit)) failed = true;
            if (__syncthreads_or(failed)) break;
            tc::fence_after_sync();
            float ya = 0.f, yb = 0.f;
#pragma unroll 1
            for (int g = 0; g < CHUNKS; g++) {
                float v[32];
                tc::tmem_ld<32>(lane_addr + 32 * g, v);
#pragma unroll
                for (int m = 0; m < 16; m++) {
                    ya = fmaf(v[2 * m], v[2 * m], ya);
                    yb = fmaf(v[2 * m + 1], v[2 * m + 1], yb);
                }
            }
            const float Y = ya + yb, X = xs;
            float delta = 0.0f;
            if (Y > 0.0f && X > 0.0f) delta = 0.5f * (X - Y) / Y;
            const uint64_t tile = job_tile(j);
#pragma unroll 1
            for (int g = 0; g < CHUNKS; g++) {
                float v[32];
                tc::tmem_ld<32>(lane_addr + 32 * g, v);
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
                float2 *gb = sv + cube_base(tile, g);
                const float4 *s4 = reinterpret_cast<const float4 *>(my_out);
#pragma unroll
                for (int jj = 0; jj < 8; jj++)
                    __stcs(reinterpret_cast<float4 *>(gb + st.g_j[jj]), s4[(s_lane ^ st.s_j[jj]) >> 1]);
                __syncwarp();
            }
            xs = 0.f;
            tc::fence_before_sync();
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    failed = __syncthreads_or(failed);
    if (failed) {
        if (tid == 0) {
            atomicOr(&g_tcc_error, 1);
            // let MMAs and bulk copies in flight land before TMEM and shared memory go away
            if (m_done0) tc::mbar_wait(&bar_m[0], (m_done0 - 1) & 1u, wait_limit);
            if (m_done1) tc::mbar_wait(&bar_m[1], (m_done1 - 1) & 1u, wait_limit);
            if (b_armed0) tc::mbar_wait(&bar_b[0], (b_armed0 - 1) & 1u, wait_limit);
            if (b_armed1) tc::mbar_wait(&bar_b[1], (b_armed1 - 1) & 1u, wait_limit);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, S::COLS);
}

float host_tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

template <int K>
size_t tcc_smem_bytes() {
    using S = TccShape<K>;
    return 1024 + 4 * size_t(S::CHUNK_BYTES) + size_t(S::NW * 2 * 512 + S::NW * 512) * 8 + 64;
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
    const size_t smem = tcc_smem_bytes<K>();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tcc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t cap = uint64_t(sm_count_cached()), groups = ntiles / S::TPC;
    const uint64_t grid = groups < cap ? groups : cap;
    ProfScope ps(sv->stream, "tc_k" + std::to_string(K) + "_c64", 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    const uint32_t inject = take_inject_limit();
    k_dense_tcc<K><<<(unsigned)grid, S::NT, smem, sv->stream>>>(reinterpret_cast<float2 *>(sv->data), ntiles, tg, W,
                                                                ct, inject ? inject : kTccWaitLimit, inject ? 1 : 0);
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
