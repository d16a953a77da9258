// Dense 7-qubit gates on complex64 states with the tcgen05 tensor cores.
//
// Same GEMM as apply_tc.cu (Eq. 3 batched: a tile of 128 slices times the
// real 2^(k+1) x 2^(k+1) form W of the gate, 3xTF32, fp32 accumulation in
// TMEM, per-slice norm restoration), but for k = 7 neither operand fits at
// once: W is 256 x 256 fp32 (256 KB for each of W_hi and W_lo) and a slice row
// is 256 reals.  The K dimension is therefore cut into 8 chunks of 16 members
// (32 reals):
//   - A (the slice rows) of chunk c is the warp's staged cube for member group
//     c (csrc/cube.cpp: 32 slices x 16 members, coalesced 16-byte cp.async
//     copies, two in flight per warp), split hi/lo in registers and written
//     into one of two TMEM chunk buffers (64 columns each);
//   - B (W^T restricted to the chunk's 32 K columns, hi and lo: 64 KB) was laid
//     out on the host as the exact 128-byte-swizzled shared-memory image and
//     arrives with two bulk copies (TMA, non-tensor) onto an mbarrier, one
//     chunk ahead of the MMAs that read it (two shared buffers);
//   - the three products of a chunk are 3 x 4 MMAs of M = 128, N = 256, K = 8
//     into one 256-column accumulator.
// After the 8th chunk the accumulator is drained: the row's |y|^2 (all 256
// columns), the norm correction against |x|^2 summed over the chunks, and the
// outputs go back to HBM through a per-warp output cube, group by group.
// TMEM: accumulator 256 + two A chunk buffers 2 x 64 = 384 columns (512
// allocated, one CTA per SM).  Shared memory: 128 KB of W chunks, 32 KB of
// input cubes, 16 KB of output cubes.
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

int tc7_error_flag_take();

namespace {

__device__ int g_tc7_error;

constexpr int kT7Threads = 128;                 // 4 warps, one per TMEM lane quarter
constexpr int kT7Chunks = 8;                    // K chunks of 16 members (32 reals)
constexpr uint32_t kT7ChunkBytes = 256u * 128u;  // W^T chunk, hi or lo: 256 rows x 32 fp32
constexpr uint32_t kT7ColA = 256;               // A chunk buffer b: hi at 256 + 64 b, lo at + 32
constexpr uint32_t kT7Cols = 512;
constexpr uint32_t kT7WaitLimit = 1u << 26;

struct T7Mat {
    const uint8_t *hi;  // 8 chunk images of kT7ChunkBytes
    const uint8_t *lo;
};

__device__ __forceinline__ float t7_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
__device__ __forceinline__ float t7_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__global__ void __launch_bounds__(kT7Threads, 1)
k_dense_tc7(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg, T7Mat W,
            const __grid_constant__ CubeTables st, uint32_t wait_limit, int skip_mma) {
    constexpr uint32_t IDESC = tc::idesc_tf32(128, 256);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sB = base;                                                        // [2 buffers][hi, lo] x 32 KB
    float2 *cubes = reinterpret_cast<float2 *>(base + 4 * kT7ChunkBytes);     // [4 warps][2 stages][512]
    float2 *outc = cubes + 4 * 2 * 512;                                        // [4 warps][512]
    uint64_t *bar_b = reinterpret_cast<uint64_t *>(outc + 4 * 512);            // [2] W chunk landed
    uint64_t *bar_m = bar_b + 2;                                               // [2] MMAs of a chunk done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_m + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&bar_b[0], 1);
        tc::mbar_init(&bar_b[1], 1);
        tc::mbar_init(&bar_m[0], 1);
        tc::mbar_init(&bar_m[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, kT7Cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t lane_addr = taddr + (uint32_t(32 * warp) << 16);

    const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t njobs = my_tiles * kT7Chunks;  // job j: tile blockIdx.x + (j / 8) * gridDim.x, chunk j % 8
    const uint64_t g_lane = st.g_lane[lane];
    const uint32_t s_lane = st.s_lane[lane], s_row = st.s_row[lane];
    auto job_tile = [&](uint64_t j) { return uint64_t(blockIdx.x) + (j >> 3) * gridDim.x; };
    // member offset of member group c (targets q4, q5, q6)
    auto group_off = [&](int c) {
        uint64_t o = 0;
#pragma unroll
        for (int i = 4; i < 7; i++)
            if ((c >> (i - 4)) & 1) o += uint64_t(1) << tg.q[i];
        return o;
    };
    auto cube_base = [&](uint64_t tile, int c) {
        return slice_base<7>(tile * 128 + uint64_t(32 * warp), tg) + group_off(c) + g_lane;
    };
    float2 *my_cubes = cubes + warp * (2 * 512);
    float2 *my_out = outc + warp * 512;
    auto copy_async = [&](uint64_t j) {
        const float2 *b = sv + cube_base(job_tile(j), int(j & 7));
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
        const int b = int(j & 1), c = int(j & 7);
        tc::mbar_expect_tx(&bar_b[b], 2 * kT7ChunkBytes);
        tc::bulk_g2s(sB + (2 * b) * kT7ChunkBytes, W.hi + size_t(c) * kT7ChunkBytes, kT7ChunkBytes, &bar_b[b]);
        tc::bulk_g2s(sB + (2 * b + 1) * kT7ChunkBytes, W.lo + size_t(c) * kT7ChunkBytes, kT7ChunkBytes, &bar_b[b]);
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
        const int b = int(j & 1), c = int(j & 7);
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
                v[2 * m] = t7_trunc(x[m].x);
                v[2 * m + 1] = t7_trunc(x[m].y);
            }
            tc::tmem_st<16>(lane_addr + kT7ColA + 64 * b + 16 * h, v);
#pragma unroll
            for (int m = 0; m < 8; m++) {
                v[2 * m] = t7_round(x[m].x - v[2 * m]);
                v[2 * m + 1] = t7_round(x[m].y - v[2 * m + 1]);
            }
            tc::tmem_st<16>(lane_addr + kT7ColA + 64 * b + 32 + 16 * h, v);
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
                const uint32_t wH = tc::smem_u32(sB + (2 * b) * kT7ChunkBytes);
                const uint32_t wL = tc::smem_u32(sB + (2 * b + 1) * kT7ChunkBytes);
#pragma unroll
                for (int pr = 0; pr < 3; pr++) {
                    const uint32_t acol = kT7ColA + 64 * b + (pr == 0 ? 32u : 0u);  // lo*W_hi, hi*W_lo, hi*W_hi
                    const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                    for (int s = 0; s < 4; s++)
                        tc::mma_tf32_ts(taddr, taddr + acol + 8 * s, tc::smem_desc_sw128(w + 32 * s), IDESC,
                                        (c > 0 || pr > 0 || s > 0) ? 1u : 0u);
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
        if (c == kT7Chunks - 1) {
            // ---- epilogue of the tile: the accumulator holds all 256 outputs of each row
            if (!tc::mbar_wait(&bar_m[b], uint32_t(j >> 1) & 1u, wait_limit)) failed = true;
            if (__syncthreads_or(failed)) break;
            tc::fence_after_sync();
            float ya = 0.f, yb = 0.f;
#pragma unroll 1
            for (int g = 0; g < 8; g++) {
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
            for (int g = 0; g < 8; g++) {
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
            atomicOr(&g_tc7_error, 1);
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
    if (warp == 0) tc::tmem_dealloc(taddr, kT7Cols);
}

float host_tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

size_t tc7_smem_bytes() { return 1024 + 4 * size_t(kT7ChunkBytes) + (4 * 2 * 512 + 4 * 512) * 8 + 64; }

}  // namespace

int tc7_error_flag_take() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc7_error, sizeof(int)) != cudaSuccess) return 0;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tc7_error, &zero, sizeof(int));
    }
    return v;
}

bool tc7_eligible(const cast_sv *sv, const PreparedGate &g) {
    return tensor_mode_tf32x3() && sv->dt == CAST_C64 && g.cls == CLS_DENSE && g.unitary && g.k == 7 &&
           sv->n >= 14;
}

cast_status launch_gate_tc7(cast_sv *sv, const PreparedGate &g) {
    constexpr int D = 128;
    // W^T chunk images: chunk c, row n (output real), column k (input real 32 c + k), in the
    // 128-byte-swizzled K-major layout the MMA reads; W = [[a, -b], [b, a]] blocks of U = a + ib
    std::vector<uint8_t> hi(size_t(kT7Chunks) * kT7ChunkBytes), lo(size_t(kT7Chunks) * kT7ChunkBytes);
    for (int n = 0; n < 2 * D; n++)
        for (int col = 0; col < 2 * D; col++) {
            const cplx u = g.m[size_t(n >> 1) * D + (col >> 1)];
            double w;
            if ((n & 1) == (col & 1)) w = u.real();
            else if (n & 1) w = u.imag();
            else w = -u.imag();
            const float wh = host_tf32_rna(float(w));
            const float wl = host_tf32_rna(float(w - double(wh)));
            const size_t off = size_t(col >> 5) * kT7ChunkBytes + tc::sw128_offset(n, col & 31, 256);
            std::memcpy(&hi[off], &wh, 4);
            std::memcpy(&lo[off], &wl, 4);
        }
    const void *dhi = nullptr, *dlo = nullptr;
    cast_status s1 = upload_matrix(sv, hi.data(), hi.size(), &dhi);
    if (s1 != CAST_OK) return s1;
    s1 = upload_matrix(sv, lo.data(), lo.size(), &dlo);
    if (s1 != CAST_OK) return s1;
    T7Mat W;
    W.hi = static_cast<const uint8_t *>(dhi);
    W.lo = static_cast<const uint8_t *>(dlo);
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = g.q[i];
    const CubeTables ct = make_cube_tables(g.q, 7);
    const uint64_t ntiles = uint64_t(1) << (sv->n - 14);
    const size_t smem = tc7_smem_bytes();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tc7, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t cap = uint64_t(sm_count_cached());
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    ProfScope ps(sv->stream, "tc_k7_c64", 16.0 * double(uint64_t(1) << sv->n), 8.0 * double(uint64_t(1) << (sv->n + 7)));
    const uint32_t inject = take_inject_limit();
    k_dense_tc7<<<(unsigned)grid, kT7Threads, smem, sv->stream>>>(reinterpret_cast<float2 *>(sv->data), ntiles, tg, W,
                                                                  ct, inject ? inject : kT7WaitLimit, inject ? 1 : 0);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace cast
