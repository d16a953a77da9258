// Dense k-qubit gates on complex64 states with the tcgen05 tensor cores
// (k = 4, 5).
//
// The 2^(n-k) matrix-vector products of Eq. 3 are batched into GEMMs.  With an
// interleaved (re, im) slice written as a real vector of 2^(k+1) entries, the
// gate is the real matrix W of 2x2 blocks [[a, -b], [b, a]] (U = a + ib), and
// a tile of 128 slices is the product
//     Y^T (128 x 2^(k+1)) = X^T (128 x 2^(k+1)) * W^T,
// one tcgen05.mma chain with M = 128 (TMEM lane = slice), N = K = 2^(k+1).
//
// Precision: 3xTF32.  Each fp32 operand x is split into hi = tf32(x) and
// lo = x - hi (exact); the three products lo*W_hi + hi*W_lo + hi*W_hi are
// accumulated in fp32 in TMEM, giving fp32-class accuracy (the dropped lo*lo
// term and the truncation of lo are ~2^-22 relative).
//
// Tile: the k target bits plus the 7 lowest non-target bits.  Every bit below
// 7 is then a tile bit, so a tile is made of contiguous runs of >= 128
// amplitudes: global loads and stores are coalesced float4 accesses.  Per tile:
//   load (registers, prefetched one tile ahead) -> split hi/lo -> shared
//   memory in the SW128 K-major layout -> 3 x 2^(k+1)/8 MMAs issued by one
//   thread -> commit to an mbarrier -> TMEM -> registers (thread = slice) ->
//   XOR-swizzled shared staging in natural index order -> coalesced stores.
// The matrix (W_hi, W_lo) is built in shared memory once per CTA from the
// hi/lo split of U passed in the launch parameters.
//
// Waits on the mbarrier are bounded; a CTA that gives up sets an error bit in
// g_tc_error (read by the host at its next synchronisation point), stops its
// tile loop, waits once more (bounded) for its MMAs and frees its TMEM.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>

#include "device.cuh"
#include "internal.h"
#include "tc.cuh"

namespace cast {

namespace {

__device__ int g_tc_error;
std::atomic<int> g_tensor_mode{CAST_TC_TF32X3};

constexpr uint32_t kWaitLimit = 1u << 26;

template <int K>
struct TcMat {
    float2 hi[1 << K][1 << K];
    float2 lo[1 << K][1 << K];
};

struct TcGeom {
    int ntb;          // number of tile bits, k + 7
    int tb[CAST_MAX_K + 7];  // tile bits, ascending
    int L;            // tile bits 0..L-1 are the index bits 0..L-1
    uint32_t tmask;   // positions (in the tile-local index) holding targets
};

__device__ __forceinline__ uint64_t tile_base(uint64_t t, const TcGeom &g) {
    for (int i = 0; i < g.ntb; i++) {
        const int q = g.tb[i];
        t = ((t >> q) << (q + 1)) | (t & ((uint64_t(1) << q) - 1));
    }
    return t;
}

__device__ __forceinline__ uint32_t staging_swizzle(uint32_t l) {
    return l ^ ((((l >> 4) ^ (l >> 7)) & 7u) << 1);
}

template <int K>
__global__ void __launch_bounds__(128)
k_dense_tc(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ TcGeom geo,
           const __grid_constant__ TcMat<K> U) {
    constexpr int D = 1 << K;       // slice members
    constexpr int NK = 2 * D;       // GEMM N = K (reals)
    constexpr int TILE = 128 * D;   // amplitudes per tile
    constexpr int PER = TILE / 2 / 128;  // float4 per thread
    constexpr int CH = 1 << (K + 7 - 7);  // upper bound of chunks (L >= 7)
    constexpr uint32_t IDESC = tc::idesc_tf32(128, NK);

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sWhi = base;
    uint8_t *sWlo = sWhi + NK * NK * 4;
    uint8_t *sAhi = sWlo + NK * NK * 4;
    uint8_t *sAlo = sAhi + 128 * NK * 4;
    uint64_t *chunk_off = reinterpret_cast<uint64_t *>(sAlo + 128 * NK * 4);
    uint64_t *mbar = chunk_off + CH;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    uint32_t *sj_lo = tslot + 1;            // 64 entries: s | j << 8 of l & 63
    uint32_t *sj_hi = sj_lo + 64;           // 2^(K+1) entries for l >> 6
    uint16_t *dep_s = reinterpret_cast<uint16_t *>(sj_hi + (1 << (K + 1)));  // 128
    uint16_t *dep_j = dep_s + 128;          // D
    float2 *stage = reinterpret_cast<float2 *>(sAhi);

    const int tid = threadIdx.x, warp = tid >> 5;

    // ---- prologue: W_hi / W_lo in SW128 K-major, index tables, barrier, TMEM
    for (int idx = tid; idx < NK * NK; idx += 128) {
        const int r = idx / NK, c = idx % NK;
        const float2 h = U.hi[r >> 1][c >> 1], l = U.lo[r >> 1][c >> 1];
        float vh, vl;
        if ((r & 1) == (c & 1)) { vh = h.x; vl = l.x; }        // a on the 2x2 diagonal
        else if (r & 1) { vh = h.y; vl = l.y; }                // b (row im, col re)
        else { vh = -h.y; vl = -l.y; }                         // -b (row re, col im)
        *reinterpret_cast<float *>(sWhi + tc::sw128_offset(r, c, NK)) = vh;
        *reinterpret_cast<float *>(sWlo + tc::sw128_offset(r, c, NK)) = vl;
    }
    const int ntb = K + 7;
    const uint32_t tm = geo.tmask;
    for (int i = tid; i < 64 + (1 << (K + 1)); i += 128) {
        const uint32_t l = i < 64 ? uint32_t(i) : uint32_t(i - 64) << 6;
        uint32_t s = 0, j = 0;
        int ps = 0, pj = 0;
        for (int b = 0; b < ntb; b++) {
            const uint32_t bit = (l >> b) & 1u;
            if ((tm >> b) & 1u) j |= bit << pj++;
            else s |= bit << ps++;
        }
        if (i < 64) sj_lo[i] = s | (j << 8);
        else sj_hi[i - 64] = s | (j << 8);
    }
    for (int i = tid; i < 128 + D; i += 128) {
        // deposit slice bits (i < 128) or member bits into local positions
        const uint32_t v = i < 128 ? uint32_t(i) : uint32_t(i - 128);
        const bool member = i >= 128;
        uint32_t l = 0;
        int p = 0;
        for (int b = 0; b < ntb; b++)
            if ((((tm >> b) & 1u) != 0) == member) l |= ((v >> p++) & 1u) << b;
        if (i < 128) dep_s[i] = uint16_t(l);
        else dep_j[i - 128] = uint16_t(l);
    }
    const int L = geo.L;
    for (int c = tid; c < (1 << (ntb - L)); c += 128) {
        uint64_t off = 0;
        for (int b = 0; b < ntb - L; b++)
            if ((c >> b) & 1) off |= uint64_t(1) << geo.tb[L + b];
        chunk_off[c] = off;
    }
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, NK);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t lmask = (1u << L) - 1u;
    const bool pair_in_slice = (tm & 1u) != 0;  // index bit 0 is a target

    auto load_tile = [&](uint64_t t, float4 (&pf)[PER]) {
        const uint64_t b0 = tile_base(t, geo);
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const uint32_t l = 2u * uint32_t(tid + 128 * i);
            pf[i] = __ldcs(reinterpret_cast<const float4 *>(sv + b0 + chunk_off[l >> L] + (l & lmask)));
        }
    };

    float4 pf[PER];
    uint64_t tile = blockIdx.x;
    if (tile < ntiles) load_tile(tile, pf);
    uint32_t phase = 0;
    bool failed = false;
    for (; tile < ntiles; tile += gridDim.x) {
        // ---- split into hi / lo and place in the A operand (row = slice)
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const uint32_t l = 2u * uint32_t(tid + 128 * i);
            const uint32_t sj = sj_lo[l & 63] | sj_hi[l >> 6];
            const int s = int(sj & 0xFF), j = int(sj >> 8);
            const float4 v = pf[i];
            float4 h, o;
            h.x = tc::to_tf32(v.x); o.x = v.x - h.x;
            h.y = tc::to_tf32(v.y); o.y = v.y - h.y;
            h.z = tc::to_tf32(v.z); o.z = v.z - h.z;
            h.w = tc::to_tf32(v.w); o.w = v.w - h.w;
            if (pair_in_slice) {  // members j, j+1 of slice s: 16 contiguous bytes
                const uint32_t off = tc::sw128_offset(s, 2 * j, 128);
                *reinterpret_cast<float4 *>(sAhi + off) = h;
                *reinterpret_cast<float4 *>(sAlo + off) = o;
            } else {  // member j of slices s and s+1
                const uint32_t o0 = tc::sw128_offset(s, 2 * j, 128), o1 = tc::sw128_offset(s + 1, 2 * j, 128);
                *reinterpret_cast<float2 *>(sAhi + o0) = make_float2(h.x, h.y);
                *reinterpret_cast<float2 *>(sAlo + o0) = make_float2(o.x, o.y);
                *reinterpret_cast<float2 *>(sAhi + o1) = make_float2(h.z, h.w);
                *reinterpret_cast<float2 *>(sAlo + o1) = make_float2(o.z, o.w);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // ---- three MMA chains into one fp32 accumulator
        if (tid == 0) {
            const uint32_t aH = tc::smem_u32(sAhi), aL = tc::smem_u32(sAlo);
            const uint32_t wH = tc::smem_u32(sWhi), wL = tc::smem_u32(sWlo);
            uint32_t acc = 0;
#pragma unroll
            for (int p = 0; p < 3; p++) {
                const uint32_t a = p == 1 ? aH : (p == 0 ? aL : aH);
                const uint32_t w = p == 1 ? wL : wH;
#pragma unroll
                for (int s = 0; s < NK / 8; s++) {
                    // k-step s: K columns 8s..8s+7 = atom column s/4, 32-byte offset (s%4) inside it
                    const uint32_t ka = uint32_t((s >> 2) * (128 / 8) * 1024 + (s & 3) * 32);
                    const uint32_t kw = uint32_t((s >> 2) * (NK / 8) * 1024 + (s & 3) * 32);
                    tc::mma_tf32(taddr, tc::smem_desc_sw128(a + ka), tc::smem_desc_sw128(w + kw), IDESC, acc);
                    acc = 1;
                }
            }
            tc::mma_commit(mbar);
        }
        // ---- prefetch the next tile while the tensor cores work
        const uint64_t next = tile + gridDim.x;
        if (next < ntiles) load_tile(next, pf);
        const bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // ---- TMEM -> registers -> staging (natural order, swizzled)
        {
            const int s = tid;
            const uint32_t ls = dep_s[s];
#pragma unroll
            for (int c0 = 0; c0 < NK; c0 += 32) {
                float v[32];
                tc::tmem_ld32(taddr + (uint32_t(32 * warp) << 16) + uint32_t(c0), v);
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int j = c0 / 2 + q;
                    stage[staging_swizzle(ls | dep_j[j])] = make_float2(v[2 * q], v[2 * q + 1]);
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // ---- coalesced stores
        {
            const uint64_t b0 = tile_base(tile, geo);
#pragma unroll
            for (int i = 0; i < PER; i++) {
                const uint32_t l = 2u * uint32_t(tid + 128 * i);
                const float4 v = *reinterpret_cast<const float4 *>(stage + staging_swizzle(l));
                __stcs(reinterpret_cast<float4 *>(sv + b0 + chunk_off[l >> L] + (l & lmask)), v);
            }
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicOr(&g_tc_error, 1);
        tc::mbar_wait(mbar, phase, kWaitLimit);  // let an MMA in flight finish before freeing TMEM
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, NK);
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

template <int K>
size_t tc_smem_bytes() {
    constexpr int D = 1 << K, NK = 2 * D;
    return 1024 + size_t(NK) * NK * 4 * 2 + size_t(128) * NK * 4 * 2 + 8 * (1 << K) + 16 + 4 * 64 +
           4 * (1 << (K + 1)) + 2 * (128 + D) + 64;
}

template <int K>
cast_status run_tc(cast_sv *sv, const PreparedGate &g) {
    constexpr int D = 1 << K;
    TcMat<K> U;
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++) {
            const cplx u = g.m[size_t(r) * D + c];
            const float hr = host_tf32((float)u.real()), hi = host_tf32((float)u.imag());
            U.hi[r][c] = make_float2(hr, hi);
            U.lo[r][c] = make_float2((float)(u.real() - (double)hr), (float)(u.imag() - (double)hi));
        }
    TcGeom geo{};
    geo.ntb = K + 7;
    // tile bits: targets plus the 7 lowest non-targets
    uint64_t tbits = 0;
    for (int i = 0; i < K; i++) tbits |= uint64_t(1) << g.q[i];
    int added = 0;
    for (int b = 0; b < sv->n && added < 7; b++)
        if (!((tbits >> b) & 1)) {
            tbits |= uint64_t(1) << b;
            added++;
        }
    int p = 0;
    for (int b = 0; b < 64; b++)
        if ((tbits >> b) & 1) geo.tb[p++] = b;
    geo.L = 0;
    while (geo.L < geo.ntb && geo.tb[geo.L] == geo.L) geo.L++;
    geo.tmask = 0;
    for (int i = 0; i < geo.ntb; i++)
        for (int t = 0; t < K; t++)
            if (geo.tb[i] == g.q[t]) geo.tmask |= 1u << i;
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const size_t smem = tc_smem_bytes<K>();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int per_sm = K <= 4 ? 4 : 2;
    const uint64_t cap = uint64_t(sm_count_cached()) * per_sm;
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    ProfScope ps(sv->stream, "tc_k" + std::to_string(K) + "_c64", 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    k_dense_tc<K><<<(unsigned)grid, 128, smem, sv->stream>>>(reinterpret_cast<float2 *>(sv->data), ntiles, geo, U);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool tc_eligible(const cast_sv *sv, const PreparedGate &g) {
    return g_tensor_mode.load() == CAST_TC_TF32X3 && sv->dt == CAST_C64 && g.cls == CLS_DENSE &&
           (g.k == 4 || g.k == 5) && sv->n >= g.k + 7;
}

cast_status launch_gate_tc(cast_sv *sv, const PreparedGate &g) {
    if (g.k == 4) return run_tc<4>(sv, g);
    if (g.k == 5) return run_tc<5>(sv, g);
    return fail(CAST_ERR_UNSUPPORTED, "tensor-core path covers k = 4, 5");
}

cast_status take_device_error() {
    int v = 0;
    CAST_CUDA(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)));
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
    if (mode != CAST_TC_OFF && mode != CAST_TC_TF32X3) return cast::fail(CAST_ERR_ARG, "unknown tensor mode");
    cast::g_tensor_mode = mode;
    return CAST_OK;
}

int cast_get_tensor_mode(void) { return cast::g_tensor_mode.load(); }

}  // extern "C"
