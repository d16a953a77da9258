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
// Precision: 3xTF32.  Each operand x is split into hi = tf32(x) and
// lo = tf32(x - hi), both rounded to nearest; the three products lo*W_hi +
// hi*W_lo + hi*W_hi are accumulated in fp32 in TMEM, giving fp32-class
// accuracy (the dropped lo*lo term and the rounding of lo are ~2^-22
// relative).  Rounding lo (rather than letting the tensor cores truncate it)
// removes one bias.  The tensor cores' fp32 accumulation itself truncates
// toward zero, which shrinks every output slightly (measured: ~2^-23 of the
// norm per gate, growing with k).  A unitary gate preserves the norm of every
// slice exactly, so each slice's outputs are rescaled by |x| / |y| (both norms
// summed with a compensated fp32 pair); what remains is unbiased rounding
// noise.  The correction is applied as y + y * delta with delta formed as a
// small number, so it is not quantised to the fp32 spacing near 1.  Only gates
// that are unitary to 1e-9 take this path.
//
// Data path per tile: thread (warp w, lane i) owns slice 32*(w%4) + i, i.e.
// TMEM lane 32*(w%4) + i, and 16 of its members (warp group w/4).  It gathers
// them from HBM with the Eq. 4 addressing (for a fixed member, 32 lanes read 32
// consecutive slices), splits hi/lo in registers and writes both into TMEM
// with tcgen05.st: the state tile never passes through shared memory.  The
// MMAs read A from TMEM and W_hi / W_lo from shared memory (128-byte swizzled
// K-major, built once per CTA from the hi/lo split of U carried in the launch
// parameters).  The next tile's loads are issued before the MMAs are waited
// for, so they stay in flight through the MMAs and the epilogue.
// TMEM per CTA: accumulator, A_hi, A_lo = 3 x 2^(k+1) columns (rounded up to a
// power of two); registers and padding of the shared-memory request keep the
// number of resident CTAs per SM within the 512 TMEM columns.
//
// Waits on the mbarrier are bounded; a CTA that gives up sets an error bit in
// g_tc_error (read by the host at its next synchronisation point), stops its
// tile loop, waits once more (bounded) for its MMAs and frees its TMEM.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
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

template <int K>
struct TcShape {
    static constexpr int D = 1 << K;           // slice members
    static constexpr int NK = 2 * D;           // GEMM N = K (reals)
    static constexpr int MPT = D < 16 ? D : 16;  // members per thread
    static constexpr int GROUPS = D / MPT;     // warps per TMEM lane quarter
    static constexpr int NT = 128 * GROUPS;    // threads per CTA
    static constexpr int NCOL = 3 * NK <= 128 ? 128 : (3 * NK <= 256 ? 256 : 512);
    static constexpr int CTAS_PER_SM = 512 / NCOL;
};

template <int K>
__global__ void __launch_bounds__(TcShape<K>::NT, TcShape<K>::CTAS_PER_SM)
k_dense_tc(float2 *__restrict__ sv, uint64_t ntiles, const __grid_constant__ Targets tg,
           const __grid_constant__ TcMat<K> U, uint32_t wait_limit, int skip_mma) {
    using S = TcShape<K>;
    constexpr int NK = S::NK, MPT = S::MPT;
    constexpr uint32_t IDESC = tc::idesc_tf32(128, NK);
    constexpr uint32_t COL_AH = NK, COL_AL = 2 * NK;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sWhi = base;
    uint8_t *sWlo = sWhi + NK * NK * 4;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sWlo + NK * NK * 4);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    float2 *xnorm = reinterpret_cast<float2 *>(tslot + 2);   // [GROUPS][128] compensated |x|^2 parts
    float2 *ynorm = xnorm + S::GROUPS * 128;                 // [GROUPS][128] compensated |y|^2 parts

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, group = warp >> 2, j0 = group * MPT;
    const int row = 32 * quarter + lane;

    // ---- prologue: W_hi / W_lo (SW128 K-major), barrier, TMEM
    for (int idx = tid; idx < NK * NK; idx += S::NT) {
        const int r = idx / NK, c = idx % NK;
        const float2 h = U.h(r >> 1, c >> 1), l = U.l(r >> 1, c >> 1);
        float vh, vl;
        if ((r & 1) == (c & 1)) { vh = h.x; vl = l.x; }   // a on the 2x2 diagonal
        else if (r & 1) { vh = h.y; vl = l.y; }           // b (row im, col re)
        else { vh = -h.y; vl = -l.y; }                    // -b (row re, col im)
        *reinterpret_cast<float *>(sWhi + tc::sw128_offset(r, c, NK)) = vh;
        *reinterpret_cast<float *>(sWlo + tc::sw128_offset(r, c, NK)) = vl;
    }
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, S::NCOL);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    const uint32_t lane_addr = taddr + (uint32_t(32 * quarter) << 16);

    // offsets of this thread's members relative to the slice base
    uint64_t p[K];
#pragma unroll
    for (int i = 0; i < K; i++) p[i] = uint64_t(1) << tg.q[i];
    uint64_t off0 = 0;
#pragma unroll
    for (int i = 0; i < K; i++)
        if ((j0 >> i) & 1) off0 += p[i];
    auto member_off = [&](int m) {  // m compile-time after unrolling
        uint64_t o = off0;
#pragma unroll
        for (int i = 0; i < K; i++)
            if ((m >> i) & 1) o += p[i];
        return o;
    };
    auto load = [&](uint64_t tile, float2 (&x)[MPT]) {
        const uint64_t b = slice_base<K>(tile * 128 + uint64_t(32 * quarter + lane), tg);
#pragma unroll
        for (int m = 0; m < MPT; m++) x[m] = sv[b + member_off(m)];
    };

    float2 cur[MPT], nxt[MPT];
    uint64_t tile = blockIdx.x;
    uint32_t phase = 0;
    bool failed = false;
    if (tile < ntiles) load(tile, cur);
    while (tile < ntiles) {
        // ---- split, TMEM stores of A_hi and A_lo (this thread's row, its members)
        float v[2 * MPT];
#pragma unroll
        for (int m = 0; m < MPT; m++) {
            v[2 * m] = tc::to_tf32(cur[m].x);
            v[2 * m + 1] = tc::to_tf32(cur[m].y);
        }
        tc::tmem_st<2 * MPT>(lane_addr + COL_AH + 2 * j0, v);
        // the remainder is rounded to tf32 as well: the tensor cores would
        // otherwise truncate it, a bias that shrinks the norm gate after gate
#pragma unroll
        for (int m = 0; m < MPT; m++) {
            v[2 * m] = tc::to_tf32(cur[m].x - v[2 * m]);
            v[2 * m + 1] = tc::to_tf32(cur[m].y - v[2 * m + 1]);
        }
        tc::tmem_st<2 * MPT>(lane_addr + COL_AL + 2 * j0, v);
        {
            Acc<float> xs;
#pragma unroll
            for (int m = 0; m < MPT; m++) xs.add(cur[m].x * cur[m].x + cur[m].y * cur[m].y);
            xnorm[group * 128 + row] = make_float2(xs.hi, xs.lo);
        }
        tc::tmem_wait_st();
        // ---- prefetch the next tile; the loads stay in flight meanwhile
        const uint64_t next = tile + gridDim.x;
        if (next < ntiles) load(next, nxt);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !skip_mma) {
            const uint32_t wH = tc::smem_u32(sWhi), wL = tc::smem_u32(sWlo);
            uint32_t acc = 0;
#pragma unroll
            for (int pr = 0; pr < 3; pr++) {
                const uint32_t acol = pr == 0 ? COL_AL : COL_AH;  // lo*W_hi, hi*W_lo, hi*W_hi
                const uint32_t w = pr == 1 ? wL : wH;
#pragma unroll
                for (int s = 0; s < NK / 8; s++) {
                    const uint32_t kw = uint32_t((s >> 2) * (NK / 8) * 1024 + (s & 3) * 32);
                    tc::mma_tf32_ts(taddr, taddr + acol + 8 * s, tc::smem_desc_sw128(w + kw), IDESC, acc);
                    acc = 1;
                }
            }
            tc::mma_commit(mbar);
        }
        const bool ok = tc::mbar_wait(mbar, phase, wait_limit);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // ---- accumulator -> registers; restore the slice norm; -> HBM
        tc::tmem_ld<2 * MPT>(lane_addr + 2 * j0, v);
        {
            Acc<float> ys;
#pragma unroll
            for (int m = 0; m < MPT; m++) ys.add(v[2 * m] * v[2 * m] + v[2 * m + 1] * v[2 * m + 1]);
            ynorm[group * 128 + row] = make_float2(ys.hi, ys.lo);
        }
        __syncthreads();
        {
            Acc<float> X, Y;
#pragma unroll
            for (int gq = 0; gq < S::GROUPS; gq++) {
                const float2 a = xnorm[gq * 128 + row], b = ynorm[gq * 128 + row];
                X.add(a.x); X.add(a.y);
                Y.add(b.x); Y.add(b.y);
            }
            // y <- y * sqrt(X / Y) = y + y * delta with delta = (X - Y) / (2 Y) to
            // first order (|delta| ~ 1e-7; the second-order term is ~1e-14).
            // delta is formed as a small number (X.hi - Y.hi is exact when the
            // two are close) so the correction keeps full fp32 precision; a
            // scale factor near 1 would be quantised to multiples of 2^-23.
            float delta = 0.0f;
            if (Y.hi > 0.0f && X.hi > 0.0f) delta = 0.5f * ((X.hi - Y.hi) + (X.lo - Y.lo)) / Y.hi;
            const uint64_t b = slice_base<K>(tile * 128 + uint64_t(row), tg);
#pragma unroll
            for (int m = 0; m < MPT; m++)
                __stcs(&sv[b + member_off(m)],
                       make_float2(fmaf(v[2 * m], delta, v[2 * m]), fmaf(v[2 * m + 1], delta, v[2 * m + 1])));
        }
        tile = next;
#pragma unroll
        for (int m = 0; m < MPT; m++) cur[m] = nxt[m];
        tc::fence_before_sync();
        __syncthreads();
    }
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

template <int K>
size_t tc_smem_bytes() {
    using S = TcShape<K>;
    const size_t need = 1024 + size_t(S::NK) * S::NK * 4 * 2 + 64 + 2 * 8 * 128 * S::GROUPS;
    // at most CTAS_PER_SM resident CTAs per SM (228 KB of shared memory each)
    const size_t floor = (228 * 1024) / (S::CTAS_PER_SM + 1) + 1024;
    return need > floor ? need : floor;
}

template <int K>
cast_status run_tc(cast_sv *sv, const PreparedGate &g) {
    constexpr int D = 1 << K;
    using S = TcShape<K>;
    std::vector<float2> hl(size_t(2) << (2 * K));
    for (int r = 0; r < D; r++)
        for (int c = 0; c < D; c++) {
            const cplx u = g.m[size_t(r) * D + c];
            const float hr = host_tf32((float)u.real()), hi = host_tf32((float)u.imag());
            hl[size_t(r) * D + c] = make_float2(hr, hi);
            hl[(size_t(1) << (2 * K)) + size_t(r) * D + c] =
                make_float2(host_tf32((float)(u.real() - (double)hr)), host_tf32((float)(u.imag() - (double)hi)));
        }
    TcMat<K> U;
    if constexpr (K <= 5) {
        std::memcpy(U.hi, hl.data(), sizeof(U.hi));
        std::memcpy(U.lo, hl.data() + (size_t(1) << (2 * K)), sizeof(U.lo));
    } else {
        const void *dev = nullptr;
        cast_status st = upload_matrix(sv, hl.data(), hl.size() * sizeof(float2), &dev);
        if (st != CAST_OK) return st;
        U.hi = static_cast<const float2 *>(dev);
    }
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const uint64_t ntiles = uint64_t(1) << (sv->n - K - 7);
    const size_t smem = tc_smem_bytes<K>();
    CAST_CUDA(cudaFuncSetAttribute(k_dense_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t cap = uint64_t(sm_count_cached()) * S::CTAS_PER_SM;
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    ProfScope ps(sv->stream, "tc_k" + std::to_string(K) + "_c64", 16.0 * double(uint64_t(1) << sv->n),
                 8.0 * double(uint64_t(1) << (sv->n + K)));
    const uint32_t inject = g_inject_limit.exchange(0);
    k_dense_tc<K><<<(unsigned)grid, S::NT, smem, sv->stream>>>(reinterpret_cast<float2 *>(sv->data), ntiles, tg, U,
                                                               inject ? inject : kWaitLimit, inject ? 1 : 0);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool tc_eligible(const cast_sv *sv, const PreparedGate &g) {
    return g_tensor_mode.load() == CAST_TC_TF32X3 && sv->dt == CAST_C64 && g.cls == CLS_DENSE && g.unitary &&
           g.k >= 4 && g.k <= 6 && sv->n >= g.k + 7;
}

cast_status launch_gate_tc(cast_sv *sv, const PreparedGate &g) {
    if (g.k == 4) return run_tc<4>(sv, g);
    if (g.k == 5) return run_tc<5>(sv, g);
    if (g.k == 6) return run_tc<6>(sv, g);
    return fail(CAST_ERR_UNSUPPORTED, "tensor-core path covers k = 4, 5, 6");
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

cast_status cast_debug_inject_timeout(uint32_t wait_limit) {
    if (wait_limit == 0) return cast::fail(CAST_ERR_ARG, "wait limit must be positive");
    cast::g_inject_limit = wait_limit;
    return CAST_OK;
}

}  // extern "C"
