// Gate-application kernels for sm_103a (Eq. 3 of the paper: 2^(n-k)
// gathered 2^k x 2^k matrix-vector products on a 2^n state).
//
// Kernel families (the host picks one per prepared gate):
//   k_dense<R,K>       K <= 5, any targets.  One slice (2^K amplitudes) per
//                      thread iteration, kept in registers.  The matrix travels
//                      in the launch's parameter space (<= 16 KB) so every
//                      thread reads the same entry from the constant bank in
//                      lockstep (broadcast).
//   k_dense_cube<K>    complex64, K <= 4, gates with two or more low targets:
//                      the same matvec per slice, but each warp moves its 32
//                      slices as one staged cube (struct CubeTables):
//                      coalesced 16-byte cp.async chunks into a ring of two
//                      swizzled shared-memory buffers, the slice rows read
//                      from there, the outputs written back through the same
//                      buffer.
//   k_dense_tile<R,K>  K = 6, 7.  A CTA stages 2^K x TS amplitudes in shared
//                      memory, then each thread forms (row, slice) outputs
//                      reading the matrix from global memory (L1-resident).
//   k_diag<R,K>        diagonal gates: one pass over the amplitudes, each
//                      multiplied by d[local index]; entries equal to 1 are
//                      neither read nor written.
//   k_mono<R,K>        monomial gates (one non-zero per row and column:
//                      X, CX, SWAP, Y, ...): gather the source of every row,
//                      multiply by its phase, scatter; fixed points with phase
//                      1 are skipped.
//
// Slice enumeration follows Eq. 4: the base index of slice t is t with a zero
// bit inserted at every target position (targets sorted ascending); member j
// of the slice adds 2^q[i] for every set bit i of j.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace cast {
namespace {

// ------------------------------------------------------------ dense, K <= 5
template <typename R, int K>
struct DenseMat {
    typename Cx<R>::T m[1 << K][1 << K];
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_dense(typename Cx<R>::T *__restrict__ sv, uint64_t nslices, Targets tg,
        const __grid_constant__ DenseMat<R, K> U) {
    using T2 = typename Cx<R>::T;
    constexpr int D = 1 << K;
    uint64_t p[K];
#pragma unroll
    for (int i = 0; i < K; i++) p[i] = uint64_t(1) << tg.q[i];
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nslices; t += stride) {
        const uint64_t base = slice_base<K>(t, tg);
        T2 x[D];
#pragma unroll
        for (int j = 0; j < D; j++) {
            uint64_t off = 0;
#pragma unroll
            for (int i = 0; i < K; i++)
                if ((j >> i) & 1) off += p[i];
            x[j] = sv[base + off];
        }
#pragma unroll
        for (int r = 0; r < D; r++) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < D; c++) {
                const T2 u = U.m[r][c];
                re = fma(u.x, x[c].x, re);
                re = fma(-u.y, x[c].y, re);
                im = fma(u.x, x[c].y, im);
                im = fma(u.y, x[c].x, im);
            }
            uint64_t off = 0;
#pragma unroll
            for (int i = 0; i < K; i++)
                if ((r >> i) & 1) off += p[i];
            T2 y;
            y.x = re;
            y.y = im;
            sv[base + off] = y;
        }
    }
}

// --------------------------------------------- dense complex64, staged cube
// A stage holds CPI = 16 / 2^K consecutive cubes (4 KB for every K), so that
// small gates keep as many bytes in flight per warp as k = 4.
template <int K>
constexpr int cube_per_stage() { return K < 4 ? (16 >> K) : 1; }

template <int K>
__global__ void __launch_bounds__(256, 3)
k_dense_cube(float2 *__restrict__ sv, uint64_t ncubes, Targets tg, const __grid_constant__ DenseMat<float, K> U,
             const __grid_constant__ CubeTables ct) {
    constexpr int D = 1 << K, E = 32 * D, CH = D / 2, NS = 2, CPI = cube_per_stage<K>();
    extern __shared__ __align__(16) unsigned char cube_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *stages = reinterpret_cast<float2 *>(cube_smem) + warp * (NS * CPI * E);
    const uint64_t g_lane = ct.g_lane[lane];
    const uint32_t s_lane = ct.s_lane[lane], s_row = ct.s_row[lane];
    const uint64_t nsup = ncubes / CPI;  // stage-sized groups of consecutive cubes
    const uint64_t wstep = uint64_t(gridDim.x) * (blockDim.x >> 5);
    auto cube_base = [&](uint64_t c) { return slice_base<K>(c * 32, tg) + g_lane; };
    auto copy_async = [&](uint64_t sc, float2 *stage) {
#pragma unroll
        for (int u = 0; u < CPI; u++) {
            const float2 *b = sv + cube_base(sc * CPI + u);
            const uint32_t d = uint32_t(__cvta_generic_to_shared(stage + u * E));
#pragma unroll
            for (int j = 0; j < CH; j++)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + ((s_lane ^ ct.s_j[j]) >> 1) * 16u),
                             "l"(b + ct.g_j[j])
                             : "memory");
        }
    };
    uint64_t sc = uint64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
#pragma unroll
    for (int si = 0; si < NS; si++) {
        if (sc + si * wstep < nsup) copy_async(sc + si * wstep, stages + si * CPI * E);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int si = 0; sc < nsup; sc += wstep, si ^= 1) {
        float2 *stage = stages + si * CPI * E;
        asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
        __syncwarp();
#pragma unroll 1
        for (int u = 0; u < CPI; u++) {
            float2 *cube = stage + u * E;
            float2 x[D];
            if (K >= 2 && ct.pair) {  // members 2m, 2m+1 in one 16-byte chunk
#pragma unroll
                for (int m = 0; m < D; m += 2) {
                    const float4 v = reinterpret_cast<const float4 *>(cube)[(s_row ^ ct.s_mem[m]) >> 1];
                    x[m] = make_float2(v.x, v.y);
                    x[m + 1] = make_float2(v.z, v.w);
                }
            } else {
#pragma unroll
                for (int m = 0; m < D; m++) x[m] = cube[s_row ^ ct.s_mem[m]];
            }
            // the row's slots belong to this lane alone: the outputs go in place
#pragma unroll
            for (int r = 0; r < D; r++) {
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int cc = 0; cc < D; cc++) {
                    const float2 uu = U.m[r][cc];
                    re = fmaf(uu.x, x[cc].x, re);
                    re = fmaf(-uu.y, x[cc].y, re);
                    im = fmaf(uu.x, x[cc].y, im);
                    im = fmaf(uu.y, x[cc].x, im);
                }
                cube[s_row ^ ct.s_mem[r]] = make_float2(re, im);
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < CPI; u++) {
            float2 *b = sv + cube_base(sc * CPI + u);
            const float4 *s4 = reinterpret_cast<const float4 *>(stage + u * E);
#pragma unroll
            for (int j = 0; j < CH; j++)
                __stcs(reinterpret_cast<float4 *>(b + ct.g_j[j]), s4[(s_lane ^ ct.s_j[j]) >> 1]);
        }
        __syncwarp();
        if (sc + NS * wstep < nsup) copy_async(sc + NS * wstep, stage);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// --------------------------------------------------------- dense, K = 6, 7
template <typename R, int K, int TS>
__global__ void __launch_bounds__(256)
k_dense_tile(typename Cx<R>::T *__restrict__ sv, uint64_t nslices, Targets tg,
             const typename Cx<R>::T *__restrict__ U) {
    using T2 = typename Cx<R>::T;
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *X = reinterpret_cast<T2 *>(smem_raw);  // [D][TS]
    const uint64_t ntiles = (nslices + TS - 1) / TS;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t t0 = tile * TS;
        for (int idx = threadIdx.x; idx < D * TS; idx += blockDim.x) {
            const int j = idx / TS, s = idx % TS;
            const uint64_t t = t0 + s;
            if (t < nslices) X[idx] = sv[slice_base<K>(t, tg) + member_offset<K>(j, tg)];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < D * TS; idx += blockDim.x) {
            const int r = idx / TS, s = idx % TS;
            const uint64_t t = t0 + s;
            if (t >= nslices) continue;
            R re = 0, im = 0;
            const T2 *urow = U + size_t(r) * D;
#pragma unroll 8
            for (int c = 0; c < D; c++) {
                const T2 u = __ldg(urow + c);
                const T2 xv = X[c * TS + s];
                re = fma(u.x, xv.x, re);
                re = fma(-u.y, xv.y, re);
                im = fma(u.x, xv.y, im);
                im = fma(u.y, xv.x, im);
            }
            T2 y;
            y.x = re;
            y.y = im;
            sv[slice_base<K>(t, tg) + member_offset<K>(r, tg)] = y;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- diagonal
template <typename R, int K>
struct DiagVec {
    typename Cx<R>::T d[1 << K];
    uint32_t skip;  // bit j set: d[j] == 1, amplitudes with local index j untouched
};

// 16-byte vectors: 2 complex64 or 1 complex128 amplitudes per access.
template <typename R> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int A = 2; };
template <> struct Vec16<double> { using T = double2; static constexpr int A = 1; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T vec_amp(const typename Vec16<R>::T &v, int a);
template <> __device__ __forceinline__ float2 vec_amp<float>(const float4 &v, int a) {
    return a == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}
template <> __device__ __forceinline__ double2 vec_amp<double>(const double2 &v, int) { return v; }
template <typename R>
__device__ __forceinline__ void vec_set(typename Vec16<R>::T &v, int a, typename Cx<R>::T x);
template <> __device__ __forceinline__ void vec_set<float>(float4 &v, int a, float2 x) {
    if (a == 0) { v.x = x.x; v.y = x.y; } else { v.z = x.x; v.w = x.y; }
}
template <> __device__ __forceinline__ void vec_set<double>(double2 &v, int, double2 x) { v = x; }

// Each thread takes UNR 16-byte vectors per round (grid stride apart), issues
// all their loads before any arithmetic, and skips a vector whose amplitudes
// all have diagonal entry 1 (neither read nor written).
template <typename R, int K>
__global__ void __launch_bounds__(256)
k_diag(typename Cx<R>::T *__restrict__ sv, uint64_t N, Targets tg,
       const __grid_constant__ DiagVec<R, K> D) {
    using V = typename Vec16<R>::T;
    constexpr int A = Vec16<R>::A, UNR = 8;  // vectors in flight per thread (4: 2% slower, 16: 55% slower)
    V *vp = reinterpret_cast<V *>(sv);
    const uint64_t nvec = N / A;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t v0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; v0 < nvec; v0 += stride * UNR) {
        V v[UNR];
        int j[UNR][A];
        bool act[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t iv = v0 + uint64_t(u) * stride;
            act[u] = false;
            if (iv < nvec) {
#pragma unroll
                for (int a = 0; a < A; a++) {
                    const uint64_t x = iv * A + a;
                    int jj = 0;
#pragma unroll
                    for (int b = 0; b < K; b++) jj |= int((x >> tg.q[b]) & 1) << b;
                    j[u][a] = jj;
                    act[u] |= (K > 5) || !((D.skip >> jj) & 1);
                }
                if (act[u]) v[u] = vp[iv];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (!act[u]) continue;
#pragma unroll
            for (int a = 0; a < A; a++) vec_set<R>(v[u], a, cmul(D.d[j[u][a]], vec_amp<R>(v[u], a)));
            vp[v0 + uint64_t(u) * stride] = v[u];
        }
    }
}

// Chunked form for states of at least 2^12 amplitudes: a CTA iteration
// covers a contiguous chunk of 256 x UNR 16-byte vectors (thread t takes
// vectors t, t + 256, ...: coalesced).  The diagonal index of an amplitude is
// the OR of three parts formed once: the chunk's (targets above the chunk),
// the thread's (its lane's address bits within a round) and the round's, plus
// the amplitude's own bit 0 when qubit 0 is a target; the per-amplitude
// bit-by-bit extraction of k_diag is gone.
// The round parts jr[u] and the bit-0 part j0 are the same for every thread
// and come with the launch parameters.
struct DiagChunkBits {
    int jr[8];
    int j0;
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_diag_chunk(typename Cx<R>::T *__restrict__ sv, uint64_t nchunks, const __grid_constant__ Targets tg,
             const __grid_constant__ DiagVec<R, K> D, const __grid_constant__ DiagChunkBits cb) {
    using V = typename Vec16<R>::T;
    constexpr int A = Vec16<R>::A, LA = A == 2 ? 1 : 0, UNR = 8, CB = 8 + 3 + LA;
    auto jbits = [&](uint64_t x) {
        int j = 0;
#pragma unroll
        for (int b = 0; b < K; b++) j |= int((x >> tg.q[b]) & 1) << b;
        return j;
    };
    const int jt = jbits(uint64_t(threadIdx.x) << LA);
    const int j0 = cb.j0;
    V *vp = reinterpret_cast<V *>(sv);
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint64_t base = c << CB;
        const int jh = jbits(base) | jt;
        V *p = vp + (base >> LA) + threadIdx.x;
        uint32_t act = 0;
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const int jj = jh | cb.jr[u];
            const bool a = K > 5 || !((D.skip >> jj) & 1) || (A == 2 && !((D.skip >> (jj | j0)) & 1));
            act |= uint32_t(a) << u;
        }
        V v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++)
            if ((act >> u) & 1) v[u] = p[256 * u];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (!((act >> u) & 1)) continue;
            const int jj = jh | cb.jr[u];
            vec_set<R>(v[u], 0, cmul(D.d[jj], vec_amp<R>(v[u], 0)));
            if (A == 2) vec_set<R>(v[u], 1, cmul(D.d[jj | j0], vec_amp<R>(v[u], 1)));
            p[256 * u] = v[u];
        }
    }
}

// ---------------------------------------------------------------- monomial
template <typename R, int K>
struct MonoVec {
    typename Cx<R>::T ph[1 << K];
    uint8_t perm[1 << K];
    int unit;  // all phases are exactly 1
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_mono(typename Cx<R>::T *__restrict__ sv, uint64_t nslices, Targets tg,
       const __grid_constant__ MonoVec<R, K> M) {
    using T2 = typename Cx<R>::T;
    constexpr int D = 1 << K;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nslices; t += stride) {
        const uint64_t base = slice_base<K>(t, tg);
        T2 v[D];
#pragma unroll
        for (int r = 0; r < D; r++) {
            const int c = M.perm[r];
            if (c != r || !M.unit) v[r] = sv[base + member_offset<K>(c, tg)];
        }
#pragma unroll
        for (int r = 0; r < D; r++) {
            const int c = M.perm[r];
            if (c == r && M.unit) continue;
            sv[base + member_offset<K>(r, tg)] = M.unit ? v[r] : cmul(M.ph[r], v[r]);
        }
    }
}

// ------------------------------------------------------------ launch glue
uint64_t grid_for(uint64_t work_items, int per_sm) {
    uint64_t cap = uint64_t(sm_count_cached()) * per_sm;
    uint64_t need = (work_items + 255) / 256;
    if (need < 1) need = 1;
    return need < cap ? need : cap;
}

template <typename R>
typename Cx<R>::T to_dev(cplx z) {
    typename Cx<R>::T v;
    v.x = (R)z.real();
    v.y = (R)z.imag();
    return v;
}

template <typename R, int K>
cast_status run_dense(cast_sv *sv, const PreparedGate &g, const Targets &tg) {
    using T2 = typename Cx<R>::T;
    const uint64_t ns = uint64_t(1) << (sv->n - K);
    if constexpr (K <= 4 && sizeof(R) == 4) {
        // Targets below the 5th non-target bit (q_i - i < 5) spread a warp's
        // 32 slices over 32 x 2^L amplitudes for one member: with L >= 2 the
        // direct kernel's loads touch 4x the lines they use, and the staged
        // cube is faster; otherwise the direct kernel is already coalesced.
        int L = 0;
        for (int i = 0; i < K; i++) L += (g.q[i] - i) < 5;
        constexpr int CPI = cube_per_stage<K>();
        if (L >= 2 && sv->n >= K + 5 + (CPI == 16 ? 4 : CPI == 8 ? 3 : CPI == 4 ? 2 : CPI == 2 ? 1 : 0)) {
            DenseMat<float, K> U;
            for (int r = 0; r < (1 << K); r++)
                for (int c = 0; c < (1 << K); c++) U.m[r][c] = to_dev<float>(g.m[size_t(r) * (1 << K) + c]);
            const CubeTables ct = make_cube_tables(g.q, K);
            const uint64_t ncubes = ns >> 5;
            const size_t smem = size_t(8) * 2 * CPI * 32 * (1 << K) * sizeof(float2);  // 64 KB
            CAST_CUDA(cudaFuncSetAttribute(k_dense_cube<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int per_sm = tuned_blocks_per_sm(sv->dt, K, CLS_DENSE, 3);
            const uint64_t want = (ncubes / CPI + 7) / 8, cap = uint64_t(sm_count_cached()) * per_sm;
            ProfScope ps(sv->stream, "dense_k" + std::to_string(K) + "_" + dt_name(sv->dt),
                         2.0 * double(sizeof(T2)) * double(ns << K), 8.0 * double(ns << (2 * K)));
            k_dense_cube<K><<<(unsigned)(want < cap ? want : cap), 256, smem, sv->stream>>>(
                reinterpret_cast<float2 *>(sv->data), ncubes, tg, U, ct);
            CAST_CUDA(cudaGetLastError());
            return CAST_OK;
        }
    }
    if constexpr (K <= 5) {
        DenseMat<R, K> U;
        for (int r = 0; r < (1 << K); r++)
            for (int c = 0; c < (1 << K); c++) U.m[r][c] = to_dev<R>(g.m[size_t(r) * (1 << K) + c]);
        const int per_sm = tuned_blocks_per_sm(sv->dt, K, CLS_DENSE, K <= 3 ? 8 : (K == 4 ? 4 : 2));
        ProfScope ps(sv->stream, "dense_k" + std::to_string(K) + "_" + dt_name(sv->dt),
                     2.0 * double(sizeof(T2)) * double(ns << K), 8.0 * double(ns << (2 * K)));
        k_dense<R, K><<<(unsigned)grid_for(ns, per_sm), 256, 0, sv->stream>>>(
            reinterpret_cast<T2 *>(sv->data), ns, tg, U);
    } else {
        constexpr int TS = 32;
        const size_t mat_bytes = sizeof(T2) << (2 * K);
        std::vector<T2> h(size_t(1) << (2 * K));
        for (size_t i = 0; i < h.size(); i++) h[i] = to_dev<R>(g.m[i]);
        const void *dmat = nullptr;
        cast_status st = upload_matrix(sv, h.data(), mat_bytes, &dmat);
        if (st != CAST_OK) return st;
        const size_t smem = sizeof(T2) * (1 << K) * TS;
        CAST_CUDA(cudaFuncSetAttribute(k_dense_tile<R, K, TS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const uint64_t ntiles = (ns + TS - 1) / TS;
        ProfScope ps(sv->stream, "tile_k" + std::to_string(K) + "_" + dt_name(sv->dt),
                     2.0 * double(sizeof(T2)) * double(ns << K), 8.0 * double(ns << (2 * K)));
        const uint64_t grid = ntiles < uint64_t(sm_count_cached()) * 4 ? ntiles : uint64_t(sm_count_cached()) * 4;
        k_dense_tile<R, K, TS><<<(unsigned)grid, 256, smem, sv->stream>>>(
            reinterpret_cast<T2 *>(sv->data), ns, tg, reinterpret_cast<const T2 *>(dmat));
    }
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

template <typename R, int K>
cast_status run_diag(cast_sv *sv, const PreparedGate &g, const Targets &tg) {
    using T2 = typename Cx<R>::T;
    DiagVec<R, K> D;
    D.skip = 0;
    for (int j = 0; j < (1 << K); j++) {
        D.d[j] = to_dev<R>(g.diag[j]);
        if (K <= 5 && g.diag[j] == cplx(1.0, 0.0)) D.skip |= 1u << j;
    }
    const uint64_t N = uint64_t(1) << sv->n;
    int touched = 0;
    for (int j = 0; j < (1 << K); j++) touched += !((D.skip >> j) & 1) || K > 5;
    const double frac = double(touched) / double(1 << K);
    ProfScope ps(sv->stream, "diag_k" + std::to_string(K) + "_" + dt_name(sv->dt),
                 2.0 * double(sizeof(T2)) * double(N) * frac, 6.0 * double(N) * frac);
    if (sv->n >= 12) {
        constexpr int LA = sizeof(R) == 4 ? 1 : 0, CB = 8 + 3 + LA;
        DiagChunkBits cb{};
        for (int u = 0; u < 8; u++)
            for (int b = 0; b < K; b++) cb.jr[u] |= int(((uint64_t(u) << (8 + LA)) >> g.q[b]) & 1) << b;
        for (int b = 0; b < K; b++)
            if (LA == 1 && g.q[b] == 0) cb.j0 = 1 << b;
        const uint64_t nchunks = N >> CB;
        const uint64_t cap = uint64_t(sm_count_cached()) * tuned_blocks_per_sm(sv->dt, K, CLS_DIAG, 8);
        k_diag_chunk<R, K><<<(unsigned)(nchunks < cap ? nchunks : cap), 256, 0, sv->stream>>>(
            reinterpret_cast<T2 *>(sv->data), nchunks, tg, D, cb);
    } else {
        k_diag<R, K><<<(unsigned)grid_for(N, tuned_blocks_per_sm(sv->dt, K, CLS_DIAG, 8)), 256, 0, sv->stream>>>(
            reinterpret_cast<T2 *>(sv->data), N, tg, D);
    }
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

template <typename R, int K>
cast_status run_mono(cast_sv *sv, const PreparedGate &g, const Targets &tg) {
    using T2 = typename Cx<R>::T;
    MonoVec<R, K> M;
    M.unit = g.unit_phases ? 1 : 0;
    for (int j = 0; j < (1 << K); j++) {
        M.ph[j] = to_dev<R>(g.phase[j]);
        M.perm[j] = (uint8_t)g.perm[j];
    }
    const uint64_t ns = uint64_t(1) << (sv->n - K);
    int moved = 0;
    for (int j = 0; j < (1 << K); j++) moved += g.perm[j] != j || !g.unit_phases;
    const double frac = double(moved) / double(1 << K);
    ProfScope ps(sv->stream, "mono_k" + std::to_string(K) + "_" + dt_name(sv->dt),
                 2.0 * double(sizeof(T2)) * double(ns << K) * frac,
                 g.unit_phases ? 0.0 : 6.0 * double(ns << K));
    k_mono<R, K><<<(unsigned)grid_for(ns, tuned_blocks_per_sm(sv->dt, K, CLS_MONO, 8)), 256, 0, sv->stream>>>(
        reinterpret_cast<T2 *>(sv->data), ns, tg, M);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

template <typename R, int K>
cast_status dispatch_k(cast_sv *sv, const PreparedGate &g) {
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < g.k ? g.q[i] : 0;
    switch (g.cls) {
        case CLS_IDENTITY: return CAST_OK;
        case CLS_DIAG: return run_diag<R, K>(sv, g, tg);
        case CLS_MONO: return run_mono<R, K>(sv, g, tg);
        default: return run_dense<R, K>(sv, g, tg);
    }
}

template <typename R>
cast_status dispatch(cast_sv *sv, const PreparedGate &g) {
    switch (g.k) {
        case 1: return dispatch_k<R, 1>(sv, g);
        case 2: return dispatch_k<R, 2>(sv, g);
        case 3: return dispatch_k<R, 3>(sv, g);
        case 4: return dispatch_k<R, 4>(sv, g);
        case 5: return dispatch_k<R, 5>(sv, g);
        case 6: return dispatch_k<R, 6>(sv, g);
        case 7: return dispatch_k<R, 7>(sv, g);
        default: return fail(CAST_ERR_ARG, "gate size out of range");
    }
}

__global__ void k_set_one(void *data, int dt, uint64_t index) {
    if (dt == CAST_C64)
        reinterpret_cast<float2 *>(data)[index] = make_float2(1.f, 0.f);
    else
        reinterpret_cast<double2 *>(data)[index] = make_double2(1.0, 0.0);
}

// Every amplitude a pseudo-random value with parts uniform in (-scale, scale)
// (splitmix64 of the index; not normalised): a state on which the kernels'
// value-dependent paths (zero rows, zero parts) behave as on a state in use.
__global__ void k_fill_random(void *data, int dt, uint64_t N, uint64_t seed, float scale) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        // two signed 31-bit integers -> (-1, 1)
        const float re = float(int32_t(uint32_t(z) >> 1) - (1 << 30)) * 0x1p-30f * scale;
        const float im = float(int32_t(uint32_t(z >> 32) >> 1) - (1 << 30)) * 0x1p-30f * scale;
        if (dt == CAST_C64)
            reinterpret_cast<float2 *>(data)[i] = make_float2(re, im);
        else
            reinterpret_cast<double2 *>(data)[i] = make_double2(double(re), double(im));
    }
}

}  // namespace

cast_status launch_fill_random(cast_sv *sv, uint64_t seed) {
    const uint64_t N = uint64_t(1) << sv->n;
    const uint64_t cap = uint64_t(sm_count_cached()) * 8, need = (N + 255) / 256;
    const float scale = std::ldexp(1.0f, -(sv->n + 1) / 2);
    k_fill_random<<<(unsigned)(need < cap ? need : cap), 256, 0, sv->stream>>>(sv->data, sv->dt, N, seed, scale);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

cast_status launch_set_one(cast_sv *sv, uint64_t index) {
    k_set_one<<<1, 1, 0, sv->stream>>>(sv->data, sv->dt, index);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

int sm_count_cached() {
    static std::mutex mu;
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (sms[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms[dev] = v > 0 ? v : 1;
    }
    return sms[dev];
}

int choose_path(const cast_sv *sv, const PreparedGate &g) {
    if (oz_eligible(sv, g)) return CAST_PATH_DIGIT;
    if (sparse_preferred(sv, g)) return CAST_PATH_LIST;
    if (tcc_eligible(sv, g)) return CAST_PATH_TENSOR_CHUNKED;
    if (tc_eligible(sv, g)) return CAST_PATH_TENSOR;
    if (df_eligible(sv, g)) return CAST_PATH_DOUBLE_FLOAT;
    return CAST_PATH_CUDA_CORE;
}

cast_status launch_gate(cast_sv *sv, const PreparedGate &g) {
    switch (choose_path(sv, g)) {
        case CAST_PATH_DIGIT: return launch_gate_oz(sv, g);
        case CAST_PATH_LIST: return launch_gate_sparse(sv, g);
        case CAST_PATH_TENSOR_CHUNKED: return launch_gate_tcc(sv, g);
        case CAST_PATH_TENSOR: return launch_gate_tc(sv, g);
        case CAST_PATH_DOUBLE_FLOAT: return launch_gate_df(sv, g);
        default: return sv->dt == CAST_C64 ? dispatch<float>(sv, g) : dispatch<double>(sv, g);
    }
}

}  // namespace cast
