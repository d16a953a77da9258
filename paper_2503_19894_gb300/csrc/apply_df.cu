// complex128 gates computed in double-float arithmetic on the FP32 pipe
// (see df64.cuh): dense k <= 5, diagonal and monomial gates.  Same slice
// enumeration (Eq. 4) and launch shapes as the FP64 kernels in apply.cu; the
// state stays complex128 in memory, the matrix travels as (hi, lo) pairs of
// its real and imaginary parts in the launch parameters.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>

#include "device.cuh"
#include "df64.cuh"
#include "internal.h"

namespace cast {
namespace {

std::atomic<int> g_f64_mode{CAST_F64_EMULATED};

using df::CF;
using df::cmac;
using df::join_c;
using df::split_c;

CF host_split(cplx z) {
    CF c;
    c.rh = (float)z.real();
    c.rl = (float)(z.real() - (double)c.rh);
    c.ih = (float)z.imag();
    c.il = (float)(z.imag() - (double)c.ih);
    return c;
}

template <int K>
struct DfMat {
    CF m[1 << K][1 << K];
};

template <int K>
__global__ void __launch_bounds__(256)
k_dense_df(double2 *__restrict__ sv, uint64_t nslices, Targets tg, const __grid_constant__ DfMat<K> U) {
    constexpr int D = 1 << K;
    uint64_t p[K];
#pragma unroll
    for (int i = 0; i < K; i++) p[i] = uint64_t(1) << tg.q[i];
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nslices; t += stride) {
        const uint64_t base = slice_base<K>(t, tg);
        CF x[D];
#pragma unroll
        for (int j = 0; j < D; j++) {
            uint64_t off = 0;
#pragma unroll
            for (int i = 0; i < K; i++)
                if ((j >> i) & 1) off += p[i];
            x[j] = split_c(sv[base + off]);
        }
#pragma unroll
        for (int r = 0; r < D; r++) {
            CF acc = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < D; c++) cmac(acc, U.m[r][c], x[c]);
            uint64_t off = 0;
#pragma unroll
            for (int i = 0; i < K; i++)
                if ((r >> i) & 1) off += p[i];
            sv[base + off] = join_c(acc);
        }
    }
}

template <int K>
struct DfDiag {
    CF d[1 << K];
    uint32_t skip;  // bit j: entry j is 1 (amplitudes untouched); K <= 5
};

template <int K>
__global__ void __launch_bounds__(256)
k_diag_df(double2 *__restrict__ sv, uint64_t N, Targets tg, const __grid_constant__ DfDiag<K> Dg) {
    constexpr int UNR = 4;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x0 < N; x0 += stride * UNR) {
        double2 v[UNR];
        int j[UNR];
        bool act[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t x = x0 + uint64_t(u) * stride;
            act[u] = false;
            if (x < N) {
                int jj = 0;
#pragma unroll
                for (int b = 0; b < K; b++) jj |= int((x >> tg.q[b]) & 1) << b;
                j[u] = jj;
                act[u] = (K > 5) || !((Dg.skip >> jj) & 1);
                if (act[u]) v[u] = sv[x];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (!act[u]) continue;
            CF acc = {0.f, 0.f, 0.f, 0.f};
            cmac(acc, Dg.d[j[u]], split_c(v[u]));
            sv[x0 + uint64_t(u) * stride] = join_c(acc);
        }
    }
}

// Chunked form for states of at least 2^11 amplitudes (as k_diag_chunk in
// apply.cu): a CTA iteration covers 256 x 8 consecutive amplitudes (thread t
// takes t, t + 256, ...); the diagonal index is the OR of the chunk's part,
// the thread's part and the round's part (rounds from the launch parameters).
struct DfChunkBits {
    int jr[8];
};

template <int K>
__global__ void __launch_bounds__(256)
k_diag_df_chunk(double2 *__restrict__ sv, uint64_t nchunks, const __grid_constant__ Targets tg,
                const __grid_constant__ DfDiag<K> Dg, const __grid_constant__ DfChunkBits cb) {
    constexpr int UNR = 8, CB = 11;
    auto jbits = [&](uint64_t x) {
        int j = 0;
#pragma unroll
        for (int b = 0; b < K; b++) j |= int((x >> tg.q[b]) & 1) << b;
        return j;
    };
    const int jt = jbits(uint64_t(threadIdx.x));
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint64_t base = c << CB;
        const int jh = jbits(base) | jt;
        double2 *p = sv + base + threadIdx.x;
        uint32_t act = 0;
#pragma unroll
        for (int u = 0; u < UNR; u++) act |= uint32_t(K > 5 || !((Dg.skip >> (jh | cb.jr[u])) & 1)) << u;
        double2 v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++)
            if ((act >> u) & 1) v[u] = p[256 * u];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (!((act >> u) & 1)) continue;
            CF acc = {0.f, 0.f, 0.f, 0.f};
            cmac(acc, Dg.d[jh | cb.jr[u]], split_c(v[u]));
            p[256 * u] = join_c(acc);
        }
    }
}

template <int K>
struct DfMono {
    CF ph[1 << K];
    uint8_t perm[1 << K];
};

// monomial with non-unit phases (unit-phase permutations stay in apply.cu)
template <int K>
__global__ void __launch_bounds__(256)
k_mono_df(double2 *__restrict__ sv, uint64_t nslices, Targets tg, const __grid_constant__ DfMono<K> M) {
    constexpr int D = 1 << K;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nslices; t += stride) {
        const uint64_t base = slice_base<K>(t, tg);
        double2 v[D];
#pragma unroll
        for (int r = 0; r < D; r++) v[r] = sv[base + member_offset<K>(M.perm[r], tg)];
#pragma unroll
        for (int r = 0; r < D; r++) {
            CF acc = {0.f, 0.f, 0.f, 0.f};
            cmac(acc, M.ph[r], split_c(v[r]));
            sv[base + member_offset<K>(r, tg)] = join_c(acc);
        }
    }
}

uint64_t grid_for(uint64_t items, int per_sm) {
    const uint64_t cap = uint64_t(sm_count_cached()) * per_sm;
    uint64_t need = (items + 255) / 256;
    if (need < 1) need = 1;
    return need < cap ? need : cap;
}

template <int K>
cast_status run_k(cast_sv *sv, const PreparedGate &g) {
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    double2 *data = reinterpret_cast<double2 *>(sv->data);
    const uint64_t N = uint64_t(1) << sv->n, ns = N >> K;
    if (g.cls == CLS_DENSE) {
        DfMat<K> U;
        for (int r = 0; r < (1 << K); r++)
            for (int c = 0; c < (1 << K); c++) U.m[r][c] = host_split(g.m[size_t(r) * (1 << K) + c]);
        ProfScope ps(sv->stream, "dfdense_k" + std::to_string(K) + "_c128", 32.0 * double(N),
                     8.0 * double(N << K));
        k_dense_df<K><<<(unsigned)grid_for(ns, tuned_blocks_per_sm(CAST_C128, K, CLS_DENSE, K <= 2 ? 8 : 4)), 256, 0,
                        sv->stream>>>(data, ns, tg, U);
    } else if (g.cls == CLS_DIAG) {
        DfDiag<K> Dg;
        Dg.skip = 0;
        int touched = 0;
        for (int j = 0; j < (1 << K); j++) {
            Dg.d[j] = host_split(g.diag[j]);
            const bool unit = g.diag[j] == cplx(1.0, 0.0);
            if (unit) Dg.skip |= 1u << j;
            touched += !unit;
        }
        const double frac = double(touched) / double(1 << K);
        ProfScope ps(sv->stream, "dfdiag_k" + std::to_string(K) + "_c128", 32.0 * double(N) * frac,
                     6.0 * double(N) * frac);
        if (sv->n >= 11) {
            DfChunkBits cb{};
            for (int u = 0; u < 8; u++)
                for (int b = 0; b < K; b++) cb.jr[u] |= int(((uint64_t(u) << 8) >> g.q[b]) & 1) << b;
            const uint64_t nchunks = N >> 11;
            const uint64_t cap = uint64_t(sm_count_cached()) * tuned_blocks_per_sm(CAST_C128, K, CLS_DIAG, 8);
            k_diag_df_chunk<K><<<(unsigned)(nchunks < cap ? nchunks : cap), 256, 0, sv->stream>>>(data, nchunks, tg,
                                                                                                  Dg, cb);
        } else {
            k_diag_df<K><<<(unsigned)grid_for(N / 4, tuned_blocks_per_sm(CAST_C128, K, CLS_DIAG, 8)), 256, 0,
                           sv->stream>>>(data, N, tg, Dg);
        }
    } else {
        DfMono<K> M;
        for (int j = 0; j < (1 << K); j++) {
            M.ph[j] = host_split(g.phase[j]);
            M.perm[j] = (uint8_t)g.perm[j];
        }
        ProfScope ps(sv->stream, "dfmono_k" + std::to_string(K) + "_c128", 32.0 * double(N), 6.0 * double(N));
        k_mono_df<K><<<(unsigned)grid_for(ns, tuned_blocks_per_sm(CAST_C128, K, CLS_MONO, 8)), 256, 0,
                       sv->stream>>>(data, ns, tg, M);
    }
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace

bool df_eligible(const cast_sv *sv, const PreparedGate &g) {
    if (g_f64_mode.load() != CAST_F64_EMULATED || sv->dt != CAST_C128 || g.k > 5) return false;
    if (g.cls == CLS_DENSE || g.cls == CLS_DIAG) return true;
    return g.cls == CLS_MONO && !g.unit_phases;
}

cast_status launch_gate_df(cast_sv *sv, const PreparedGate &g) {
    switch (g.k) {
        case 1: return run_k<1>(sv, g);
        case 2: return run_k<2>(sv, g);
        case 3: return run_k<3>(sv, g);
        case 4: return run_k<4>(sv, g);
        case 5: return run_k<5>(sv, g);
        default: return fail(CAST_ERR_UNSUPPORTED, "double-float path covers k <= 5");
    }
}

int f64_mode() { return g_f64_mode.load(); }

}  // namespace cast

extern "C" {

cast_status cast_set_f64_mode(int mode) {
    if (mode != CAST_F64_EMULATED && mode != CAST_F64_NATIVE) return cast::fail(CAST_ERR_ARG, "unknown FP64 mode");
    cast::g_f64_mode = mode;
    return CAST_OK;
}

int cast_get_f64_mode(void) { return cast::g_f64_mode.load(); }

}  // extern "C"
