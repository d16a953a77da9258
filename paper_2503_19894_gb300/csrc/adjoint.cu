// Adjoint differentiation step for a rotation U = exp(-i theta P / 2) on one
// qubit (P in {X, Y, Z}).
//
// With psi_j the state after gate j and lam_j = U_{j+1}^dag ... U_G^dag H psi_G,
//   dE/dtheta_j = 2 Re <lam_j| dU_j/dtheta psi_{j-1}> = Im <lam_j| P |psi_j>,
// because dU/dtheta = (-i/2) P U.  One pass over the amplitude pairs
// (x, x + 2^q) reads psi and lam, accumulates Im(conj(lam) . P psi) with an
// FP64-class accumulator, and writes back U^dag psi and U^dag lam, where
// U^dag = cos(theta/2) I + i sin(theta/2) P.  Each block leaves one partial
// sum; they are reduced in a fixed order afterwards.  complex128 computes in
// double-float arithmetic unless native FP64 is selected.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "device.cuh"
#include "df64.cuh"
#include "internal.h"

namespace cast {
namespace {

// (P v)_0, (P v)_1 for P = X (1), Y (2), Z (3)
template <typename T2>
__device__ __forceinline__ void pauli_pair(int pauli, T2 v0, T2 v1, T2 &o0, T2 &o1) {
    if (pauli == 1) {
        o0 = v1;
        o1 = v0;
    } else if (pauli == 2) {  // Y|0> = i|1>, Y|1> = -i|0>
        o0.x = v1.y;
        o0.y = -v1.x;  // -i v1
        o1.x = -v0.y;
        o1.y = v0.x;   // i v0
    } else {
        o0 = v0;
        o1.x = -v1.x;
        o1.y = -v1.y;
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_adj_rot(typename Cx<R>::T *__restrict__ psi, typename Cx<R>::T *__restrict__ lam, uint64_t npairs,
          int q, int pauli, R c, R s, double *__restrict__ partials) {
    using T2 = typename Cx<R>::T;
    constexpr int UNR = 2;
    Acc<R> acc;
    const uint64_t bit = uint64_t(1) << q;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t0 < npairs; t0 += stride * UNR) {
        T2 p0[UNR], p1[UNR], l0[UNR], l1[UNR];
        uint64_t i0[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t t = t0 + uint64_t(u) * stride;
            i0[u] = ((t >> q) << (q + 1)) | (t & (bit - 1));
            if (t < npairs) {
                p0[u] = psi[i0[u]];
                p1[u] = psi[i0[u] | bit];
                l0[u] = lam[i0[u]];
                l1[u] = lam[i0[u] | bit];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (t0 + uint64_t(u) * stride >= npairs) continue;
            T2 pp0, pp1, pl0, pl1;
            pauli_pair(pauli, p0[u], p1[u], pp0, pp1);
            pauli_pair(pauli, l0[u], l1[u], pl0, pl1);
            // Im(conj(l) * pp) = l.x * pp.y - l.y * pp.x
            acc.add(l0[u].x * pp0.y - l0[u].y * pp0.x);
            acc.add(l1[u].x * pp1.y - l1[u].y * pp1.x);
            // U^dag v = c v + i s (P v)
            T2 o;
            o.x = c * p0[u].x - s * pp0.y; o.y = c * p0[u].y + s * pp0.x; psi[i0[u]] = o;
            o.x = c * p1[u].x - s * pp1.y; o.y = c * p1[u].y + s * pp1.x; psi[i0[u] | bit] = o;
            o.x = c * l0[u].x - s * pl0.y; o.y = c * l0[u].y + s * pl0.x; lam[i0[u]] = o;
            o.x = c * l1[u].x - s * pl1.y; o.y = c * l1[u].y + s * pl1.x; lam[i0[u] | bit] = o;
        }
    }
    const double v = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// The same step for complex128 in double-float arithmetic on the FP32 pipe
// (df64.cuh): the FP64 pipe of this part would make the step arithmetic-bound
// at twice its memory time.  c, s arrive as (hi, lo) pairs.
__device__ __forceinline__ void pauli_pair_df(int pauli, const df::CF &v0, const df::CF &v1, df::CF &o0, df::CF &o1) {
    if (pauli == 1) {
        o0 = v1;
        o1 = v0;
    } else if (pauli == 2) {  // Y|0> = i|1>, Y|1> = -i|0>
        o0 = {v1.ih, v1.il, -v1.rh, -v1.rl};  // -i v1
        o1 = {-v0.ih, -v0.il, v0.rh, v0.rl};  // i v0
    } else {
        o0 = v0;
        o1 = {-v1.rh, -v1.rl, -v1.ih, -v1.il};
    }
}

// U^dag v = c v + i s (P v)
__device__ __forceinline__ double2 rot_df(const df::CF &v, const df::CF &pv, float ch, float cl, float sh, float sl) {
    df::CF o = {0.f, 0.f, 0.f, 0.f};
    df::mac(o.rh, o.rl, ch, cl, v.rh, v.rl);
    df::msub(o.rh, o.rl, sh, sl, pv.ih, pv.il);
    df::mac(o.ih, o.il, ch, cl, v.ih, v.il);
    df::mac(o.ih, o.il, sh, sl, pv.rh, pv.rl);
    return df::join_c(o);
}

__global__ void __launch_bounds__(256)
k_adj_rot_df(double2 *__restrict__ psi, double2 *__restrict__ lam, uint64_t npairs, int q, int pauli, float ch,
             float cl, float sh, float sl, double *__restrict__ partials) {
    constexpr int UNR = 2;
    float gh = 0.f, gl = 0.f;  // double-float sum of Im(conj(l) . P p)
    const uint64_t bit = uint64_t(1) << q;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t t0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; t0 < npairs; t0 += stride * UNR) {
        double2 p0[UNR], p1[UNR], l0[UNR], l1[UNR];
        uint64_t i0[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t t = t0 + uint64_t(u) * stride;
            i0[u] = ((t >> q) << (q + 1)) | (t & (bit - 1));
            if (t < npairs) {
                p0[u] = psi[i0[u]];
                p1[u] = psi[i0[u] | bit];
                l0[u] = lam[i0[u]];
                l1[u] = lam[i0[u] | bit];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            if (t0 + uint64_t(u) * stride >= npairs) continue;
            const df::CF a0 = df::split_c(p0[u]), a1 = df::split_c(p1[u]);
            const df::CF b0 = df::split_c(l0[u]), b1 = df::split_c(l1[u]);
            df::CF pa0, pa1, pb0, pb1;
            pauli_pair_df(pauli, a0, a1, pa0, pa1);
            pauli_pair_df(pauli, b0, b1, pb0, pb1);
            // Im(conj(l) * pp) = l.re * pp.im - l.im * pp.re
            df::mac(gh, gl, b0.rh, b0.rl, pa0.ih, pa0.il);
            df::msub(gh, gl, b0.ih, b0.il, pa0.rh, pa0.rl);
            df::mac(gh, gl, b1.rh, b1.rl, pa1.ih, pa1.il);
            df::msub(gh, gl, b1.ih, b1.il, pa1.rh, pa1.rl);
            psi[i0[u]] = rot_df(a0, pa0, ch, cl, sh, sl);
            psi[i0[u] | bit] = rot_df(a1, pa1, ch, cl, sh, sl);
            lam[i0[u]] = rot_df(b0, pb0, ch, cl, sh, sl);
            lam[i0[u] | bit] = rot_df(b1, pb1, ch, cl, sh, sl);
        }
    }
    const double v = block_sum(double(gh) + double(gl));
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// grad[p] = sum of the gate values whose parameter index is p, in gate order
__global__ void k_param_sum(const double *__restrict__ gate_vals, const int *__restrict__ gate_pidx,
                            int ngates, double *__restrict__ grad, int nparams) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparams) return;
    double s = 0.0;
    for (int g = 0; g < ngates; g++)
        if (gate_pidx[g] == p) s += gate_vals[g];
    grad[p] = s;
}

}  // namespace

cast_status launch_adjoint_rotation(cast_sv *psi, cast_sv *lam, int q, int pauli, double theta,
                                    double *d_partials) {
    const uint64_t npairs = uint64_t(1) << (psi->n - 1);
    const int G = reduce_grid_blocks();
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    ProfScope ps(psi->stream, std::string("adj_rot_") + dt_name(psi->dt),
                 4.0 * double(amp_bytes(psi->dt)) * double(npairs * 2), 28.0 * double(npairs * 2));
    if (psi->dt == CAST_C64)
        k_adj_rot<float><<<G, 256, 0, psi->stream>>>(reinterpret_cast<float2 *>(psi->data),
                                                      reinterpret_cast<float2 *>(lam->data), npairs, q,
                                                      pauli, (float)c, (float)s, d_partials);
    else if (f64_mode() == CAST_F64_EMULATED) {
        const float ch = float(c), cl = float(c - double(ch)), sh = float(s), sl = float(s - double(sh));
        k_adj_rot_df<<<G, 256, 0, psi->stream>>>(reinterpret_cast<double2 *>(psi->data),
                                                 reinterpret_cast<double2 *>(lam->data), npairs, q, pauli, ch, cl,
                                                 sh, sl, d_partials);
    } else
        k_adj_rot<double><<<G, 256, 0, psi->stream>>>(reinterpret_cast<double2 *>(psi->data),
                                                       reinterpret_cast<double2 *>(lam->data), npairs, q,
                                                       pauli, c, s, d_partials);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

cast_status launch_param_sum(cudaStream_t st, const double *gate_vals, const int *gate_pidx, int ngates,
                             double *grad, int nparams) {
    if (nparams <= 0) return CAST_OK;
    k_param_sum<<<(nparams + 127) / 128, 128, 0, st>>>(gate_vals, gate_pidx, ngates, grad, nparams);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

}  // namespace cast
