// Reductions over a state: Pauli-sum expectation values, inner products, and
// lambda = H |psi> for adjoint differentiation.
//
// A Pauli string is encoded by two masks (x: X or Y on the qubit, z: Z or Y).
// P|x> = i^{ny} (-1)^{popc(x & z)} |x ^ xm>, ny = popc(xm & zm), hence
//   <psi|P|psi> = sum_x conj(psi[x ^ xm]) psi[x] i^{ny} (-1)^{popc(x & z)}.
// Terms that share x_mask are evaluated in one pass over the state.
//
// Accumulation is FP64-class for both state types: complex128 states
// accumulate in FP64; complex64 states form each product in FP32 and add it to
// a compensated (hi, lo) FP32 pair with Knuth's TwoSum (error-free
// transformation), converted to FP64 once per thread.  GB300's FP64 pipe runs
// at about 1/67 of the FP32 rate, so an FP64 add per complex64 amplitude would
// make these passes compute-bound.  Partial sums (one per block) are reduced in
// a fixed order by k_finalize, so results are bit-reproducible run to run.
#include <cuda_runtime.h>

#include <string>

#include "internal.h"
#include "device.cuh"

namespace cast {

__global__ void k_finalize(const double *__restrict__ partials, int per_slot, int nslots,
                           double *__restrict__ out) {
    // one block per output slot; fixed summation order
    for (int s = blockIdx.x; s < nslots; s += gridDim.x) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < per_slot; i += blockDim.x) acc += partials[size_t(s) * per_slot + i];
        acc = block_sum(acc);
        if (threadIdx.x == 0) out[s] = acc;
        __syncthreads();
    }
}

namespace {

constexpr int kMaxTerms = 32;

template <typename R>
struct PauliGroupParams {
    uint64_t xm;
    int nt;
    uint64_t z[kMaxTerms];
    R cr[kMaxTerms];  // coefficient times Re(i^ny)
    R ci[kMaxTerms];  // coefficient times -Im(i^ny)
};

// sum_x [A(x) Re w(x) + B(x) Im w(x)],  w = conj(psi[x ^ xm]) psi[x].
// UNR independent loads per thread per round keep enough bytes in flight.
template <typename R>
__global__ void __launch_bounds__(256)
k_pauli(const typename Cx<R>::T *__restrict__ sv, uint64_t N,
        const __grid_constant__ PauliGroupParams<R> P, double *__restrict__ partials) {
    using T2 = typename Cx<R>::T;
    constexpr int UNR = 8;
    // two independent accumulators (alternating rounds) shorten the
    // dependency chain; each round's UNR products are summed in the state's
    // precision first, then added to the compensated accumulator once
    Acc<R> acc0, acc1;
    int round = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x0 < N; x0 += stride * UNR, round++) {
        T2 a[UNR], b[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t x = x0 + uint64_t(u) * stride;
            if (x < N) {
                a[u] = sv[x];
                b[u] = P.xm ? sv[x ^ P.xm] : a[u];
            }
        }
        R part = 0;
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t x = x0 + uint64_t(u) * stride;
            if (x >= N) continue;
            const R wr = b[u].x * a[u].x + b[u].y * a[u].y;
            const R wi = b[u].x * a[u].y - b[u].y * a[u].x;
            R A = 0, B = 0;
            for (int t = 0; t < P.nt; t++) {
                const bool odd = __popcll(x & P.z[t]) & 1;
                A += odd ? -P.cr[t] : P.cr[t];
                B += odd ? -P.ci[t] : P.ci[t];
            }
            part += A * wr + B * wi;
        }
        if (round & 1) acc1.add(part);
        else acc0.add(part);
    }
    double v = block_sum(acc0.value() + acc1.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// <a|b> as two partial arrays (re, im)
template <typename R>
__global__ void __launch_bounds__(256)
k_inner(const typename Cx<R>::T *__restrict__ a, const typename Cx<R>::T *__restrict__ b, uint64_t N,
        double *__restrict__ partials_re, double *__restrict__ partials_im) {
    using T2 = typename Cx<R>::T;
    constexpr int UNR = 4;
    Acc<R> re, im;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x0 < N; x0 += stride * UNR) {
        T2 u[UNR], v[UNR];
#pragma unroll
        for (int k = 0; k < UNR; k++) {
            const uint64_t x = x0 + uint64_t(k) * stride;
            if (x < N) { u[k] = a[x]; v[k] = b[x]; }
        }
#pragma unroll
        for (int k = 0; k < UNR; k++) {
            if (x0 + uint64_t(k) * stride >= N) continue;
            re.add(u[k].x * v[k].x);
            re.add(u[k].y * v[k].y);
            im.add(u[k].x * v[k].y);
            im.add(-u[k].y * v[k].x);
        }
    }
    double r = block_sum(re.value());
    double i = block_sum(im.value());
    if (threadIdx.x == 0) {
        partials_re[blockIdx.x] = r;
        partials_im[blockIdx.x] = i;
    }
}

// out[x] (=|+=) sum_t c_t i^{ny_t} (-1)^{popc((x ^ xm) & z_t)} psi[x ^ xm]
template <typename R>
__global__ void __launch_bounds__(256)
k_pauli_apply(const typename Cx<R>::T *__restrict__ psi, typename Cx<R>::T *__restrict__ out,
              uint64_t N, const __grid_constant__ PauliGroupParams<R> P, int accumulate) {
    using T2 = typename Cx<R>::T;
    constexpr int UNR = 4;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x0 < N; x0 += stride * UNR) {
        T2 v[UNR], o[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t x = x0 + uint64_t(u) * stride;
            if (x < N) {
                v[u] = psi[x ^ P.xm];
                if (accumulate) o[u] = out[x];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const uint64_t x = x0 + uint64_t(u) * stride;
            if (x >= N) continue;
            const uint64_t src = x ^ P.xm;
            // factor f = sum_t (-1)^{popc(src & z_t)} c_t i^{ny_t} = fr + i fi
            R fr = 0, fi = 0;
            for (int t = 0; t < P.nt; t++) {
                const bool odd = __popcll(src & P.z[t]) & 1;
                fr += odd ? -P.cr[t] : P.cr[t];
                fi += odd ? P.ci[t] : -P.ci[t];
            }
            T2 y;
            y.x = fr * v[u].x - fi * v[u].y;
            y.y = fr * v[u].y + fi * v[u].x;
            if (accumulate) {
                y.x += o[u].x;
                y.y += o[u].y;
            }
            out[x] = y;
        }
    }
}

template <typename R>
void fill_group(PauliGroupParams<R> *P, uint64_t xm, int nt, const double *coeffs, const uint64_t *zm) {
    P->xm = xm;
    P->nt = nt;
    for (int t = 0; t < kMaxTerms; t++) {
        P->z[t] = 0;
        P->cr[t] = 0;
        P->ci[t] = 0;
    }
    for (int t = 0; t < nt; t++) {
        const int ny = __builtin_popcountll(xm & zm[t]) & 3;
        // Re(i^ny w) = cr*Re w + ci*Im w with (cr, ci) = (1,0), (0,-1), (-1,0), (0,1)
        const double re[4] = {1, 0, -1, 0}, im[4] = {0, -1, 0, 1};
        P->z[t] = zm[t];
        P->cr[t] = (R)(coeffs[t] * re[ny]);
        P->ci[t] = (R)(coeffs[t] * im[ny]);
    }
}

}  // namespace

int reduce_grid_blocks() { return sm_count_cached() * 4; }

size_t pauli_partials_needed(const PauliGroups &G) {
    size_t launches = 0;
    for (size_t g = 0; g < G.xm.size(); g++) launches += (G.c[g].size() + kMaxTerms - 1) / kMaxTerms;
    return launches * size_t(reduce_grid_blocks());
}

cast_status launch_pauli_group(const cast_sv *sv, uint64_t xm, int nt, const double *coeffs,
                               const uint64_t *zm, double *d_partials, int *n_partials) {
    const uint64_t N = uint64_t(1) << sv->n;
    const int G = reduce_grid_blocks();
    int done = 0;
    for (int start = 0; start < nt; start += kMaxTerms) {
        const int cnt = nt - start < kMaxTerms ? nt - start : kMaxTerms;
        ProfScope ps(sv->stream, std::string("pauli_") + dt_name(sv->dt), double(amp_bytes(sv->dt)) * double(N),
                     double(N) * (8.0 + 2.0 * cnt));
        if (sv->dt == CAST_C64) {
            PauliGroupParams<float> P;
            fill_group(&P, xm, cnt, coeffs + start, zm + start);
            k_pauli<float><<<G, 256, 0, sv->stream>>>(reinterpret_cast<const float2 *>(sv->data), N, P,
                                                       d_partials + size_t(done) * G);
        } else {
            PauliGroupParams<double> P;
            fill_group(&P, xm, cnt, coeffs + start, zm + start);
            k_pauli<double><<<G, 256, 0, sv->stream>>>(reinterpret_cast<const double2 *>(sv->data), N, P,
                                                        d_partials + size_t(done) * G);
        }
        CAST_CUDA(cudaGetLastError());
        done++;
    }
    *n_partials = done * G;
    return CAST_OK;
}

cast_status launch_finalize(cudaStream_t st, const double *d_partials, int per_slot, int nslots,
                            double *d_out) {
    const int grid = nslots < 1024 ? nslots : 1024;
    k_finalize<<<grid, 256, 0, st>>>(d_partials, per_slot, nslots, d_out);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

cast_status launch_inner(const cast_sv *a, const cast_sv *b, double *d_partials_re, double *d_partials_im) {
    const uint64_t N = uint64_t(1) << a->n;
    const int G = reduce_grid_blocks();
    ProfScope ps(a->stream, std::string("inner_") + dt_name(a->dt), 2.0 * double(amp_bytes(a->dt)) * double(N),
                 8.0 * double(N));
    if (a->dt == CAST_C64)
        k_inner<float><<<G, 256, 0, a->stream>>>(reinterpret_cast<const float2 *>(a->data),
                                                  reinterpret_cast<const float2 *>(b->data), N,
                                                  d_partials_re, d_partials_im);
    else
        k_inner<double><<<G, 256, 0, a->stream>>>(reinterpret_cast<const double2 *>(a->data),
                                                   reinterpret_cast<const double2 *>(b->data), N,
                                                   d_partials_re, d_partials_im);
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

cast_status launch_pauli_apply(const cast_sv *psi, cast_sv *out, uint64_t xm, int nt, const double *coeffs,
                               const uint64_t *zm, bool accumulate) {
    const uint64_t N = uint64_t(1) << psi->n;
    const int G = reduce_grid_blocks() * 2;
    bool acc = accumulate;
    for (int start = 0; start < nt; start += kMaxTerms) {
        const int cnt = nt - start < kMaxTerms ? nt - start : kMaxTerms;
        ProfScope ps(psi->stream, std::string("pauli_apply_") + dt_name(psi->dt),
                     double(amp_bytes(psi->dt)) * double(N) * (acc ? 3.0 : 2.0), double(N) * (6.0 + 2.0 * cnt));
        if (psi->dt == CAST_C64) {
            PauliGroupParams<float> P;
            fill_group(&P, xm, cnt, coeffs + start, zm + start);
            k_pauli_apply<float><<<G, 256, 0, psi->stream>>>(reinterpret_cast<const float2 *>(psi->data),
                                                              reinterpret_cast<float2 *>(out->data), N, P,
                                                              acc ? 1 : 0);
        } else {
            PauliGroupParams<double> P;
            fill_group(&P, xm, cnt, coeffs + start, zm + start);
            k_pauli_apply<double><<<G, 256, 0, psi->stream>>>(reinterpret_cast<const double2 *>(psi->data),
                                                               reinterpret_cast<double2 *>(out->data), N, P,
                                                               acc ? 1 : 0);
        }
        CAST_CUDA(cudaGetLastError());
        acc = true;
    }
    return CAST_OK;
}

}  // namespace cast
