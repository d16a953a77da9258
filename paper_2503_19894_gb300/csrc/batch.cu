// Batched variational circuits of any shape: many instances, each with its own
// qubit count, gate list (1- and 2-qubit gates, fixed or RX/RY/RZ carrying a
// parameter) and Pauli sum, evaluated together (the training form of the
// paper's Eq. 3 that its VQA motivation calls for; the hardware-efficient
// ansatz has the faster tile executor in hea.cu).
//
// Layout: every instance's state sits in one arena (offsets multiples of 256
// amplitudes).  Gate step s applies the s-th gate of every instance that has
// one, in a single launch whose work items are the slices of all those
// instances (an entry table per step: first work item, state offset, qubits,
// matrix slot, parameter); a work item finds its entry by binary search.
// Rotation matrices are formed on the device from the parameters at the start
// of every replay, so the whole launch sequence (initial states, gate steps,
// energies; for gradients also lambda = H psi and the backward sweep) is
// captured once into a CUDA graph and replayed per parameter set.
//
// Energies: one pass over every instance's amplitudes, each thread summing
// c_t Re(conj(psi[x ^ xm_t]) phase_t(x) psi[x]) over its instance's terms in
// FP64; warps add into the instance's slot with FP64 atomics.  Gradients:
// lambda = H psi, then steps in reverse; a step forms Im<lambda|P_q|psi> for
// every rotation in it (the derivative of exp(-i theta P / 2), accumulated in
// FP64 into the parameter's slot) and un-applies each gate from psi and lambda
// in the same pass.
//
// complex64 runs in FP32 (products summed per thread in FP32, per-slice sums
// in FP64); complex128 in double-float arithmetic on the FP32 pipe
// (df64.cuh), the arena holding FP64 amplitudes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "df64.cuh"
#include "internal.h"

namespace cast {
namespace {

constexpr int kBThreads = 256;

// kind of a step entry
enum : int32_t { BK_FIXED = 0, BK_RX = 1, BK_RY = 2, BK_RZ = 3 };

struct BEntry {
    uint64_t work0;  // first work item (slice) of this entry within the step
    uint64_t off;    // state offset (amplitudes)
    int32_t inst;
    int32_t k;       // 1 or 2
    int32_t q0, q1;  // qubits (q1 unused for k = 1); bit i of the matrix index <-> q_i
    int32_t mat;     // matrix slot (16 complex entries)
    int32_t kind;    // BK_FIXED or the rotation's generator
    int32_t param;   // parameter index (global), -1 if fixed
};

struct BTerm {
    double c;
    uint64_t xm, zm;
};

__device__ __forceinline__ int find_entry(const BEntry *e, int count, uint64_t w) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e[mid].work0 <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t t, int q) {
    return ((t >> q) << (q + 1)) | (t & ((uint64_t(1) << q) - 1));
}

// ---------------------------------------------------------- arithmetic
struct BA64 {
    using Amp = float2;
    using V = float2;
    __device__ static V in(Amp a) { return a; }
    __device__ static Amp out(V v) { return v; }
    __device__ static V mul(double2 u, V x) {
        const float ur = float(u.x), ui = float(u.y);
        return make_float2(ur * x.x - ui * x.y, ur * x.y + ui * x.x);
    }
    __device__ static V add(V a, V b) { return make_float2(a.x + b.x, a.y + b.y); }
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    // conj(a) * b (re, im) for the gradient sums; converted once per slice
    __device__ static double2 cdot(V a, V b) {
        return make_double2(double(a.x * b.x + a.y * b.y), double(a.x * b.y - a.y * b.x));
    }
    __device__ static V scale(V a, double2 c) { return mul(c, a); }
    // energies: c Re(ph conj(a) b) summed per thread in FP32, then once to FP64
    using Acc = float;
    __device__ static float term(Amp a, Amp b, double2 ph, double c) {
        const float dr = a.x * b.x + a.y * b.y, di = a.x * b.y - a.y * b.x;
        return float(c) * (float(ph.x) * dr - float(ph.y) * di);
    }
};

struct BA128 {
    using Amp = double2;
    using V = df::CF;
    __device__ static V in(Amp a) { return df::split_c(a); }
    __device__ static Amp out(V v) { return df::join_c(v); }
    __device__ static V cf(double2 u) {
        const float rh = float(u.x), ih = float(u.y);
        return {rh, float(u.x - double(rh)), ih, float(u.y - double(ih))};
    }
    __device__ static V mul(double2 u, V x) {
        V acc = {0.f, 0.f, 0.f, 0.f};
        df::cmac(acc, cf(u), x);
        return acc;
    }
    __device__ static V add(V a, V b) {
        V r = a;
        auto two = [](float &sh, float &sl, float xh, float xl) {
            const float s = sh + xh, bb = s - sh;
            const float t = (sh - (s - bb)) + (xh - bb);
            sh = s;
            sl += t + xl;
        };
        two(r.rh, r.rl, b.rh, b.rl);
        two(r.ih, r.il, b.ih, b.il);
        return r;
    }
    __device__ static V zero() { return {0.f, 0.f, 0.f, 0.f}; }
    __device__ static double2 cdot(V a, V b) {
        const double ar = double(a.rh) + double(a.rl), ai = double(a.ih) + double(a.il);
        const double br = double(b.rh) + double(b.rl), bi = double(b.ih) + double(b.il);
        return make_double2(ar * br + ai * bi, ar * bi - ai * br);
    }
    __device__ static V scale(V a, double2 c) { return mul(c, a); }
    // energies in FP64 on the stored amplitudes
    using Acc = double;
    __device__ static double term(Amp a, Amp b, double2 ph, double c) {
        const double dr = a.x * b.x + a.y * b.y, di = a.x * b.y - a.y * b.x;
        return c * (ph.x * dr - ph.y * di);
    }
};

// ------------------------------------------------------------- kernels
// Rotation matrices of this replay: exp(-i theta P / 2) into their slots.
__global__ void k_batch_prep(const BEntry *entries, int n, const double *params, double2 *mats) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BEntry e = entries[i];
    if (e.kind == BK_FIXED) return;
    double s, c;
    sincos(0.5 * params[e.param], &s, &c);
    double2 *m = mats + size_t(e.mat) * 16;
    for (int j = 0; j < 16; j++) m[j] = make_double2(0.0, 0.0);
    if (e.kind == BK_RX) {
        m[0] = make_double2(c, 0); m[1] = make_double2(0, -s); m[2] = make_double2(0, -s); m[3] = make_double2(c, 0);
    } else if (e.kind == BK_RY) {
        m[0] = make_double2(c, 0); m[1] = make_double2(-s, 0); m[2] = make_double2(s, 0); m[3] = make_double2(c, 0);
    } else {
        m[0] = make_double2(c, -s); m[3] = make_double2(c, s);
    }
}

__global__ void k_batch_set_zero_state(void *arena, int amp_bytes, const uint64_t *offs, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
    if (amp_bytes == 8) reinterpret_cast<float2 *>(arena)[offs[i]] = make_float2(1.f, 0.f);
    else reinterpret_cast<double2 *>(arena)[offs[i]] = make_double2(1.0, 0.0);
}

// u (row-major 2^k x 2^k) or its adjoint applied to slice amplitudes v
template <class A>
__device__ __forceinline__ void apply_small(const double2 *u, int k, bool adj, typename A::V (&v)[4]) {
    using V = typename A::V;
    const int d = 1 << k;
    V y[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (r >= d) break;
        V acc = A::zero();
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (c >= d) break;
            double2 m = adj ? u[c * d + r] : u[r * d + c];
            if (adj) m.y = -m.y;
            if (m.x == 0.0 && m.y == 0.0) continue;
            acc = A::add(acc, A::mul(m, v[c]));
        }
        y[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
        if (r < d) v[r] = y[r];
}

template <class A>
__device__ __forceinline__ void slice_addr(const BEntry &e, uint64_t t, uint64_t (&a)[4]) {
    if (e.k == 1) {
        const uint64_t b = e.off + insert_zero(t, e.q0);
        a[0] = b;
        a[1] = b + (uint64_t(1) << e.q0);
    } else {
        const int lo = min(e.q0, e.q1), hi = max(e.q0, e.q1);
        const uint64_t b = e.off + insert_zero(insert_zero(t, lo), hi);
        const uint64_t p0 = uint64_t(1) << e.q0, p1 = uint64_t(1) << e.q1;
        a[0] = b;
        a[1] = b + p0;
        a[2] = b + p1;
        a[3] = b + p0 + p1;
    }
}

// one gate step: the step's entries (one per participating instance)
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_gate(typename A::Amp *__restrict__ psi, const BEntry *__restrict__ entries, int count, uint64_t total,
             const double2 *__restrict__ mats) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total; w += stride) {
        const BEntry e = entries[find_entry(entries, count, w)];
        uint64_t a[4];
        slice_addr<A>(e, w - e.work0, a);
        typename A::V v[4];
        const int d = 1 << e.k;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d) v[j] = A::in(psi[a[j]]);
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, false, v);
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d) psi[a[j]] = A::out(v[j]);
    }
}

__device__ __forceinline__ double2 pauli_phase(uint64_t x, uint64_t xm, uint64_t zm) {
    // P|x> = i^ny (-1)^{popc(x & zm)} |x ^ xm>, ny = popc(xm & zm)
    const int ny = __popcll(xm & zm) & 3;
    const int sg = __popcll(x & zm) & 1;
    double2 ph = ny == 0 ? make_double2(1, 0) : ny == 1 ? make_double2(0, 1) : ny == 2 ? make_double2(-1, 0) : make_double2(0, -1);
    if (sg) ph = make_double2(-ph.x, -ph.y);
    return ph;
}

// energies[i] += sum over instance i's amplitudes and terms.  The loop is
// uniform per warp (every lane runs the same iterations; lanes past the end
// contribute nothing), so the warp shuffles always see all 32 lanes.
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_energy(const typename A::Amp *__restrict__ psi, const uint64_t *__restrict__ amp0, const uint64_t *offs,
               const int *__restrict__ tbeg, const BTerm *__restrict__ terms, int ninst, uint64_t total,
               double *energies) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t wb = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); wb < total; wb += stride) {
        const uint64_t w = wb + lane;
        const bool act = w < total;
        int lo = -1;
        typename A::Acc acc = 0;
        if (act) {
            int l = 0, hi = ninst - 1;
            while (l < hi) {
                const int mid = (l + hi + 1) >> 1;
                if (amp0[mid] <= w) l = mid;
                else hi = mid - 1;
            }
            lo = l;
            const uint64_t x = w - amp0[lo];
            const typename A::Amp px = psi[offs[lo] + x];
            for (int t = tbeg[lo]; t < tbeg[lo + 1]; t++) {
                const BTerm T = terms[t];
                acc += A::term(psi[offs[lo] + (x ^ T.xm)], px, pauli_phase(x, T.xm, T.zm), T.c);
            }
        }
        double v = double(acc);
        const unsigned full = 0xffffffffu;
        const int first = __shfl_sync(full, lo, 0);
        if (__all_sync(full, !act || lo == first)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(full, v, o);
            if (lane == 0) atomicAdd(energies + first, v);
        } else if (act) {
            atomicAdd(energies + lo, v);
        }
    }
}

// lambda = H psi per instance
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_hpsi(const typename A::Amp *__restrict__ psi, typename A::Amp *__restrict__ lam,
             const uint64_t *__restrict__ amp0, const uint64_t *offs, const int *__restrict__ tbeg,
             const BTerm *__restrict__ terms, int ninst, uint64_t total) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total; w += stride) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (amp0[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t y = w - amp0[lo];
        typename A::V acc = A::zero();
        for (int t = tbeg[lo]; t < tbeg[lo + 1]; t++) {
            const BTerm T = terms[t];
            const uint64_t x = y ^ T.xm;
            const double2 ph = pauli_phase(x, T.xm, T.zm);
            acc = A::add(acc, A::scale(A::in(psi[offs[lo] + x]), make_double2(T.c * ph.x, T.c * ph.y)));
        }
        lam[offs[lo] + y] = A::out(acc);
    }
}

// backward step: Im<lam|P|psi> for rotations, then psi, lam <- U^dag
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_back(typename A::Amp *__restrict__ psi, typename A::Amp *__restrict__ lam,
             const BEntry *__restrict__ entries, int count, uint64_t total, const double2 *__restrict__ mats,
             double *grads) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t wb = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); wb < total; wb += stride) {
        const uint64_t w = wb + lane;
        const bool act = w < total;
        const int ei = act ? find_entry(entries, count, w) : -1;
        double g = 0.0;
        bool rot = false;
        if (act) {
        const BEntry e = entries[ei];
        rot = e.kind != BK_FIXED;
        uint64_t a[4];
        slice_addr<A>(e, w - e.work0, a);
        typename A::V v[4], l[4];
        const int d = 1 << e.k;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d) {
                v[j] = A::in(psi[a[j]]);
                l[j] = A::in(lam[a[j]]);
            }
        if (e.kind != BK_FIXED) {  // 1-qubit rotation: <lam|P|psi> on the slice
            double2 s;
            if (e.kind == BK_RX) {
                const double2 t0 = A::cdot(l[0], v[1]), t1 = A::cdot(l[1], v[0]);
                s = make_double2(t0.x + t1.x, t0.y + t1.y);
            } else if (e.kind == BK_RY) {  // Y|0> = i|1>, Y|1> = -i|0>
                const double2 t0 = A::cdot(l[0], v[1]), t1 = A::cdot(l[1], v[0]);
                s = make_double2(t0.y - t1.y, -t0.x + t1.x);  // -i t0 + i t1
            } else {
                const double2 t0 = A::cdot(l[0], v[0]), t1 = A::cdot(l[1], v[1]);
                s = make_double2(t0.x - t1.x, t0.y - t1.y);
            }
            g = s.y;
        }
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, true, v);
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, true, l);
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d) {
                psi[a[j]] = A::out(v[j]);
                lam[a[j]] = A::out(l[j]);
            }
        }
        // the warp's lanes usually share an entry: one atomic per warp then
        const unsigned full = 0xffffffffu;
        const int first = __shfl_sync(full, ei, 0);
        if (__all_sync(full, !act || ei == first)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(full, g, o);
            if (lane == 0 && rot) atomicAdd(grads + entries[first].param, g);
        } else if (act && rot) {
            atomicAdd(grads + entries[ei].param, g);
        }
    }
}

}  // namespace
}  // namespace cast

// ------------------------------------------------------------------ host
struct cast_batch {
    int ninst = 0;
    cast_dtype dt = CAST_C64;
    bool grad = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nparams = 0;
    uint64_t total_amps = 0;   // amplitudes of all instances (no padding)
    uint64_t arena_amps = 0;   // including padding
    std::vector<uint64_t> offs, amp0;
    std::vector<int> nq, tbeg;
    std::vector<cast::BTerm> terms;
    std::vector<cast::BEntry> entries;   // all steps, in step order
    std::vector<int> step_begin;         // entries of step s: [step_begin[s], step_begin[s+1])
    std::vector<uint64_t> step_work;
    int nmat = 0;
    std::vector<double2> fixed_mats;  // 16 per slot (rotation slots filled on the device)
    // device
    void *psi = nullptr, *lam = nullptr;
    cast::BEntry *d_entries = nullptr;
    cast::BTerm *d_terms = nullptr;
    uint64_t *d_offs = nullptr, *d_amp0 = nullptr;
    int *d_nq = nullptr, *d_tbeg = nullptr;
    double2 *d_mats = nullptr;
    double *d_params = nullptr, *d_energy = nullptr, *d_grads = nullptr;
    cudaGraphExec_t g_energy = nullptr, g_grad = nullptr;
};

namespace cast {
namespace {

int grid_of(uint64_t work) {
    const uint64_t cap = uint64_t(sm_count_cached()) * 8, need = (work + kBThreads - 1) / kBThreads;
    return int(std::max<uint64_t>(1, std::min(cap, need)));
}

template <class A>
void queue_forward(cast_batch *b) {
    using Amp = typename A::Amp;
    const int S = int(b->step_work.size());
    cudaMemsetAsync(b->psi, 0, b->arena_amps * sizeof(Amp), b->stream);
    k_batch_set_zero_state<<<(b->ninst + 127) / 128, 128, 0, b->stream>>>(b->psi, int(sizeof(Amp)), b->d_offs, b->ninst);
    const int ne = int(b->entries.size());
    if (ne > 0) k_batch_prep<<<(ne + 127) / 128, 128, 0, b->stream>>>(b->d_entries, ne, b->d_params, b->d_mats);
    for (int s = 0; s < S; s++) {
        const int e0 = b->step_begin[s], cnt = b->step_begin[s + 1] - e0;
        k_batch_gate<A><<<grid_of(b->step_work[s]), kBThreads, 0, b->stream>>>(
            reinterpret_cast<Amp *>(b->psi), b->d_entries + e0, cnt, b->step_work[s], b->d_mats);
    }
    cudaMemsetAsync(b->d_energy, 0, sizeof(double) * b->ninst, b->stream);
    k_batch_energy<A><<<grid_of(b->total_amps), kBThreads, 0, b->stream>>>(
        reinterpret_cast<const Amp *>(b->psi), b->d_amp0, b->d_offs, b->d_tbeg, b->d_terms, b->ninst,
        b->total_amps, b->d_energy);
}

template <class A>
void queue_backward(cast_batch *b) {
    using Amp = typename A::Amp;
    const int S = int(b->step_work.size());
    k_batch_hpsi<A><<<grid_of(b->total_amps), kBThreads, 0, b->stream>>>(
        reinterpret_cast<const Amp *>(b->psi), reinterpret_cast<Amp *>(b->lam), b->d_amp0, b->d_offs, b->d_tbeg,
        b->d_terms, b->ninst, b->total_amps);
    cudaMemsetAsync(b->d_grads, 0, sizeof(double) * std::max(1, b->nparams), b->stream);
    for (int s = S - 1; s >= 0; s--) {
        const int e0 = b->step_begin[s], cnt = b->step_begin[s + 1] - e0;
        k_batch_back<A><<<grid_of(b->step_work[s]), kBThreads, 0, b->stream>>>(
            reinterpret_cast<Amp *>(b->psi), reinterpret_cast<Amp *>(b->lam), b->d_entries + e0, cnt,
            b->step_work[s], b->d_mats, b->d_grads);
    }
}

// captured on a private stream (the caller's may be the legacy default
// stream, which cannot be captured), replayed on the batch's stream
cast_status build_graph(cast_batch *b, bool grad, cudaGraphExec_t *out) {
    cudaStream_t cap = nullptr, orig = b->stream;
    CAST_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    b->stream = cap;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (b->dt == CAST_C64) {
            queue_forward<BA64>(b);
            if (grad) queue_backward<BA64>(b);
        } else {
            queue_forward<BA128>(b);
            if (grad) queue_backward<BA128>(b);
        }
        e = cudaStreamEndCapture(cap, &g);
    }
    b->stream = orig;
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture (batch)");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
    return CAST_OK;
}

void free_batch(cast_batch *b) {
    if (b->g_energy) cudaGraphExecDestroy(b->g_energy);
    if (b->g_grad) cudaGraphExecDestroy(b->g_grad);
    void *ptrs[] = {b->psi, b->lam, b->d_entries, b->d_terms, b->d_offs, b->d_amp0, b->d_nq, b->d_tbeg,
                    b->d_mats, b->d_params, b->d_energy, b->d_grads};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

cast_status run(cast_batch *b, const double *params, double *energies, double *grads, bool grad) {
    if (!b) return fail(CAST_ERR_ARG, "null batch");
    if (b->nparams > 0 && !params) return fail(CAST_ERR_ARG, "null parameters");
    if (!energies || (grad && b->nparams > 0 && !grads)) return fail(CAST_ERR_ARG, "null outputs");
    if (grad && !b->grad) return fail(CAST_ERR_ARG, "batch created without gradient buffers");
    for (int p = 0; p < b->nparams; p++)
        if (!std::isfinite(params[p])) return fail(CAST_ERR_ARG, "non-finite parameter");
    int dev = -1;
    CAST_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) return fail(CAST_ERR_ARG, "make the batch's device current before this call");
    cudaGraphExec_t *ge = grad ? &b->g_grad : &b->g_energy;
    if (!*ge) {
        cast_status st = build_graph(b, grad, ge);
        if (st != CAST_OK) return st;
    }
    if (b->nparams > 0)
        CAST_CUDA(cudaMemcpyAsync(b->d_params, params, sizeof(double) * b->nparams, cudaMemcpyHostToDevice, b->stream));
    CAST_CUDA(cudaGraphLaunch(*ge, b->stream));
    CAST_CUDA(cudaMemcpyAsync(energies, b->d_energy, sizeof(double) * b->ninst, cudaMemcpyDeviceToHost, b->stream));
    if (grad && b->nparams > 0)
        CAST_CUDA(cudaMemcpyAsync(grads, b->d_grads, sizeof(double) * b->nparams, cudaMemcpyDeviceToHost, b->stream));
    CAST_CUDA(cudaStreamSynchronize(b->stream));
    return take_device_error();
}

}  // namespace
}  // namespace cast

using namespace cast;

extern "C" {

cast_status cast_batch_create(int n_instances, const cast_circuit *circuits, const int32_t *param_offsets,
                              const cast_pauli_sum *hams, cast_dtype dt, int with_grad, void *cuda_stream,
                              cast_batch **out) {
    if (!out) return fail(CAST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (n_instances < 1 || !circuits || !hams) return fail(CAST_ERR_ARG, "need at least one instance");
    if (dt != CAST_C64 && dt != CAST_C128) return fail(CAST_ERR_ARG, "unknown dtype");
    cast_batch *b = new cast_batch();
    b->ninst = n_instances;
    b->dt = dt;
    b->grad = with_grad != 0;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&b->device);
    uint64_t off = 0, a0 = 0;
    int maxg = 0;
    std::vector<int> poff(n_instances, 0);
    for (int i = 0; i < n_instances; i++) {
        const cast_circuit &c = circuits[i];
        if (c.n_qubits < 1 || c.n_qubits > 30) {
            delete b;
            return fail(CAST_ERR_ARG, "instance qubit count must be 1..30");
        }
        if (c.n_gates < 0 || (c.n_gates > 0 && !c.gates) || c.n_params < 0) {
            delete b;
            return fail(CAST_ERR_ARG, "bad gate list");
        }
        for (int g = 0; g < c.n_gates; g++) {
            const cast_gate &gt = c.gates[g];
            if (gt.k > 2 && gt.k <= CAST_MAX_K) {
                delete b;
                return fail(CAST_ERR_UNSUPPORTED, "batched circuits take 1- and 2-qubit gates");
            }
            const bool ok = gt.k >= 1 && gt.k <= 2 && gt.qubits[0] >= 0 && gt.qubits[0] < c.n_qubits &&
                            (gt.k == 1 || (gt.qubits[1] >= 0 && gt.qubits[1] < c.n_qubits && gt.qubits[1] != gt.qubits[0])) &&
                            gt.param_index < c.n_params && (gt.kind == CAST_GATE_MATRIX ? gt.matrix != nullptr : gate_table_arity(gt.kind) == gt.k);
            if (!ok) {
                delete b;
                return fail(CAST_ERR_ARG, "instance " + std::to_string(i) + ", gate " + std::to_string(g) +
                                              ": 1- or 2-qubit gate with valid, distinct qubits and parameter index");
            }
        }
        cast_status st = check_pauli(&hams[i], c.n_qubits);
        if (st != CAST_OK) {
            delete b;
            return st;
        }
        poff[i] = param_offsets ? param_offsets[i] : b->nparams;
        if (poff[i] < 0) {
            delete b;
            return fail(CAST_ERR_ARG, "negative parameter offset");
        }
        b->nparams = std::max(b->nparams, poff[i] + c.n_params);
        b->offs.push_back(off);
        b->amp0.push_back(a0);
        b->nq.push_back(c.n_qubits);
        const uint64_t na = uint64_t(1) << c.n_qubits;
        a0 += na;
        off += (na + 255) & ~uint64_t(255);
        maxg = std::max(maxg, c.n_gates);
        b->tbeg.push_back(int(b->terms.size()));
        for (int t = 0; t < hams[i].n_terms; t++)
            b->terms.push_back({hams[i].coeffs[t], hams[i].x_masks[t], hams[i].z_masks[t]});
    }
    b->tbeg.push_back(int(b->terms.size()));
    b->amp0.push_back(a0);
    b->total_amps = a0;
    b->arena_amps = off;
    // gate steps
    b->step_begin.push_back(0);
    for (int s = 0; s < maxg; s++) {
        uint64_t work = 0;
        for (int i = 0; i < n_instances; i++) {
            const cast_circuit &c = circuits[i];
            if (s >= c.n_gates) continue;
            const cast_gate &g = c.gates[s];
            if (g.k > 2) {
                delete b;
                return fail(CAST_ERR_UNSUPPORTED, "batched circuits take 1- and 2-qubit gates");
            }
            BEntry e{};
            e.work0 = work;
            e.off = b->offs[i];
            e.inst = i;
            e.k = g.k;
            e.q0 = g.qubits[0];
            e.q1 = g.k == 2 ? g.qubits[1] : 0;
            e.mat = b->nmat++;
            e.param = -1;
            e.kind = BK_FIXED;
            std::vector<double2> slot(16, make_double2(0.0, 0.0));
            if (g.param_index >= 0) {
                if (g.kind == CAST_GATE_RX) e.kind = BK_RX;
                else if (g.kind == CAST_GATE_RY) e.kind = BK_RY;
                else if (g.kind == CAST_GATE_RZ) e.kind = BK_RZ;
                else {
                    delete b;
                    return fail(CAST_ERR_UNSUPPORTED, "batched circuits: only RX, RY, RZ may carry parameters");
                }
                e.param = poff[i] + g.param_index;
            } else {
                std::vector<cplx> m;
                cast_status st = gate_matrix_of(g, nullptr, 0, &m);
                if (st != CAST_OK) {
                    delete b;
                    return st;
                }
                for (size_t j = 0; j < m.size(); j++) slot[j] = make_double2(m[j].real(), m[j].imag());
            }
            b->fixed_mats.insert(b->fixed_mats.end(), slot.begin(), slot.end());
            b->entries.push_back(e);
            work += uint64_t(1) << (c.n_qubits - g.k);
        }
        b->step_begin.push_back(int(b->entries.size()));
        b->step_work.push_back(work);
    }
    // device buffers
    const size_t S = dt == CAST_C64 ? 8 : 16;
    auto alloc = [&](void **p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)); };
    cudaError_t e = alloc(&b->psi, b->arena_amps * S);
    if (e == cudaSuccess && b->grad) e = alloc(&b->lam, b->arena_amps * S);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_entries), b->entries.size() * sizeof(BEntry));
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_terms), b->terms.size() * sizeof(BTerm));
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_offs), b->offs.size() * 8);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_amp0), b->amp0.size() * 8);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_nq), b->nq.size() * 4);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_tbeg), b->tbeg.size() * 4);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_mats), size_t(b->nmat) * 16 * sizeof(double2));
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_params), size_t(b->nparams) * 8);
    if (e == cudaSuccess) e = alloc(reinterpret_cast<void **>(&b->d_energy), size_t(b->ninst) * 8);
    if (e == cudaSuccess && b->grad) e = alloc(reinterpret_cast<void **>(&b->d_grads), size_t(b->nparams) * 8);
    auto up = [&](void *d, const void *h, size_t bytes) {
        return bytes ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    if (e == cudaSuccess) e = up(b->d_entries, b->entries.data(), b->entries.size() * sizeof(BEntry));
    if (e == cudaSuccess) e = up(b->d_terms, b->terms.data(), b->terms.size() * sizeof(BTerm));
    if (e == cudaSuccess) e = up(b->d_offs, b->offs.data(), b->offs.size() * 8);
    if (e == cudaSuccess) e = up(b->d_amp0, b->amp0.data(), b->amp0.size() * 8);
    if (e == cudaSuccess) e = up(b->d_nq, b->nq.data(), b->nq.size() * 4);
    if (e == cudaSuccess) e = up(b->d_tbeg, b->tbeg.data(), b->tbeg.size() * 4);
    if (e == cudaSuccess) e = up(b->d_mats, b->fixed_mats.data(), b->fixed_mats.size() * sizeof(double2));
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch buffers");
    }
    *out = b;
    return CAST_OK;
}

cast_status cast_batch_energy(cast_batch *b, const double *params, double *energies) {
    return run(b, params, energies, nullptr, false);
}

cast_status cast_batch_grad(cast_batch *b, const double *params, double *energies, double *grads) {
    return run(b, params, energies, grads, true);
}

cast_status cast_batch_info(const cast_batch *b, int *n_params, int *n_steps) {
    if (!b) return fail(CAST_ERR_ARG, "null batch");
    if (n_params) *n_params = b->nparams;
    if (n_steps) *n_steps = int(b->step_work.size());
    return CAST_OK;
}

cast_status cast_batch_destroy(cast_batch *b) {
    if (!b) return CAST_OK;
    free_batch(b);
    return CAST_OK;
}

}  // extern "C"
