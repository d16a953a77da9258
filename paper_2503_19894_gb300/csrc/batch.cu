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
// matrix slot, parameter); each CTA takes a contiguous range of work items,
// so a thread finds its entry once and then steps forward.
// Rotation matrices are formed on the device from the parameters at the start
// of every replay, so the whole launch sequence (initial states, gate steps,
// energies; for gradients also lambda = H psi and the backward sweep) is
// captured once into a CUDA graph and replayed per parameter set.
//
// Energies: one pass over every instance's amplitudes, each thread summing
// c_t Re(conj(psi[x ^ xm_t]) i^q psi[x]) over its instance's terms (the Pauli
// phase as a quarter-turn count q); warps add into the instance's FP64 slot.
// Gradients: lambda = H psi, then steps in reverse; a step forms
// Im<lambda|P_q|psi> for every rotation in it (the derivative of
// exp(-i theta P / 2)) and un-applies each gate from psi and lambda in the same
// pass; a thread's share for one parameter is summed in the state's
// arithmetic and added to the parameter's FP64 slot once.
//
// complex64 runs in FP32 (energy terms summed per thread in FP32, then FP64);
// complex128 in double-float arithmetic on the FP32 pipe (df64.cuh), the
// arena holding FP64 amplitudes, energies in FP64.  Matrices are converted to
// the arithmetic's format once per call, so no FP64 instruction runs per gate
// application.
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
    int32_t skip;    // bit j: member j has an identity row and column (not loaded or stored)
};

struct BTerm {
    double c;
    uint64_t xm, zm;
    float ch, cl;  // c as a double-float pair (ch alone for complex64)
};

// Work distribution: CTA b takes the contiguous range [b c, b c + c) of the
// work items (c a multiple of 32, so every warp's lanes run the same
// iterations); a thread finds its first entry by binary search and then only
// steps forward, since its items increase and entries are contiguous ranges.
__device__ __forceinline__ void cta_range(uint64_t total, uint64_t &beg, uint64_t &end) {
    const uint64_t c = ((total + gridDim.x - 1) / gridDim.x + 31) & ~uint64_t(31);
    beg = uint64_t(blockIdx.x) * c;
    end = beg + c < total ? beg + c : total;
}

template <class F>
__device__ __forceinline__ int advance(int cur, uint64_t w, int count, F first_of) {
    if (cur < 0) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first_of(mid) <= w) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }
    while (cur + 1 < count && first_of(cur + 1) <= w) cur++;
    return cur;
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
    using M = float2;  // matrix entry in the arithmetic's format
    __device__ static M mat(double2 u) { return make_float2(float(u.x), float(u.y)); }
    __device__ static V mulm(M u, V x) { return make_float2(u.x * x.x - u.y * x.y, u.x * x.y + u.y * x.x); }
    __device__ static M conjm(M u) { return make_float2(u.x, -u.y); }
    __device__ static bool nonzero(M u) { return u.x != 0.f || u.y != 0.f; }
    __device__ static V add(V a, V b) { return make_float2(a.x + b.x, a.y + b.y); }
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    // energies: c Re(i^q conj(a) b) summed per thread in FP32, then once to FP64
    using Acc = float;
    __device__ static float term(Amp a, Amp b, int q, const BTerm &T) {
        const float dr = a.x * b.x + a.y * b.y, di = a.x * b.y - a.y * b.x;
        const float re = q == 0 ? dr : q == 1 ? -di : q == 2 ? -dr : di;
        return T.ch * re;
    }
    // acc += c i^q x
    __device__ static void add_scaled(V &acc, V x, int q, const BTerm &T) {
        const V r = q == 0 ? x : q == 1 ? make_float2(-x.y, x.x) : q == 2 ? make_float2(-x.x, -x.y) : make_float2(x.y, -x.x);
        acc.x = fmaf(T.ch, r.x, acc.x);
        acc.y = fmaf(T.ch, r.y, acc.y);
    }
    // gradient sums: Re and Im of conj(a) b
    using G = float;
    __device__ static void gzero(G &g) { g = 0.f; }
    __device__ static void gadd(G &g, float sgn, V a, V b, bool imag) {
        g += sgn * (imag ? (a.x * b.y - a.y * b.x) : (a.x * b.x + a.y * b.y));
    }
    __device__ static double gval(const G &g) { return double(g); }
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
    using M = float4;  // (re hi, re lo, im hi, im lo)
    __device__ static M mat(double2 u) {
        const V c = cf(u);
        return make_float4(c.rh, c.rl, c.ih, c.il);
    }
    __device__ static V mulm(M u, V x) {
        V acc = {0.f, 0.f, 0.f, 0.f};
        const V uc = {u.x, u.y, u.z, u.w};
        df::cmac(acc, uc, x);
        return acc;
    }
    __device__ static M conjm(M u) { return make_float4(u.x, u.y, -u.z, -u.w); }
    __device__ static bool nonzero(M u) { return u.x != 0.f || u.z != 0.f; }
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
    // energies in FP64 on the stored amplitudes (the reductions of the method
    // stay FP64; one pass per call)
    using Acc = double;
    __device__ static double term(Amp a, Amp b, int q, const BTerm &T) {
        const double dr = a.x * b.x + a.y * b.y, di = a.x * b.y - a.y * b.x;
        const double re = q == 0 ? dr : q == 1 ? -di : q == 2 ? -dr : di;
        return T.c * re;
    }
    // acc += c i^q x, in double-float
    __device__ static void add_scaled(V &acc, V x, int q, const BTerm &T) {
        const V r = q == 0 ? x : q == 1 ? V{-x.ih, -x.il, x.rh, x.rl} : q == 2 ? V{-x.rh, -x.rl, -x.ih, -x.il}
                                                                        : V{x.ih, x.il, -x.rh, -x.rl};
        df::mac(acc.rh, acc.rl, T.ch, T.cl, r.rh, r.rl);
        df::mac(acc.ih, acc.il, T.ch, T.cl, r.ih, r.il);
    }
    // gradient sums in double-float: Re or Im of conj(a) b
    struct G {
        float h, l;
    };
    __device__ static void gzero(G &g) { g = {0.f, 0.f}; }
    __device__ static void gadd(G &g, float sgn, V a, V b, bool imag) {
        if (imag) {  // a.re b.im - a.im b.re
            df::mac(g.h, g.l, sgn * a.rh, sgn * a.rl, b.ih, b.il);
            df::msub(g.h, g.l, sgn * a.ih, sgn * a.il, b.rh, b.rl);
        } else {     // a.re b.re + a.im b.im
            df::mac(g.h, g.l, sgn * a.rh, sgn * a.rl, b.rh, b.rl);
            df::mac(g.h, g.l, sgn * a.ih, sgn * a.il, b.ih, b.il);
        }
    }
    __device__ static double gval(const G &g) { return double(g.h) + double(g.l); }
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

// u (row-major 2^k x 2^k, entries in the arithmetic's format) or its adjoint
// applied to slice amplitudes v
template <class A>
__device__ __forceinline__ void apply_small(const typename A::M *u, int k, bool adj, typename A::V (&v)[4]) {
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
            const typename A::M m = adj ? A::conjm(u[c * d + r]) : u[r * d + c];
            if (!A::nonzero(m)) continue;
            acc = A::add(acc, A::mulm(m, v[c]));
        }
        y[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
        if (r < d) v[r] = y[r];
}

// every slot's matrix in the arithmetic's format (once per replay, after the
// rotations were formed)
template <class A>
__global__ void k_batch_convert(const double2 *mats, typename A::M *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = A::mat(mats[i]);
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
             const typename A::M *__restrict__ mats) {
    uint64_t beg, end;
    cta_range(total, beg, end);
    int ei = -1;
    auto first_of = [&](int i) { return entries[i].work0; };
    for (uint64_t w = beg + threadIdx.x; w < end; w += blockDim.x) {
        ei = advance(ei, w, count, first_of);
        const BEntry e = entries[ei];
        uint64_t a[4];
        slice_addr<A>(e, w - e.work0, a);
        typename A::V v[4];
        const int d = 1 << e.k;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            v[j] = A::zero();
            if (j < d && !((e.skip >> j) & 1)) v[j] = A::in(psi[a[j]]);
        }
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, false, v);
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d && !((e.skip >> j) & 1)) psi[a[j]] = A::out(v[j]);
    }
}

// P|x> = i^q |x ^ xm> with q = popc(xm & zm) + 2 popc(x & zm) (mod 4)
__device__ __forceinline__ int pauli_quarter(uint64_t x, uint64_t xm, uint64_t zm) {
    return (__popcll(xm & zm) + 2 * (__popcll(x & zm) & 1)) & 3;
}

// energies[i] += sum over instance i's amplitudes and terms.  The loop is
// uniform per warp (every lane runs the same iterations; lanes past the end
// contribute nothing), so the warp shuffles always see all 32 lanes.
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_energy(const typename A::Amp *__restrict__ psi, const uint64_t *__restrict__ amp0, const uint64_t *offs,
               const int *__restrict__ tbeg, const BTerm *__restrict__ terms, int ninst, uint64_t total,
               double *energies) {
    uint64_t beg, end;
    cta_range(total, beg, end);
    const int lane = threadIdx.x & 31;
    int cur = -1;
    auto first_of = [&](int i) { return amp0[i]; };
    for (uint64_t wb = beg + (threadIdx.x & ~31u); wb < end; wb += blockDim.x) {
        const uint64_t w = wb + lane;
        const bool act = w < end;
        int lo = -1;
        typename A::Acc acc = 0;
        if (act) {
            cur = advance(cur, w, ninst, first_of);
            lo = cur;
            const uint64_t x = w - amp0[lo];
            const typename A::Amp px = psi[offs[lo] + x];
            for (int t = tbeg[lo]; t < tbeg[lo + 1]; t++) {
                const BTerm T = terms[t];
                acc += A::term(psi[offs[lo] + (x ^ T.xm)], px, pauli_quarter(x, T.xm, T.zm), T);
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
    uint64_t beg, end;
    cta_range(total, beg, end);
    int lo = -1;
    auto first_of = [&](int i) { return amp0[i]; };
    for (uint64_t w = beg + threadIdx.x; w < end; w += blockDim.x) {
        lo = advance(lo, w, ninst, first_of);
        const uint64_t y = w - amp0[lo];
        typename A::V acc = A::zero();
        for (int t = tbeg[lo]; t < tbeg[lo + 1]; t++) {
            const BTerm T = terms[t];
            const uint64_t x = y ^ T.xm;
            A::add_scaled(acc, A::in(psi[offs[lo] + x]), pauli_quarter(x, T.xm, T.zm), T);
        }
        lam[offs[lo] + y] = A::out(acc);
    }
}

// backward step: Im<lam|P|psi> for rotations, then psi, lam <- U^dag
template <class A>
__global__ void __launch_bounds__(kBThreads)
k_batch_back(typename A::Amp *__restrict__ psi, typename A::Amp *__restrict__ lam,
             const BEntry *__restrict__ entries, int count, uint64_t total, const typename A::M *__restrict__ mats,
             double *grads) {
    uint64_t beg, end;
    cta_range(total, beg, end);
    int cur = -1, gparam = -1;
    typename A::G g;
    A::gzero(g);
    auto first_of = [&](int i) { return entries[i].work0; };
    // a thread's items run through few entries: its gradient share of the
    // current entry is summed in the state's arithmetic and added to the
    // parameter's FP64 slot when the entry changes
    auto flush = [&]() {
        if (gparam >= 0) atomicAdd(grads + gparam, A::gval(g));
        A::gzero(g);
        gparam = -1;
    };
    for (uint64_t w = beg + threadIdx.x; w < end; w += blockDim.x) {
        const int prev = cur;
        cur = advance(cur, w, count, first_of);
        if (cur != prev) flush();
        const BEntry e = entries[cur];
        uint64_t a[4];
        slice_addr<A>(e, w - e.work0, a);
        typename A::V v[4], l[4];
        const int d = 1 << e.k;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            v[j] = l[j] = A::zero();
            if (j < d && !((e.skip >> j) & 1)) {
                v[j] = A::in(psi[a[j]]);
                l[j] = A::in(lam[a[j]]);
            }
        }
        if (e.kind != BK_FIXED) {  // 1-qubit rotation: Im<lam|P|psi> on the slice
            gparam = e.param;
            if (e.kind == BK_RX) {         // Im(conj(l0) v1 + conj(l1) v0)
                A::gadd(g, 1.f, l[0], v[1], true);
                A::gadd(g, 1.f, l[1], v[0], true);
            } else if (e.kind == BK_RY) {  // Y|0> = i|1>, Y|1> = -i|0>: -Re(conj(l0) v1) + Re(conj(l1) v0)
                A::gadd(g, -1.f, l[0], v[1], false);
                A::gadd(g, 1.f, l[1], v[0], false);
            } else {                       // Im(conj(l0) v0 - conj(l1) v1)
                A::gadd(g, 1.f, l[0], v[0], true);
                A::gadd(g, -1.f, l[1], v[1], true);
            }
        }
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, true, v);
        apply_small<A>(mats + size_t(e.mat) * 16, e.k, true, l);
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (j < d && !((e.skip >> j) & 1)) {
                psi[a[j]] = A::out(v[j]);
                lam[a[j]] = A::out(l[j]);
            }
    }
    flush();
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
    void *d_mats_a = nullptr;  // the same matrices in the arithmetic's format
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
    const int nm = b->nmat * 16;
    if (nm > 0)
        k_batch_convert<A><<<(nm + 255) / 256, 256, 0, b->stream>>>(b->d_mats, static_cast<typename A::M *>(b->d_mats_a), nm);
    const typename A::M *mats = static_cast<const typename A::M *>(b->d_mats_a);
    for (int s = 0; s < S; s++) {
        const int e0 = b->step_begin[s], cnt = b->step_begin[s + 1] - e0;
        k_batch_gate<A><<<grid_of(b->step_work[s]), kBThreads, 0, b->stream>>>(
            reinterpret_cast<Amp *>(b->psi), b->d_entries + e0, cnt, b->step_work[s], mats);
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
            b->step_work[s], static_cast<const typename A::M *>(b->d_mats_a), b->d_grads);
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
                    b->d_mats, b->d_mats_a, b->d_params, b->d_energy, b->d_grads};
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
        {
            const double c = hams[i].coeffs[t];
            const float ch = float(c);
            b->terms.push_back({c, hams[i].x_masks[t], hams[i].z_masks[t], ch, float(c - double(ch))});
        }
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
                // members whose row and column are those of the identity stay
                // in memory untouched (CZ: three of four; a rotation never)
                const int d = 1 << g.k;
                for (int j = 0; j < d; j++) {
                    bool id = m[size_t(j) * d + j] == cplx(1.0, 0.0);
                    for (int o = 0; o < d && id; o++)
                        if (o != j && (m[size_t(j) * d + o] != cplx(0.0, 0.0) || m[size_t(o) * d + j] != cplx(0.0, 0.0)))
                            id = false;
                    if (id) e.skip |= 1 << j;
                }
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
    if (e == cudaSuccess) e = alloc(&b->d_mats_a, size_t(b->nmat) * 16 * 16);  // float4 covers both formats
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
