// Sparsity-specialised gate kernels (Section V-A's sparse kernel generation,
// restated for GB300): a fused k-qubit gate (k = 3..7) is applied through a
// per-row list of its non-zero entries, each tagged with its kind, so that
// the work per slice follows the gate's operation count (Section IV-C)
// instead of 4^k complex products:
//   general complex u = a + ib      4 multiply-adds
//   real (b = 0) / imaginary (a = 0) 2 multiply-adds
//   +1, -1, +i, -i                   2 additions, no multiply
//   zero                             nothing (not in the list)
// The paper generates one kernel per matrix; here one kernel per (k, state
// type) reads the list at run time.  Its kind tests are uniform across a warp
// (every thread walks the same row), so they cost a branch, not divergence.
//
// Memory: a CTA takes super-tiles of 2^(12-k) consecutive slices x 2^k
// members (Eq. 4), 4096 amplitudes for every k: the addresses whose bits at
// the 12 - k lowest non-target positions and at the targets vary.  Enumerated
// in ascending address order they form runs of at least 32 contiguous
// amplitudes, so the gather and the scatter are coalesced for every target
// placement.  The super-tile sits in shared memory as X[g][member][lane]
// (slice row = 32 g + lane, row stride 33 elements); warp w computes rows
// w, w + 8, ... of every slice its lane owns, writes them back over X once
// every warp has read its inputs, and the super-tile is stored in address
// order.
//
// complex128 runs in double-float arithmetic (df64.cuh) like the dense
// complex128 kernels; complex64 in FP32.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "df64.cuh"
#include "internal.h"

namespace cast {
namespace {

enum EntryKind : uint32_t { E_GEN = 0, E_RE = 1, E_IM = 2, E_P1 = 3, E_M1 = 4, E_PI = 5, E_MI = 6 };

constexpr int kSpThreads = 256, kSpWarps = kSpThreads / 32, kSP = 33;  // slice-row stride of X, padded
// The address and shared-memory slot of a thread's element u are this
// thread's part (cube bits 0..7) plus u's part (bits 8..11, the same for every
// thread), taken from a 16-entry table built once per CTA instead of being
// assembled bit by bit at each of the three uses.  Measured per 30-qubit
// complex128 gate at 6-20% density: 13.4-15.8 ms against 14.7-17.2 ms.
constexpr bool kSpUTable = true;

// ------------------------------------------------------------ arithmetic
// apply<G>: y[g] += u * x[g] for G slices at once (one entry decode serves
// all of them); x[g] = xs[g * gs].
struct C64 {
    using Amp = float2;  // in HBM
    using X = float2;    // in shared memory
    using Acc = float2;
    using Val = float2;
    __device__ static X in(Amp a) { return a; }
    __device__ static Amp out(X x) { return x; }
    __device__ static void zero(Acc &a) { a = make_float2(0.f, 0.f); }
    __device__ static void merge(Acc &a, const Acc &b) { a.x += b.x; a.y += b.y; }
    template <int G>
    __device__ static void apply(Acc (&y)[G], uint32_t kind, const Val u, const X *xs, int gs) {
        switch (kind) {
            case E_GEN: {
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const X x = xs[g * gs];
                    y[g].x = fmaf(u.x, x.x, y[g].x);
                    y[g].x = fmaf(-u.y, x.y, y[g].x);
                    y[g].y = fmaf(u.x, x.y, y[g].y);
                    y[g].y = fmaf(u.y, x.x, y[g].y);
                }
                break;
            }
            case E_RE: {
                const float a = u.x;
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const X x = xs[g * gs];
                    y[g].x = fmaf(a, x.x, y[g].x);
                    y[g].y = fmaf(a, x.y, y[g].y);
                }
                break;
            }
            case E_IM: {
                const float b = u.y;
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const X x = xs[g * gs];
                    y[g].x = fmaf(-b, x.y, y[g].x);
                    y[g].y = fmaf(b, x.x, y[g].y);
                }
                break;
            }
            case E_P1:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; y[g].x += x.x; y[g].y += x.y; }
                break;
            case E_M1:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; y[g].x -= x.x; y[g].y -= x.y; }
                break;
            case E_PI:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; y[g].x -= x.y; y[g].y += x.x; }
                break;
            default:  // E_MI
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; y[g].x += x.y; y[g].y -= x.x; }
                break;
        }
    }
};

struct C128 {
    using Amp = double2;
    using X = df::CF;
    using Acc = df::CF;
    using Val = float4;  // (re hi, re lo, im hi, im lo)
    __device__ static X in(Amp a) { return df::split_c(a); }
    __device__ static Amp out(X x) { return df::join_c(x); }
    __device__ static void zero(Acc &a) { a = {0.f, 0.f, 0.f, 0.f}; }
    // (sh, sl) += (xh, xl), TwoSum on the heads
    __device__ static void add(float &sh, float &sl, float xh, float xl) {
        const float s = sh + xh;
        const float bb = s - sh;
        const float t = (sh - (s - bb)) + (xh - bb);
        sh = s;
        sl += t + xl;
    }
    __device__ static void merge(Acc &a, const Acc &b) {
        add(a.rh, a.rl, b.rh, b.rl);
        add(a.ih, a.il, b.ih, b.il);
    }
    template <int G>
    __device__ static void apply(Acc (&y)[G], uint32_t kind, const Val u, const X *xs, int gs) {
        switch (kind) {
            case E_GEN: {
                const df::CF uc = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int g = 0; g < G; g++) df::cmac(y[g], uc, xs[g * gs]);
                break;
            }
            case E_RE: {
                const float2 a = make_float2(u.x, u.y);
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const X x = xs[g * gs];
                    df::mac(y[g].rh, y[g].rl, a.x, a.y, x.rh, x.rl);
                    df::mac(y[g].ih, y[g].il, a.x, a.y, x.ih, x.il);
                }
                break;
            }
            case E_IM: {
                const float2 b = make_float2(u.z, u.w);
#pragma unroll
                for (int g = 0; g < G; g++) {
                    const X x = xs[g * gs];
                    df::msub(y[g].rh, y[g].rl, b.x, b.y, x.ih, x.il);
                    df::mac(y[g].ih, y[g].il, b.x, b.y, x.rh, x.rl);
                }
                break;
            }
            case E_P1:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; add(y[g].rh, y[g].rl, x.rh, x.rl); add(y[g].ih, y[g].il, x.ih, x.il); }
                break;
            case E_M1:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; add(y[g].rh, y[g].rl, -x.rh, -x.rl); add(y[g].ih, y[g].il, -x.ih, -x.il); }
                break;
            case E_PI:
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; add(y[g].rh, y[g].rl, -x.ih, -x.il); add(y[g].ih, y[g].il, x.rh, x.rl); }
                break;
            default:  // E_MI
#pragma unroll
                for (int g = 0; g < G; g++) { const X x = xs[g * gs]; add(y[g].rh, y[g].rl, x.ih, x.il); add(y[g].ih, y[g].il, -x.rh, -x.rl); }
                break;
        }
    }
};

// ---------------------------------------------------------------- kernel
// A CTA iteration takes a super-tile of G = 2^(7-k) tiles (32 G consecutive
// slices x 2^k members = 4096 amplitudes for every k): its 12 cube bits are
// the 5 + log2 G lowest non-target positions and the k targets.  Each thread
// moves 16 amplitudes per iteration; each entry of a row is decoded once and
// applied to the G slices a lane owns.  For G < 4 a row's entries alternate
// between 4 / G accumulator sets, so every thread keeps four independent
// dependency chains; an entry's code and value are loaded together, ahead of
// the kind test that consumes them.
template <int K> struct SpShape {
    static constexpr int D = 1 << K, G = 1 << (7 - K), E = 4096, PER = E / kSpThreads;
    static constexpr int RPW = D / kSpWarps;  // rows per warp
    static constexpr int NCH = G >= 4 ? 1 : 4 / G;  // independent chains per row
};

template <class A, int K>
__global__ void __launch_bounds__(kSpThreads)
k_sparse(typename A::Amp *__restrict__ sv, uint64_t nsuper, const __grid_constant__ Targets tg,
         const __grid_constant__ SpTile lay, const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ code,
         const typename A::Val *__restrict__ val) {
    using X = typename A::X;
    using S = SpShape<K>;
    constexpr int D = S::D, G = S::G, PER = S::PER, NCH = S::NCH, GS = D * kSP;
    static_assert(K >= 3 && K <= 7, "sparse kernel covers k = 3..7");
    extern __shared__ __align__(16) unsigned char sp_smem[];
    X *Xs = reinterpret_cast<X *>(sp_smem);  // [G][D][kSP]: slice row = g * 32 + lane
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // this thread's elements e = tid + 256 u (u < 16); the cube bits of tid
    // (positions 0..7) and of u (positions 8..11) are additive
    uint64_t a_lo = 0;
    uint32_t s_lo = 0, j_lo = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        if (!((tid >> b) & 1)) continue;
        a_lo += uint64_t(1) << lay.pos[b];
        const int r = lay.role[b];
        if (r < 16) s_lo |= 1u << r;
        else j_lo |= 1u << (r - 16);
    }
    // shared-memory slot of slice row s (g = s >> 5) and member j; linear in
    // (s, j) for disjoint bits, so the two parts' slots add
    auto slot = [](uint32_t s, uint32_t j) { return ((s >> 5) * D + j) * kSP + (s & 31); };
    __shared__ uint4 sU[PER];  // u's part: address (lo, hi), slot
    if constexpr (kSpUTable) {
        if (tid < PER) {
            uint64_t a = 0;
            uint32_t s = 0, j = 0;
            for (int b = 8; b < 12; b++) {
                if (!((tid >> (b - 8)) & 1)) continue;
                a += uint64_t(1) << lay.pos[b];
                const int r = lay.role[b];
                if (r < 16) s |= 1u << r;
                else j |= 1u << (r - 16);
            }
            sU[tid] = make_uint4(uint32_t(a), uint32_t(a >> 32), slot(s, j), 0u);
        }
        __syncthreads();
    }
    const uint32_t sl_lo = slot(s_lo, j_lo);
    auto elem = [&](int u, uint64_t &a, uint32_t &sl) {
        if constexpr (kSpUTable) {
            const uint4 t = sU[u];
            a = a_lo + (uint64_t(t.y) << 32 | t.x);
            sl = sl_lo + t.z;
            return;
        }
        a = a_lo;
        uint32_t s = s_lo, j = j_lo;
#pragma unroll
        for (int b = 8; b < 12; b++) {
            if (!((u >> (b - 8)) & 1)) continue;
            a += uint64_t(1) << lay.pos[b];
            const int r = lay.role[b];
            if (r < 16) s |= 1u << r;
            else j |= 1u << (r - 16);
        }
        sl = slot(s, j);
    };

    for (uint64_t st = blockIdx.x; st < nsuper; st += gridDim.x) {
        const uint64_t base = slice_base<K>(st * (32 * G), tg);
        // gather: coalesced loads in address order, all issued before the stores
        typename A::Amp v[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            uint64_t a;
            uint32_t sl;
            elem(u, a, sl);
            v[u] = __ldcs(sv + base + a);
        }
#pragma unroll
        for (int u = 0; u < PER; u++) {
            uint64_t a;
            uint32_t sl;
            elem(u, a, sl);
            Xs[sl] = A::in(v[u]);
        }
        __syncthreads();
        // rows r = warp + 8 i, for the G slices of this lane, entry by entry
        typename A::Acc y[S::RPW][G];
#pragma unroll
        for (int i = 0; i < S::RPW; i++) {
            const int r = warp + kSpWarps * i;
            typename A::Acc acc[NCH][G];
#pragma unroll
            for (int h = 0; h < NCH; h++)
#pragma unroll
                for (int g = 0; g < G; g++) A::zero(acc[h][g]);
            const uint32_t e0 = __ldg(row_ptr + r), e1 = __ldg(row_ptr + r + 1);
            uint32_t e = e0;
            if constexpr (NCH > 1) {
                for (; e + NCH <= e1; e += NCH) {
                    uint32_t c[NCH];
                    typename A::Val u[NCH];
#pragma unroll
                    for (int h = 0; h < NCH; h++) {
                        c[h] = __ldg(code + e + h);
                        u[h] = __ldg(val + e + h);
                    }
#pragma unroll
                    for (int h = 0; h < NCH; h++)
                        A::template apply<G>(acc[h], c[h] >> 8, u[h], Xs + (c[h] & 0xFFu) * kSP + lane, GS);
                }
            }
            for (; e < e1; e++) {
                const uint32_t c = __ldg(code + e);
                const typename A::Val u = __ldg(val + e);
                A::template apply<G>(acc[0], c >> 8, u, Xs + (c & 0xFFu) * kSP + lane, GS);
            }
#pragma unroll
            for (int g = 0; g < G; g++) {
#pragma unroll
                for (int h = 1; h < NCH; h++) A::merge(acc[0][g], acc[h][g]);
                y[i][g] = acc[0][g];
            }
        }
        __syncthreads();  // every warp has read its inputs
#pragma unroll
        for (int i = 0; i < S::RPW; i++)
#pragma unroll
            for (int g = 0; g < G; g++) Xs[(g * D + warp + kSpWarps * i) * kSP + lane] = y[i][g];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; u++) {
            uint64_t a;
            uint32_t sl;
            elem(u, a, sl);
            __stcs(sv + base + a, A::out(Xs[sl]));
        }
        __syncthreads();  // the outputs are read before the next gather overwrites them
    }
}

// ------------------------------------------------------------- host side
// Entries within this distance of 1, -1, i or -i are taken as exactly that
// value (the paper's one tolerance), applied after the zero tolerance.
constexpr double kOneTol = 1e-14;

uint32_t entry_kind(cplx u) {
    auto near = [](cplx a, cplx b) { return std::abs(a.real() - b.real()) <= kOneTol && std::abs(a.imag() - b.imag()) <= kOneTol; };
    if (near(u, cplx(1, 0))) return E_P1;
    if (near(u, cplx(-1, 0))) return E_M1;
    if (near(u, cplx(0, 1))) return E_PI;
    if (near(u, cplx(0, -1))) return E_MI;
    if (u.imag() == 0.0) return E_RE;
    if (u.real() == 0.0) return E_IM;
    return E_GEN;
}

template <class A, int K>
cast_status run_sparse(cast_sv *sv, const PreparedGate &g) {
    using Val = typename A::Val;
    constexpr int D = 1 << K;
    // entry list: row_ptr[D + 1], code[nnz], val[nnz], each 16-byte aligned
    std::vector<uint32_t> rp(D + 1, 0), code;
    std::vector<Val> val;
    int64_t gen = 0;
    for (int r = 0; r < D; r++) {
        for (int c = 0; c < D; c++) {
            const cplx u = g.m[size_t(r) * D + c];
            if (u == cplx(0.0, 0.0)) continue;
            const uint32_t kind = entry_kind(u);
            code.push_back(uint32_t(c) | (kind << 8));
            Val v;
            if constexpr (sizeof(Val) == 8) {
                v.x = (float)u.real();
                v.y = (float)u.imag();
            } else {
                const float rh = (float)u.real(), ih = (float)u.imag();
                v = make_float4(rh, (float)(u.real() - (double)rh), ih, (float)(u.imag() - (double)ih));
            }
            val.push_back(v);
            gen += kind == E_GEN;
        }
        rp[r + 1] = (uint32_t)code.size();
    }
    const size_t nnz = code.size();
    auto up16 = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t o_code = up16(rp.size() * 4), o_val = o_code + up16(nnz * 4), bytes = o_val + nnz * sizeof(Val);
    std::vector<unsigned char> buf(bytes > 0 ? bytes : 16, 0);
    std::memcpy(buf.data(), rp.data(), rp.size() * 4);
    if (nnz) {
        std::memcpy(buf.data() + o_code, code.data(), nnz * 4);
        std::memcpy(buf.data() + o_val, val.data(), nnz * sizeof(Val));
    }
    const void *dev = nullptr;
    cast_status st = upload_matrix(sv, buf.data(), buf.size(), &dev);
    if (st != CAST_OK) return st;
    const unsigned char *d = static_cast<const unsigned char *>(dev);
    Targets tg;
    for (int i = 0; i < CAST_MAX_K; i++) tg.q[i] = i < K ? g.q[i] : 0;
    const SpTile lay = make_tile_layout(g.q, K);
    const uint64_t ntiles = uint64_t(1) << (sv->n - 12);  // super-tiles of 4096 amplitudes
    const size_t smem = sizeof(typename A::X) * (4096 / 32) * kSP;
    CAST_CUDA(cudaFuncSetAttribute(k_sparse<A, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CAST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse<A, K>, kSpThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const uint64_t cap = uint64_t(sm_count_cached()) * uint64_t(per_sm);
    const uint64_t grid = ntiles < cap ? ntiles : cap;
    const double N = double(uint64_t(1) << sv->n);
    // flops: 8 per general entry, 4 per real or imaginary one, per slice
    int64_t half = 0;
    for (size_t e = 0; e < nnz; e++) half += ((code[e] >> 8) == E_RE || (code[e] >> 8) == E_IM);
    const double flops = (8.0 * double(gen) + 4.0 * double(half)) * N / double(D);
    ProfScope ps(sv->stream, std::string("sparse_k") + std::to_string(K) + "_" + dt_name(sv->dt),
                 2.0 * double(sizeof(typename A::Amp)) * N, flops);
    k_sparse<A, K><<<(unsigned)grid, kSpThreads, smem, sv->stream>>>(
        reinterpret_cast<typename A::Amp *>(sv->data), ntiles, tg, lay, reinterpret_cast<const uint32_t *>(d),
        reinterpret_cast<const uint32_t *>(d + o_code), reinterpret_cast<const Val *>(d + o_val));
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

template <class A>
cast_status run_sparse_k(cast_sv *sv, const PreparedGate &g) {
    switch (g.k) {
        case 3: return run_sparse<A, 3>(sv, g);
        case 4: return run_sparse<A, 4>(sv, g);
        case 5: return run_sparse<A, 5>(sv, g);
        case 6: return run_sparse<A, 6>(sv, g);
        case 7: return run_sparse<A, 7>(sv, g);
        default: return fail(CAST_ERR_UNSUPPORTED, "sparse kernel covers k = 3..7");
    }
}

std::atomic<int> g_sparse_mode{CAST_SPARSE_AUTO};

}  // namespace

int64_t dense_opcount(int k) { return int64_t(1) << (2 * k + 2); }

bool sparse_preferred(const cast_sv *sv, const PreparedGate &g) {
    const int mode = g_sparse_mode.load();
    if (mode == CAST_SPARSE_OFF || g.cls != CLS_DENSE || g.k < 3 || sv->n < 12) return false;
    if (mode == CAST_SPARSE_ALWAYS) return sv->dt == CAST_C64 || f64_mode() == CAST_F64_EMULATED;
    const int64_t ops = opcount(g.m.data(), g.k, 0.0);
    if (sv->dt == CAST_C128) {
        // measured on a random 30-qubit state: the list kernel is at least as
        // fast as the unrolled double-float kernels for every dense-class gate of
        // k >= 3 (dense k = 3: 25 vs 27 ms; k = 4: 39 vs 42 ms; k = 5: 70 vs 69
        // ms), and k = 6, 7 have no other double-float kernel; the digit kernels
        // (apply_oz.cu) take the denser gates before this test is reached
        return f64_mode() == CAST_F64_EMULATED;
    }
    // complex64: unitary gates of k >= 4 run on the tensor cores at about one
    // memory pass (measured faster than the list at every density).  Other
    // dense-class gates (non-unitary, or with the tensor cores off) run on the
    // CUDA cores; measured per 30-qubit gate, the list kernel beats the dense
    // FP32 kernels for k = 5 up to ~80% of the dense operation count (15.6 ms
    // dense vs 12.8-15.9), for k = 6, 7 up to ~40% (74 / 145 ms dense vs
    // 32 / 61 ms), and for k = 4 up to 24 operations per amplitude
    if (tensor_cores_on() && g.unitary && g.k >= 4) return false;
    if (g.k == 4) return (ops >> g.k) <= 24;
    if (g.k == 5) return 5 * ops <= 4 * dense_opcount(g.k);
    return g.k >= 6 && 5 * ops <= 2 * dense_opcount(g.k);
}

int sparse_mode() { return g_sparse_mode.load(); }

cast_status launch_gate_sparse(cast_sv *sv, const PreparedGate &g) {
    if (sv->dt == CAST_C64) return run_sparse_k<C64>(sv, g);
    return run_sparse_k<C128>(sv, g);
}

}  // namespace cast

extern "C" {

cast_status cast_set_sparse_mode(int mode) {
    if (mode != CAST_SPARSE_AUTO && mode != CAST_SPARSE_OFF && mode != CAST_SPARSE_ALWAYS)
        return cast::fail(CAST_ERR_ARG, "unknown sparse-kernel mode");
    cast::g_sparse_mode = mode;
    return CAST_OK;
}

int cast_get_sparse_mode(void) { return cast::g_sparse_mode.load(); }

}  // extern "C"
