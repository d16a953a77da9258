// Batched variational circuits: the hardware-efficient ansatz (per layer: RY
// on every qubit, RZ on every qubit, then CZ(i, i+1) for i < n-1) on many
// instances of uneven qubit counts, with energies of
//     H = zz * sum_i Z_i Z_{i+1} + hx * sum_i X_i   (open boundary)
// and adjoint gradients.
//
// Tile executor.  Per-gate passes would read and write the whole state 3n-1
// times per layer.  Here a tile of 2^T amplitudes (T = 12 for complex64,
// 11 for complex128: 32 KB) is loaded into shared memory once per "group" of
// qubits and every rotation of that group is applied while the tile is
// resident:
//   group 0      qubits 0 .. T-1            (the tile is contiguous)
//   group g >= 1 qubits T+(g-1)G .. T+gG-1  (G = T-5, the last group may be
//                narrower); tile = index bits 0..4 (runs of 32 amplitudes
//                stay coalesced) plus a window of G consecutive index bits
//                that holds the group's qubits: those qubits and above, or
//                for a narrow last group the top G bits.  Every tile of an
//                instance with n >= T is thus a full 2^T amplitudes; the
//                window bits that are not rotated are batch bits.
// A layer is then ~n/G passes.  Rotations on different qubits commute, so the
// layer "RY on all, RZ on all, CZ ladder" is applied per group as: the RY
// gates in register rounds of up to three qubits (each thread gathers the 8
// amplitudes of a sub-slice, applies three 2x2 rotations, scatters them back),
// then the group's RZ gates together as one diagonal phase looked up from two
// small tables, then (last group) the CZ ladder as a sign from the global
// index, both while the tile is stored.  The tile is XOR-swizzled in shared
// memory so that sub-slices of low qubits do not collide in the banks.
//
// Energies: one read-only pass per group; group 0 also forms the diagonal
// ZZ part; the X_q terms of a group's qubits are formed from amplitude pairs
// inside the tile.  lambda = H psi is built the same way (group 0 writes, the
// others accumulate).  The adjoint backward sweep visits the layers in reverse
// and, per layer, the groups in reverse (the last group first, undoing the CZ
// ladder at load); it forms every Im<lam|Z_q|psi> of the group from one sweep
// (the RZ gates commute with each other and act last) and un-applies their
// diagonal, then per qubit forms Im<lam|Y_q|psi> and un-applies RY, on psi and
// lam together.  Because the gradient of a gate is unchanged by reordering
// gates that commute with it, this gives the gradients of the layer-ordered
// circuit.
//
// Work distribution: one launch per (layer, group) covers the tiles of every
// instance that has that group; each CTA takes a contiguous range of the tile
// list, so it mostly stays within one instance.  Per-instance energy and
// gradient sums go through shared-memory accumulators flushed with FP64
// atomics when the instance changes.  The whole sequence of launches is
// captured once into a CUDA graph and replayed for every parameter set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace cast {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxGroups = 8;

struct HeaInst {
    uint64_t off;      // amplitude offset of the state in the arena
    int n;
    int ngroups;
    int param_off;     // offset of this instance's 2 n L parameters
    int rot_off;       // offset of its L x n rotation entries
};

// Arithmetic of a batch: complex64 (float), complex128 on the FP64 pipe
// (double), or complex128-class double-float arithmetic on the FP32 pipe (DF:
// a real is an unevaluated sum hi + lo of two floats, ~48 significant bits,
// an amplitude (re_hi, re_lo, im_hi, im_lo)).  The batch's state arena is
// private to it, so a DF batch keeps its amplitudes in that layout in HBM as
// well (16 bytes, like complex128) and no FP64 conversion touches the
// state; only the sums that leave a warp are formed in FP64.  Amp is the
// amplitude type (HBM, registers and shared memory), Real a scalar.
struct DF {};
template <typename R> struct HT;
template <> struct HT<float> {
    using Amp = float2;
    using Real = float;
    static constexpr int T = 12;  // tile bits: 32 KB tiles
};
template <> struct HT<double> {
    using Amp = double2;
    using Real = double;
    static constexpr int T = 11;
};
template <> struct HT<DF> {
    using Amp = float4;
    using Real = float2;
    static constexpr int T = 11;
};

template <typename R>
struct Rot {  // RY: [[c, -s], [s, c]];  RZ: diag(cz - i sz, cz + i sz)
    typename HT<R>::Real cy, sy, cz, sz;
};

// ---- scalar and complex helpers per arithmetic
__device__ __forceinline__ float rmul(float a, float b) { return a * b; }
__device__ __forceinline__ double rmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 rmul(float2 a, float2 b) {  // double-float product
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float s = p + e;
    return make_float2(s, e - (s - p));
}
__device__ __forceinline__ float radd(float a, float b) { return a + b; }
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 radd(float2 a, float2 b) {  // double-float sum (TwoSum of the heads)
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float rneg(float a) { return -a; }
__device__ __forceinline__ double rneg(double a) { return -a; }
__device__ __forceinline__ float2 rneg(float2 a) { return make_float2(-a.x, -a.y); }
// a b + c d
__device__ __forceinline__ float rdot2(float a, float b, float c, float d) { return fmaf(a, b, c * d); }
__device__ __forceinline__ double rdot2(double a, double b, double c, double d) { return fma(a, b, c * d); }
__device__ __forceinline__ float2 rdot2(float2 a, float2 b, float2 c, float2 d) {
    // exact head products (FMA error terms), TwoSum of the heads, the cross
    // terms of the tails folded into the error, one renormalisation
    const float p1 = a.x * b.x, p2 = c.x * d.x;
    const float e1 = fmaf(a.x, b.x, -p1), e2 = fmaf(c.x, d.x, -p2);
    const float s = p1 + p2;
    const float bb = s - p1;
    float t = (p1 - (s - bb)) + (p2 - bb);
    t += e1 + e2;
    t = fmaf(a.x, b.y, t);
    t = fmaf(a.y, b.x, t);
    t = fmaf(c.x, d.y, t);
    t = fmaf(c.y, d.x, t);
    const float h = s + t;
    return make_float2(h, t - (h - s));
}
__device__ __forceinline__ double to_double(float a) { return double(a); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(float2 a) { return double(a.x) + double(a.y); }
// an integer (|v| < 2^24) as an exact Real
template <typename Re> __device__ __forceinline__ Re rfrom_i(int v);
template <> __device__ __forceinline__ float rfrom_i<float>(int v) { return float(v); }
template <> __device__ __forceinline__ double rfrom_i<double>(int v) { return double(v); }
template <> __device__ __forceinline__ float2 rfrom_i<float2>(int v) { return make_float2(float(v), 0.f); }
// shuffles of a Real
__device__ __forceinline__ float rshfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double rshfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float2 rshfl_xor(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ float rshfl(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double rshfl(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float2 rshfl(float2 v, int l) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
template <typename Re> __host__ __device__ __forceinline__ Re rfrom_d(double v);
template <> __host__ __device__ __forceinline__ float rfrom_d<float>(double v) { return float(v); }
template <> __host__ __device__ __forceinline__ double rfrom_d<double>(double v) { return v; }
template <> __host__ __device__ __forceinline__ float2 rfrom_d<float2>(double v) {
    const float h = float(v);
    return make_float2(h, float(v - double(h)));
}
template <typename Re> __device__ __forceinline__ Re rzero();
template <> __device__ __forceinline__ float rzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double rzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 rzero<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ float re_of(float2 v) { return v.x; }
__device__ __forceinline__ float im_of(float2 v) { return v.y; }
__device__ __forceinline__ double re_of(double2 v) { return v.x; }
__device__ __forceinline__ double im_of(double2 v) { return v.y; }
__device__ __forceinline__ float2 re_of(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 im_of(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 make_amp(float re, float im) { return make_float2(re, im); }
__device__ __forceinline__ double2 make_amp(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ float4 make_amp(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }

template <typename A>
__device__ __forceinline__ A amul(A a, A b) {  // complex product
    return make_amp(rdot2(re_of(a), re_of(b), rneg(im_of(a)), im_of(b)), rdot2(re_of(a), im_of(b), im_of(a), re_of(b)));
}
template <typename A>
__device__ __forceinline__ A aneg(A a) {
    return make_amp(rneg(re_of(a)), rneg(im_of(a)));
}
template <typename A>
__device__ __forceinline__ A aconj(A a) {
    return make_amp(re_of(a), rneg(im_of(a)));
}
template <typename A, typename Re>
__device__ __forceinline__ A ascale(A a, Re r) {
    return make_amp(rmul(re_of(a), r), rmul(im_of(a), r));
}
template <typename A>
__device__ __forceinline__ A aadd(A a, A b) {
    return make_amp(radd(re_of(a), re_of(b)), radd(im_of(a), im_of(b)));
}
// Im(conj(b) a) and Re(conj(a) c)
template <typename A>
__device__ __forceinline__ auto im_conj_mul(A b, A a) {
    return rdot2(re_of(b), im_of(a), rneg(im_of(b)), re_of(a));
}
template <typename A>
__device__ __forceinline__ auto re_conj_mul(A a, A c) {
    return rdot2(re_of(a), re_of(c), im_of(a), im_of(c));
}

// warp sum of a Real in its own arithmetic (fp32 for complex64)
template <typename Re>
__device__ __forceinline__ Re warp_sum_r(Re v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = radd(v, rshfl_xor(v, o));
    return v;
}

// A running sum of Real values: compensated fp32 for complex64, FP64 on the
// FP64 pipe, double-float for DF (no FP64 instruction until value()).  A
// plain aggregate, so it can live in shared memory; zero() or {} clears it.
// get() returns the sum as a Real, value() as a double.
template <typename R> struct RAcc;
template <> struct RAcc<float> {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float v) {
        const float s = hi + v;
        const float bb = s - hi;
        lo += (hi - (s - bb)) + (v - bb);
        hi = s;
    }
    __device__ __forceinline__ float get() const { return hi + lo; }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};
template <> struct RAcc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct RAcc<DF> {
    float2 s;
    __device__ __forceinline__ void zero() { s = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float2 v) { s = radd(s, v); }
    __device__ __forceinline__ float2 get() const { return s; }
    __device__ __forceinline__ double value() const { return double(s.x) + double(s.y); }
};

// one launch = (layer, group); instances with that group and their tile ranges
struct PassArgs {
    int layer;
    int group;
    int ninst;
    const int *inst;         // instance ids having this group
    const uint64_t *prefix;  // tile prefix sums (ninst + 1)
};

template <typename R> constexpr int tile_bits() { return HT<R>::T; }
constexpr int kDfRoundBits = 2;

// Geometry of group g of an n-qubit instance for tile width T.
struct Geo {
    int T0;        // number of tile bits
    int rb0;       // first rotated local bit
    int nrot;      // number of rotated qubits (local bits rb0 .. rb0+nrot-1)
    int q0;        // qubit of local bit rb0
    int p0;        // global position of local bit 5 (g >= 1): local bits 5 .. T0-1 are global p0 .. p0+T0-6
    bool contiguous;
};

__host__ __device__ inline Geo geometry(int n, int g, int T) {
    Geo G;
    if (g == 0) {
        G.T0 = n < T ? n : T;
        G.rb0 = 0;
        G.nrot = G.T0;
        G.q0 = 0;
        G.p0 = 0;
        G.contiguous = true;
    } else {
        const int W = T - 5;
        const int lo = T + (g - 1) * W, hi = (T + g * W < n) ? T + g * W : n;
        const int w0 = lo + W <= n ? lo : n - W;  // window [w0, w0 + W) holds [lo, hi); w0 >= 5 as n > T
        G.nrot = hi - lo;
        G.T0 = T;
        G.rb0 = 5 + (lo - w0);
        G.q0 = lo;
        G.p0 = w0;
        G.contiguous = false;
    }
    return G;
}

__host__ __device__ inline int group_count(int n, int T) {
    if (n <= T) return 1;
    const int W = T - 5;
    return 1 + (n - T + W - 1) / W;
}

// global amplitude index of local index l in tile t of group geometry G
__device__ __forceinline__ uint64_t tile_global(const Geo &G, uint64_t t, uint32_t l) {
    if (G.contiguous) return (t << G.T0) | l;
    // non-tile bits: 5 .. p0-1 (low part of t) and p0+T0-5 .. n-1 (high part)
    const int lowbits = G.p0 - 5;
    const uint64_t tlo = t & ((uint64_t(1) << lowbits) - 1), thi = t >> lowbits;
    return (thi << (G.p0 + G.T0 - 5)) | (uint64_t(l >> 5) << G.p0) | (tlo << 5) | (l & 31u);
}

__device__ __forceinline__ bool cz_ladder_odd(uint64_t x, int n) {
    const uint64_t m = n > 1 ? ((uint64_t(1) << (n - 1)) - 1) : 0;
    return __popcll(x & (x >> 1) & m) & 1;
}

// XOR swizzle of the shared tile, linear over disjoint bits and bijective
// on any tile; it only reads index bits 3..6, so sw(l + 256 i) = sw(l) + 256 i.
// A shared-memory phase serves 32 banks = 16 complex64 or 8 complex128
// amplitudes, so the lanes of a phase must land on distinct low slot bits
// for every access pattern: consecutive indices (loads, stores), and the
// register rounds on bits 0-2 (lanes vary index bits 3-6), 3-5 (lanes vary
// bits 0-2 and 6), 6-7 and 5-7 (lanes vary bits 0-3).
//   complex64:  bit 4 -> slot bit 0, bit 5 -> 1, bit 6 -> 2 and 3
//   complex128: bits 3, 4, 5 -> slot bits 0, 1, 2
//   double-float (16-byte elements too, backward rounds of two bits, whose
//   round on bits 2-3 has lanes varying bits 0, 1, 4): bit 3 -> slot bit 0,
//   bit 4 -> slot bits 1 and 2, bit 5 -> slot bit 2
template <typename R> __device__ __forceinline__ uint32_t sw(uint32_t l);
template <> __device__ __forceinline__ uint32_t sw<float>(uint32_t l) {
    return l ^ ((l >> 4) & 3u) ^ (((l >> 6) & 1u) * 12u);
}
template <> __device__ __forceinline__ uint32_t sw<double>(uint32_t l) { return l ^ ((l >> 3) & 7u); }
template <> __device__ __forceinline__ uint32_t sw<DF>(uint32_t l) {
    return l ^ ((l >> 3) & 1u) ^ (((l >> 4) & 1u) * 6u) ^ (((l >> 5) & 1u) << 2);
}

// A thread's share of a tile: register i holds local index l = threadIdx.x +
// 256 i, global index x0 + i * stride (the register index occupies global
// bits s .. s + log2(IT) - 1, zero in x0) and shared slot sw<R>(threadIdx.x) + 256 i
// (the swizzle only mixes bits 0..5).
struct TileAddr {
    uint64_t x0, stride;
    int s;
};
__device__ __forceinline__ TileAddr tile_addr(const Geo &G, uint64_t t) {
    TileAddr a;
    a.x0 = tile_global(G, t, threadIdx.x);
    a.s = G.contiguous ? 8 : G.p0 + 3;
    a.stride = uint64_t(1) << a.s;
    return a;
}

// CZ-ladder signs of a thread's registers (bit i set: odd number of adjacent
// set pairs below bit n in x0 | (i << s)).  The pairs split into those of x0,
// those inside i, and the two that straddle the register bits: (s-1, s) and
// (s+w-1, s+w), w = number of register bits that hold amplitudes.
__device__ __forceinline__ uint32_t cz_mask(const TileAddr &a, int w, int n) {
    constexpr uint32_t kInner = 0xB848u;  // bit i: parity of popc(i & (i >> 1)), i < 16
    const uint32_t c0 = cz_ladder_odd(a.x0, n) ? 0xFFFFu : 0u;
    const uint32_t lo = a.s > 0 && ((a.x0 >> (a.s - 1)) & 1) ? 0xAAAAu : 0u;  // i bit 0 pairs with bit s-1
    const uint32_t top = w == 1 ? 0xAAAAu : (w == 2 ? 0xCCCCu : (w == 3 ? 0xF0F0u : 0xFF00u));  // i bit w-1
    const uint32_t hi = (w > 0 && ((a.x0 >> (a.s + w)) & 1)) ? top : 0u;
    return c0 ^ kInner ^ lo ^ hi;
}

// Phase of the group's RZ gates, split by where the rotated local bits sit:
// pa[l & 255] covers the bits below 8 (a thread's own), pb[i] the bits from 8
// on (its register index); each entry is a product over those qubits of
// (cz - i sz) for bit 0 or (cz + i sz) for bit 1.
template <typename R>
__device__ void phase_factors(typename HT<R>::Amp *pa, typename HT<R>::Amp *pb, const Geo &G, const Rot<R> *rots) {
    using A = typename HT<R>::Amp;
    using Re = typename HT<R>::Real;
    for (int e = threadIdx.x; e < 256 + 16; e += blockDim.x) {
        const bool low = e < 256;
        const uint32_t idx = low ? uint32_t(e) : uint32_t(e - 256);
        A v = make_amp(rfrom_d<Re>(1.0), rzero<Re>());
        for (int r = 0; r < G.nrot; r++) {
            const int lb = G.rb0 + r;
            if (low != (lb < 8)) continue;
            const Rot<R> q = rots[G.q0 + r];
            const Re sg = ((idx >> (low ? lb : lb - 8)) & 1) ? q.sz : rneg(q.sz);  // cz + i sg
            v = amul(v, make_amp(q.cz, sg));
        }
        if (low) pa[idx] = v;
        else pb[idx] = v;
    }
}

// pa and pb, plus (groups whose rotated bits start at 5 or above, where pa
// depends on the warp only) their products pc[warp * 16 + i]: the phase of a
// register is then one broadcast load.  Ends with a barrier.
template <typename R>
__device__ void build_split_phase(typename HT<R>::Amp *pa, typename HT<R>::Amp *pb, typename HT<R>::Amp *pc,
                                  const Geo &G, const Rot<R> *rots) {
    phase_factors<R>(pa, pb, G, rots);
    __syncthreads();
    if (G.rb0 >= 5 && threadIdx.x < 128) pc[threadIdx.x] = amul(pa[(threadIdx.x >> 4) << 5], pb[threadIdx.x & 15u]);
    __syncthreads();
}


// locate the instance of global tile index gt (binary search on the prefix)
__device__ __forceinline__ int find_inst(const PassArgs &P, uint64_t gt) {
    int lo = 0, hi = P.ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.prefix[mid] <= gt) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// (a, b) <- (c a - s b, s a + c b)
template <typename A, typename Re>
__device__ __forceinline__ void ry(A &a, A &b, Re c, Re s) {
    const A x = a, y = b;
    const Re ns = rneg(s);
    a = make_amp(rdot2(c, re_of(x), ns, re_of(y)), rdot2(c, im_of(x), ns, im_of(y)));
    b = make_amp(rdot2(s, re_of(x), c, re_of(y)), rdot2(s, im_of(x), c, im_of(y)));
}
// forward: RY_q on the pair (a, b) of qubit q (the group's RZ gates follow as
// one diagonal phase when the tile is stored)
template <typename T2, typename R>
__device__ __forceinline__ void fwd_pair(T2 &a, T2 &b, const Rot<R> &r) {
    ry(a, b, r.cy, r.sy);
}

// apply the forward rotations of local bits bits[0..nb) (nb <= 3) to the tile
template <typename R, int NB>
__device__ void tile_round(typename HT<R>::Amp *tile, int T0, const int *bits, const Rot<R> *rot) {
    using T2 = typename HT<R>::Amp;
    const uint32_t nsub = 1u << (T0 - NB);
    for (uint32_t s = threadIdx.x; s < nsub; s += blockDim.x) {
        uint32_t base = s;
#pragma unroll
        for (int i = 0; i < NB; i++) {  // bits ascending
            const int b = bits[i];
            base = ((base >> b) << (b + 1)) | (base & ((1u << b) - 1));
        }
        T2 v[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            uint32_t o = base;
#pragma unroll
            for (int i = 0; i < NB; i++)
                if ((j >> i) & 1) o |= 1u << bits[i];
            v[j] = tile[sw<R>(o)];
        }
#pragma unroll
        for (int i = 0; i < NB; i++)
#pragma unroll
            for (int j = 0; j < (1 << NB); j++)
                if (!((j >> i) & 1)) fwd_pair(v[j], v[j | (1 << i)], rot[i]);
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            uint32_t o = base;
#pragma unroll
            for (int i = 0; i < NB; i++)
                if ((j >> i) & 1) o |= 1u << bits[i];
            tile[sw<R>(o)] = v[j];
        }
    }
}

// The same round with the NB rotated bits B0 .. B0+NB-1 fixed at compile
// time.  The swizzle is linear over disjoint bits (sw<R>(a | b) = sw<R>(a) ^ sw<R>(b)),
// so each member's slot is the sub-slice's slot XOR a constant.
template <typename R, int B0, int NB>
__device__ void tile_round_ct(typename HT<R>::Amp *tile, int T0, const Rot<R> *rot) {
    using T2 = typename HT<R>::Amp;
    const uint32_t nsub = 1u << (T0 - NB);
    for (uint32_t s = threadIdx.x; s < nsub; s += blockDim.x) {
        const uint32_t sb = sw<R>(((s >> B0) << (B0 + NB)) | (s & ((1u << B0) - 1)));
        T2 v[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) v[j] = tile[sb ^ sw<R>(uint32_t(j) << B0)];
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const Rot<R> ri = rot[i];
#pragma unroll
            for (int j = 0; j < (1 << NB); j++)
                if (!((j >> i) & 1)) fwd_pair(v[j], v[j | (1 << i)], ri);
        }
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) tile[sb ^ sw<R>(uint32_t(j) << B0)] = v[j];
    }
}

// A thread's loaded share of a tile (local index l = threadIdx.x + 256 i)
// holds complete sub-slices over local bits 8 .. 8 + log2(IT) - 1, so the RY
// gates on those bits are applied in registers before the tile is parked.
template <typename R> constexpr int reg_bits() { return tile_bits<R>() - 8; }

template <typename R, typename Regs>
__device__ __forceinline__ void reg_rotations(Regs &b, const Geo &G, int T0, const Rot<R> *rots) {
    constexpr int IT = 1 << reg_bits<R>();
#pragma unroll
    for (int rb = 0; rb < reg_bits<R>(); rb++) {
        const int lb = 8 + rb;
        if (lb >= T0 || lb < G.rb0 || lb >= G.rb0 + G.nrot) continue;
        const Rot<R> r = rots[G.q0 + lb - G.rb0];
        const int nact = 1 << (T0 - 8);  // registers holding amplitudes
#pragma unroll
        for (int i = 0; i < IT; i++)
            if (!((i >> rb) & 1) && i < nact) fwd_pair(b.v[i], b.v[i | (1 << rb)], r);
    }
}

// The RY gates of the rotated bits below 8 (those above were applied in
// registers): fixed rounds for the full-width groups, else rounds of three
// with runtime bit positions.
template <typename R>
__device__ __forceinline__ void smem_rotations(typename HT<R>::Amp *tile, const Geo &G, int T0, const Rot<R> *rots) {
    const int hi = G.rb0 + G.nrot < 8 ? G.rb0 + G.nrot : 8;
    if (G.rb0 >= hi) return;
    const Rot<R> *r = rots + G.q0;  // RY/RZ entries of the group's rotated qubits, in order
    if (T0 >= 8 && G.rb0 == 0 && hi == 8) {
        tile_round_ct<R, 0, 3>(tile, T0, r);
        __syncthreads();
        tile_round_ct<R, 3, 3>(tile, T0, r + 3);
        __syncthreads();
        tile_round_ct<R, 6, 2>(tile, T0, r + 6);
        __syncthreads();
        return;
    }
    if (G.rb0 == 5 && hi == 8) {
        tile_round_ct<R, 5, 3>(tile, T0, r);
        __syncthreads();
        return;
    }
    for (int b0 = G.rb0; b0 < hi; b0 += 3) {
        const int nb = hi - b0 < 3 ? hi - b0 : 3;
        int bits[3];
        Rot<R> rr[3];
        for (int i = 0; i < nb; i++) {
            bits[i] = b0 + i;
            rr[i] = rots[G.q0 + b0 - G.rb0 + i];
        }
        if (nb == 3) tile_round<R, 3>(tile, T0, bits, rr);
        else if (nb == 2) tile_round<R, 2>(tile, T0, bits, rr);
        else tile_round<R, 1>(tile, T0, bits, rr);
        __syncthreads();
    }
}

// A thread's share of one tile: IT = 2^T / 256 amplitudes, loaded together so
// that all of them are in flight at once.
template <typename R>
struct TileRegs {
    static constexpr int IT = (1 << tile_bits<R>()) / kThreads;
    typename HT<R>::Amp v[IT];
};

template <typename R>
__device__ __forceinline__ void tile_load(TileRegs<R> &b, const typename HT<R>::Amp *__restrict__ sv, const TileAddr &a,
                                          uint32_t sz) {
#pragma unroll
    for (int i = 0; i < TileRegs<R>::IT; i++)
        if (threadIdx.x + uint32_t(i) * kThreads < sz) b.v[i] = (sv[a.x0 + uint64_t(i) * a.stride]);
}

template <typename R>
__device__ __forceinline__ void tile_put(const TileRegs<R> &b, typename HT<R>::Amp *tile, uint32_t sz) {
    const uint32_t s0 = sw<R>(threadIdx.x);
#pragma unroll
    for (int i = 0; i < TileRegs<R>::IT; i++)
        if (threadIdx.x + uint32_t(i) * kThreads < sz) tile[s0 + uint32_t(i) * kThreads] = b.v[i];
}

// FULL: every tile of the pass has 2^T amplitudes (all its instances have
// n >= T), so the tile size is a compile-time constant and the per-element
// guards fold away
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 2)
k_hea_forward(typename HT<R>::Amp *__restrict__ arena, const HeaInst *__restrict__ insts,
              const Rot<R> *__restrict__ rot, const __grid_constant__ PassArgs P) {
    using T2 = typename HT<R>::Amp;
    constexpr int T = tile_bits<R>();
    constexpr int IT = TileRegs<R>::IT;
    __shared__ __align__(16) T2 tile[1 << T];
    __shared__ __align__(16) T2 pa[256], pb[16], pc[128];
    const uint64_t total = P.prefix[P.ninst];
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t t_begin = uint64_t(blockIdx.x) * per;
    const uint64_t t_end = t_begin + per < total ? t_begin + per : total;
    if (t_begin >= t_end) return;
    int table_inst = -1;
    // the next tile's loads are issued before this tile's rotations run
    TileRegs<R> buf;
    int k = find_inst(P, t_begin);
    HeaInst I = insts[P.inst[k]];
    Geo G = geometry(I.n, P.group, T);
    uint64_t t = t_begin - P.prefix[k];
    tile_load<R>(buf, arena + I.off, tile_addr(G, t), FULL ? (1u << T) : (1u << G.T0));
    for (uint64_t gt = t_begin; gt < t_end; gt++) {
        const int T0 = FULL ? T : G.T0;
        const uint32_t sz = 1u << T0;
        const Rot<R> *lr = rot + I.rot_off + size_t(P.layer) * I.n;
        reg_rotations<R>(buf, G, T0, lr);
        tile_put<R>(buf, tile, sz);
        const HeaInst Ic = I;
        const Geo Gc = G;
        const uint64_t tc = t;
        // the phase tables depend on the instance only (the tile list of an
        // instance starts at prefix = gt - tc); rebuilt when it changes
        const int inst_id = int(gt - tc);
        if (inst_id != table_inst) {
            build_split_phase<R>(pa, pb, pc, Gc, lr);
            table_inst = inst_id;
        } else {
            __syncthreads();
        }
        if (gt + 1 < t_end) {
            k = find_inst(P, gt + 1);
            I = insts[P.inst[k]];
            G = geometry(I.n, P.group, T);
            t = gt + 1 - P.prefix[k];
            tile_load<R>(buf, arena + I.off, tile_addr(G, t), FULL ? (1u << T) : (1u << G.T0));
        }
        smem_rotations<R>(tile, Gc, T0, lr);
        // the group's RZ gates as one diagonal, then (last group) the CZ ladder
        const TileAddr a = tile_addr(Gc, tc);
        const uint32_t czm = (P.group == Ic.ngroups - 1)
                                 ? cz_mask(a, T0 > 8 ? T0 - 8 : 0, Ic.n) : 0u;
        const uint32_t s0 = sw<R>(threadIdx.x);
        typename HT<R>::Amp *sv = arena + Ic.off;
        auto store = [&](auto warp_phase) {
            const T2 pt = pa[threadIdx.x & 255u];
            const T2 *pw = pc + ((threadIdx.x >> 5) << 4);
#pragma unroll
            for (int i = 0; i < IT; i++) {
                if (threadIdx.x + uint32_t(i) * kThreads >= sz) continue;
                const T2 ph = warp_phase.value ? pw[i] : amul(pt, pb[i]);
                T2 v = amul(ph, tile[s0 + uint32_t(i) * kThreads]);
                if ((czm >> i) & 1) v = aneg(v);
                sv[a.x0 + uint64_t(i) * a.stride] = (v);
            }
        };
        if (Gc.rb0 >= 5) store(std::true_type{});
        else store(std::false_type{});
        __syncthreads();
    }
}

// shared-memory FP64 accumulator slots flushed to global when the instance changes
__device__ __forceinline__ void flush_slots(double *acc, int nslots, double *dst) {
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        if (acc[i] != 0.0) atomicAdd(dst + i, acc[i]);
        acc[i] = 0.0;
    }
}

// energy contribution of one group: ZZ (group 0 only) and X_q of the group's qubits
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_hea_energy(const typename HT<R>::Amp *__restrict__ arena, const HeaInst *__restrict__ insts,
             const __grid_constant__ PassArgs P, double zz, double hx, double *__restrict__ energy) {
    using T2 = typename HT<R>::Amp;
    constexpr int T = tile_bits<R>();
    __shared__ __align__(16) T2 tile[1 << T];
    __shared__ double slot;
    const uint64_t total = P.prefix[P.ninst];
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t t_begin = uint64_t(blockIdx.x) * per;
    const uint64_t t_end = t_begin + per < total ? t_begin + per : total;
    if (threadIdx.x == 0) slot = 0.0;
    int cur = -1;
    for (uint64_t gt = t_begin; gt < t_end; gt++) {
        const int k = find_inst(P, gt);
        const int id = P.inst[k];
        if (id != cur) {
            __syncthreads();
            if (cur >= 0) flush_slots(&slot, 1, energy + cur);
            __syncthreads();
            cur = id;
        }
        const HeaInst I = insts[id];
        const Geo G = geometry(I.n, P.group, T);
        const uint64_t t = gt - P.prefix[k];
        const typename HT<R>::Amp *sv = arena + I.off;
        const uint32_t sz = FULL ? (1u << T) : (1u << G.T0);
        using Re = typename HT<R>::Real;
        RAcc<R> acc{};
        const uint64_t zmask = I.n > 1 ? ((uint64_t(1) << (I.n - 1)) - 1) : 0;
        TileRegs<R> buf;
        const TileAddr ta = tile_addr(G, t);
        tile_load<R>(buf, sv, ta, sz);
        tile_put<R>(buf, tile, sz);
        if (P.group == 0) {
            const Re zzr = rfrom_d<Re>(zz);
#pragma unroll
            for (int i = 0; i < TileRegs<R>::IT; i++) {
                const uint32_t l = threadIdx.x + uint32_t(i) * kThreads;
                if (l >= sz) continue;
                const uint64_t x = ta.x0 + uint64_t(i) * ta.stride;
                const int odd = __popcll((x ^ (x >> 1)) & zmask);
                const T2 v = buf.v[i];
                acc.add(rmul(rmul(zzr, rfrom_i<Re>(I.n - 1 - 2 * odd)), re_conj_mul(v, v)));
            }
        }
        __syncthreads();
        // <X_q> = sum_x Re(conj(psi_x) psi_{x ^ 2^q}) = 2 sum_{x_q = 0} Re(...)
        const Re hx2 = rfrom_d<Re>(2.0 * hx);
        for (int r = 0; r < G.nrot; r++) {
            const int b = G.rb0 + r;
            for (uint32_t p = threadIdx.x; p < (sz >> 1); p += blockDim.x) {
                const uint32_t l0 = ((p >> b) << (b + 1)) | (p & ((1u << b) - 1));
                const T2 a = tile[sw<R>(l0)], c = tile[sw<R>(l0 | (1u << b))];
                acc.add(rmul(hx2, re_conj_mul(a, c)));
            }
        }
        const double v = to_double(warp_sum_r(acc.get()));
        if ((threadIdx.x & 31) == 0) atomicAdd(&slot, v);
        __syncthreads();
    }
    __syncthreads();
    if (cur >= 0) flush_slots(&slot, 1, energy + cur);
}

// lam = H psi for one group (group 0 writes, the others add)
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_hea_lambda(const typename HT<R>::Amp *__restrict__ psi, typename HT<R>::Amp *__restrict__ lam,
             const HeaInst *__restrict__ insts, const __grid_constant__ PassArgs P, double zz, double hx) {
    using T2 = typename HT<R>::Amp;
    constexpr int T = tile_bits<R>();
    __shared__ __align__(16) T2 tile[1 << T];
    const uint64_t total = P.prefix[P.ninst];
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t t_begin = uint64_t(blockIdx.x) * per;
    const uint64_t t_end = t_begin + per < total ? t_begin + per : total;
    for (uint64_t gt = t_begin; gt < t_end; gt++) {
        const int k = find_inst(P, gt);
        const HeaInst I = insts[P.inst[k]];
        const Geo G = geometry(I.n, P.group, T);
        const uint64_t t = gt - P.prefix[k];
        const uint32_t sz = FULL ? (1u << T) : (1u << G.T0);
        const TileAddr ta = tile_addr(G, t);
        {
            TileRegs<R> buf;
            tile_load<R>(buf, psi + I.off, ta, sz);
            tile_put<R>(buf, tile, sz);
        }
        __syncthreads();
        const uint64_t zmask = I.n > 1 ? ((uint64_t(1) << (I.n - 1)) - 1) : 0;
        using Re = typename HT<R>::Real;
        const Re zzr = rfrom_d<Re>(zz), hxr = rfrom_d<Re>(hx);
        for (uint32_t l = threadIdx.x, i = 0; l < sz; l += blockDim.x, i++) {
            const uint64_t x = ta.x0 + uint64_t(i) * ta.stride;
            T2 out;
            if (P.group == 0) {
                const int odd = __popcll((x ^ (x >> 1)) & zmask);
                out = ascale(tile[sw<R>(l)], rmul(zzr, rfrom_i<Re>(I.n - 1 - 2 * odd)));
            } else {
                out = (lam[I.off + x]);
            }
            for (int r = 0; r < G.nrot; r++) out = aadd(out, ascale(tile[sw<R>(l ^ (1u << (G.rb0 + r)))], hxr));
            lam[I.off + x] = (out);
        }
        __syncthreads();
    }
}

// One RY_q pair of psi and lam in the backward sweep: the pair's share of
// dE/dtheta_q = Im<lam|Y_q|psi> (Y psi = (-i p1, i p0):
// Im(conj(l0)(-i p1)) = -Re(conj(l0) p1), Im(conj(l1)(i p0)) = Re(conj(l1) p0)),
// then RY(-theta) on both.
template <typename T2, typename R>
__device__ __forceinline__ typename HT<R>::Real adj_pair(T2 &p0, T2 &p1, T2 &l0, T2 &l1, const Rot<R> &r) {
    const auto g = radd(re_conj_mul(l1, p0), rneg(re_conj_mul(l0, p1)));
    const auto ns = rneg(r.sy);
    ry(p0, p1, r.cy, ns);
    ry(l0, l1, r.cy, ns);
    return g;
}

// backward sweep of one (layer, group) on psi and lam, with gradients: the RY
// part of a round (the RZ gates were handled as one diagonal beforehand)
template <typename R, int NB>
__device__ void adj_round(typename HT<R>::Amp *tp, typename HT<R>::Amp *tl, int T0, const int *bits, const Rot<R> *rot,
                          RAcc<R> (&gy)[3]) {
    using T2 = typename HT<R>::Amp;
    const uint32_t nsub = 1u << (T0 - NB);
    for (uint32_t s = threadIdx.x; s < nsub; s += blockDim.x) {
        uint32_t base = s;
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const int b = bits[i];
            base = ((base >> b) << (b + 1)) | (base & ((1u << b) - 1));
        }
        T2 p[1 << NB], l[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            uint32_t o = base;
#pragma unroll
            for (int i = 0; i < NB; i++)
                if ((j >> i) & 1) o |= 1u << bits[i];
            p[j] = tp[sw<R>(o)];
            l[j] = tl[sw<R>(o)];
        }
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const Rot<R> r = rot[i];
            auto sy = rzero<typename HT<R>::Real>();  // this sub-slice's share, added to the sum once
#pragma unroll
            for (int j = 0; j < (1 << NB); j++)
                if (!((j >> i) & 1)) sy = radd(sy, adj_pair(p[j], p[j | (1 << i)], l[j], l[j | (1 << i)], r));
            gy[i].add(sy);
        }
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            uint32_t o = base;
#pragma unroll
            for (int i = 0; i < NB; i++)
                if ((j >> i) & 1) o |= 1u << bits[i];
            tp[sw<R>(o)] = p[j];
            tl[sw<R>(o)] = l[j];
        }
    }
}

// adj_round with the NB bits B0 .. B0+NB-1 fixed at compile time (see
// tile_round_ct for the addressing)
template <typename R, int B0, int NB>
__device__ void adj_round_ct(typename HT<R>::Amp *tp, typename HT<R>::Amp *tl, int T0, const Rot<R> *rot,
                             RAcc<R> (&gy)[3]) {
    using T2 = typename HT<R>::Amp;
    const uint32_t nsub = 1u << (T0 - NB);
    for (uint32_t s = threadIdx.x; s < nsub; s += blockDim.x) {
        const uint32_t sb = sw<R>(((s >> B0) << (B0 + NB)) | (s & ((1u << B0) - 1)));
        T2 p[1 << NB], l[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            p[j] = tp[sb ^ sw<R>(uint32_t(j) << B0)];
            l[j] = tl[sb ^ sw<R>(uint32_t(j) << B0)];
        }
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const Rot<R> r = rot[i];
            auto sy = rzero<typename HT<R>::Real>();
#pragma unroll
            for (int j = 0; j < (1 << NB); j++)
                if (!((j >> i) & 1)) sy = radd(sy, adj_pair(p[j], p[j | (1 << i)], l[j], l[j | (1 << i)], r));
            gy[i].add(sy);
        }
#pragma unroll
        for (int j = 0; j < (1 << NB); j++) {
            tp[sb ^ sw<R>(uint32_t(j) << B0)] = p[j];
            tl[sb ^ sw<R>(uint32_t(j) << B0)] = l[j];
        }
    }
}

// SR: every RY of the group is un-applied in shared-memory rounds (the
// registers only carry the tile from HBM through the RZ step), so the kernel
// fits two CTAs per SM; otherwise the RY gates of register-held bits 8.. are
// un-applied in registers.  Double-float takes SR (measured: 26-qubit
// adjoint 454 -> 334 ms), complex64 the register form (70 vs 75 ms).
template <typename R> constexpr bool bwd_smem_ry() { return std::is_same<R, DF>::value; }
// bits per generic shared-memory round of the backward
template <typename R> constexpr int bwd_round_bits() { return std::is_same<R, DF>::value ? kDfRoundBits : 3; }
template <typename R, bool SR, bool FULL>
__global__ void __launch_bounds__(kThreads, SR ? 2 : (sizeof(R) == 4 ? 2 : 1))
k_hea_backward(typename HT<R>::Amp *__restrict__ psi, typename HT<R>::Amp *__restrict__ lam,
               const HeaInst *__restrict__ insts, const Rot<R> *__restrict__ rot,
               const __grid_constant__ PassArgs P, double *__restrict__ grad) {
    using T2 = typename HT<R>::Amp;
    constexpr int T = tile_bits<R>();
    constexpr int IT = TileRegs<R>::IT;
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char hea_smem[];  // psi tile, lam tile (64 KB)
    T2 *tp = reinterpret_cast<T2 *>(hea_smem);
    T2 *tl = tp + (1 << T);
    // per-warp gradient sums, [warp][RY of each rotated qubit, RZ of each]:
    // each warp's lane 0 adds its per-tile sums, no atomics; summed over the
    // warps and sent to global memory when the instance changes
    __shared__ RAcc<R> gacc[NW][2 * T];
    __shared__ __align__(16) T2 pa[256], pb[16], pc[128];
    int table_inst = -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t total = P.prefix[P.ninst];
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t t_begin = uint64_t(blockIdx.x) * per;
    const uint64_t t_end = t_begin + per < total ? t_begin + per : total;
    for (int i = threadIdx.x; i < NW * 2 * T; i += blockDim.x) (&gacc[0][0])[i].zero();
    int cur = -1, cur_n = 0, cur_q0 = 0, cur_nrot = 0;
    int cur_poff = 0;
    auto flush = [&]() {
        // gacc[.][r] -> RY of qubit q0 + r, gacc[.][T + r] -> RZ of qubit q0 + r
        for (int i = threadIdx.x; i < 2 * T; i += blockDim.x) {
            const int r = i % T;
            double v = 0.0;
            for (int w = 0; w < NW; w++) {
                v += gacc[w][i].value();
                gacc[w][i].zero();
            }
            if (r < cur_nrot && v != 0.0) {
                const int q = cur_q0 + r;
                const int p = cur_poff + 2 * cur_n * P.layer + (i < T ? q : cur_n + q);
                atomicAdd(grad + p, v);
            }
        }
    };
    using Re = typename HT<R>::Real;
    auto add = [&](int slot, Re v) {  // lane 0 holds the warp's sum
        if (lane == 0) gacc[warp][slot].add(v);
    };
    __syncthreads();
    for (uint64_t gt = t_begin; gt < t_end; gt++) {
        const int k = find_inst(P, gt);
        const int id = P.inst[k];
        const HeaInst I = insts[id];
        const Geo G = geometry(I.n, P.group, T);
        if (id != cur) {
            __syncthreads();
            if (cur >= 0) flush();
            __syncthreads();
            cur = id;
            cur_n = I.n;
            cur_q0 = G.q0;
            cur_nrot = G.nrot;
            cur_poff = I.param_off;
        }
        const uint64_t t = gt - P.prefix[k];
        const int T0 = FULL ? T : G.T0;
        const uint32_t sz = 1u << T0;
        const bool last = P.group == I.ngroups - 1;
        const Rot<R> *lr = rot + I.rot_off + size_t(P.layer) * I.n;
        if (int(gt - t) != table_inst) {  // new instance: its RZ phase tables
            __syncthreads();
            build_split_phase<R>(pa, pb, pc, G, lr);
            table_inst = int(gt - t);
        }
        const TileAddr ta = tile_addr(G, t);
        {
            // psi and lam of the thread's share, both in flight together
            TileRegs<R> bp, bl;
            tile_load<R>(bp, psi + I.off, ta, sz);
            tile_load<R>(bl, lam + I.off, ta, sz);
            const uint32_t czm = last ? cz_mask(ta, T0 > 8 ? T0 - 8 : 0, I.n) : 0u;
            // the group's RZ gates act last in the layer and commute: every
            // dE/dphi_q = Im<lam|Z_q|psi> = sum_x (1 - 2 x_q) Im(conj(lam_x) psi_x)
            // is taken from the same state, then the diagonal is un-applied.
            // Rotated bits below 8 depend on the thread only, bits 8.. on i.
            Re wsum = rzero<Re>(), wreg[reg_bits<R>()];
#pragma unroll
            for (int rb = 0; rb < reg_bits<R>(); rb++) wreg[rb] = rzero<Re>();
            auto rz = [&](auto warp_phase) {
                const T2 pt = pa[threadIdx.x & 255u];
                const T2 *pw = pc + ((threadIdx.x >> 5) << 4);
#pragma unroll
                for (int i = 0; i < IT; i++) {
                    if (threadIdx.x + uint32_t(i) * kThreads >= sz) continue;
                    T2 a = bp.v[i], b = bl.v[i];
                    if ((czm >> i) & 1) {  // undo the CZ ladder (self-inverse)
                        a = aneg(a);
                        b = aneg(b);
                    }
                    const Re w = im_conj_mul(b, a);
                    wsum = radd(wsum, w);
#pragma unroll
                    for (int rb = 0; rb < reg_bits<R>(); rb++) wreg[rb] = radd(wreg[rb], ((i >> rb) & 1) ? rneg(w) : w);
                    const T2 ph = aconj(warp_phase.value ? pw[i] : amul(pt, pb[i]));
                    bp.v[i] = amul(ph, a);
                    bl.v[i] = amul(ph, b);
                }
            };
            if (G.rb0 >= 5) rz(std::true_type{});
            else rz(std::false_type{});
            // sums over the warp with lane-dependent signs (rotated bits 0..4):
            // a Walsh-Hadamard butterfly leaves sum_l (-1)^popc(j & l) w_l in lane j
            Re h = wsum;
#pragma unroll
            for (int b = 0; b < 5; b++) {
                const Re o = rshfl_xor(h, 1 << b);
                h = ((lane >> b) & 1) ? radd(o, rneg(h)) : radd(h, o);
            }
            Re hl[5];
#pragma unroll
            for (int b = 0; b < 5; b++) hl[b] = rshfl(h, 1 << b);
            const Re htot = rshfl(h, 0);
            for (int r = 0; r < G.nrot; r++) {
                const int lb = G.rb0 + r;
                if (lb < 5) {
                    Re v = rzero<Re>();
#pragma unroll
                    for (int b = 0; b < 5; b++)
                        if (lb == b) v = hl[b];
                    add(T + r, v);
                } else if (lb < 8) {
                    add(T + r, ((threadIdx.x >> lb) & 1) ? rneg(htot) : htot);
                }
            }
#pragma unroll
            for (int rb = 0; rb < reg_bits<R>(); rb++) {
                const int lb = 8 + rb;
                if (lb >= T0 || lb < G.rb0 || lb >= G.rb0 + G.nrot) continue;
                add(T + lb - G.rb0, warp_sum_r(wreg[rb]));
            }
            // RY gradients and un-rotation of the register-held bits 8..
            if constexpr (!SR) {
#pragma unroll
                for (int rb = 0; rb < reg_bits<R>(); rb++) {
                    const int lb = 8 + rb;
                    if (lb >= T0 || lb < G.rb0 || lb >= G.rb0 + G.nrot) continue;
                    const Rot<R> r = lr[G.q0 + lb - G.rb0];
                    const int nact = int(sz >> 8);  // registers holding amplitudes (lb < T0, so >= 2)
                    Re sy = rzero<Re>();
#pragma unroll
                    for (int i = 0; i < IT; i++)
                        if (!((i >> rb) & 1) && i < nact)
                            sy = radd(sy, adj_pair(bp.v[i], bp.v[i | (1 << rb)], bl.v[i], bl.v[i | (1 << rb)], r));
                    add(lb - G.rb0, warp_sum_r(sy));
                }
            }
            tile_put<R>(bp, tp, sz);
            tile_put<R>(bl, tl, sz);
        }
        __syncthreads();
        // RY gradients and un-rotation of the rotated bits below 8 (all of
        // them for SR), through shared memory
        {
            const int hi = SR ? G.rb0 + G.nrot : (G.rb0 + G.nrot < 8 ? G.rb0 + G.nrot : 8);
            const Rot<R> *r = lr + G.q0;
            auto flush_gy = [&](RAcc<R> (&gy)[3], int r0, int nb) {
                for (int i = 0; i < nb; i++) add(r0 + i, warp_sum_r(gy[i].get()));
            };
            if (SR && std::is_same<R, float>::value && T0 == 12 && G.rb0 == 0 && hi == 12) {
                // complex64 group 0: four fixed rounds of three bits
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 0, 3>(tp, tl, T0, r, gy);
                    flush_gy(gy, 0, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 3, 3>(tp, tl, T0, r + 3, gy);
                    flush_gy(gy, 3, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 6, 3>(tp, tl, T0, r + 6, gy);
                    flush_gy(gy, 6, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 9, 3>(tp, tl, T0, r + 9, gy);
                    flush_gy(gy, 9, 3);
                }
                __syncthreads();
            } else if (SR && std::is_same<R, float>::value && G.rb0 == 5 && hi == 12) {
                // complex64 full-width group: rounds of three bits from bit 5
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 5, 3>(tp, tl, T0, r, gy);
                    flush_gy(gy, 0, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 8, 3>(tp, tl, T0, r + 3, gy);
                    flush_gy(gy, 3, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 11, 1>(tp, tl, T0, r + 6, gy);
                    flush_gy(gy, 6, 1);
                }
                __syncthreads();
            } else if (!SR && T0 >= 8 && G.rb0 == 0 && hi == 8) {
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 0, 3>(tp, tl, T0, r, gy);
                    flush_gy(gy, 0, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 3, 3>(tp, tl, T0, r + 3, gy);
                    flush_gy(gy, 3, 3);
                }
                __syncthreads();
                {
                    RAcc<R> gy[3]{};
                    adj_round_ct<R, 6, 2>(tp, tl, T0, r + 6, gy);
                    flush_gy(gy, 6, 2);
                }
                __syncthreads();
            } else if (!SR && G.rb0 == 5 && hi == 8) {
                RAcc<R> gy[3]{};
                adj_round_ct<R, 5, 3>(tp, tl, T0, r, gy);
                flush_gy(gy, 0, 3);
                __syncthreads();
            } else {
                constexpr int NBM = bwd_round_bits<R>();
                for (int b0 = G.rb0; b0 < hi; b0 += NBM) {
                    const int nb = hi - b0 < NBM ? hi - b0 : NBM;
                    int bits[3];
                    Rot<R> rr[3];
                    for (int i = 0; i < nb; i++) {
                        bits[i] = b0 + i;
                        rr[i] = lr[G.q0 + b0 - G.rb0 + i];
                    }
                    RAcc<R> gy[3]{};
                    if constexpr (NBM == 3) {
                        if (nb == 3) adj_round<R, 3>(tp, tl, T0, bits, rr, gy);
                        else if (nb == 2) adj_round<R, 2>(tp, tl, T0, bits, rr, gy);
                        else adj_round<R, 1>(tp, tl, T0, bits, rr, gy);
                    } else {
                        if (nb == 2) adj_round<R, 2>(tp, tl, T0, bits, rr, gy);
                        else adj_round<R, 1>(tp, tl, T0, bits, rr, gy);
                    }
                    flush_gy(gy, b0 - G.rb0, nb);
                    __syncthreads();
                }
            }
        }
        {
            const uint32_t s0 = sw<R>(threadIdx.x);
#pragma unroll
            for (int i = 0; i < IT; i++) {
                if (threadIdx.x + uint32_t(i) * kThreads >= sz) continue;
                const uint64_t x = ta.x0 + uint64_t(i) * ta.stride;
                psi[I.off + x] = (tp[s0 + uint32_t(i) * kThreads]);
                lam[I.off + x] = (tl[s0 + uint32_t(i) * kThreads]);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (cur >= 0) flush();
}

// rotation table from the parameters: rot[inst][layer][q]
template <typename R>
__global__ void k_hea_prep(const HeaInst *__restrict__ insts, int ninst, int layers,
                           const double *__restrict__ params, Rot<R> *__restrict__ rot) {
    const int id = blockIdx.x;
    if (id >= ninst) return;
    const HeaInst I = insts[id];
    for (int e = threadIdx.x; e < layers * I.n; e += blockDim.x) {
        const int l = e / I.n, q = e % I.n;
        const double th = params[I.param_off + 2 * I.n * l + q];
        const double ph = params[I.param_off + 2 * I.n * l + I.n + q];
        using Re = typename HT<R>::Real;
        Rot<R> r;
        r.cy = rfrom_d<Re>(cos(0.5 * th));
        r.sy = rfrom_d<Re>(sin(0.5 * th));
        r.cz = rfrom_d<Re>(cos(0.5 * ph));
        r.sz = rfrom_d<Re>(sin(0.5 * ph));
        rot[I.rot_off + e] = r;
    }
}

// every instance to |0...0>
template <typename R>
__global__ void k_hea_reset(typename HT<R>::Amp *__restrict__ arena, const HeaInst *__restrict__ insts, int ninst) {
    const int id = blockIdx.y;
    if (id >= ninst) return;
    const HeaInst I = insts[id];
    using Re = typename HT<R>::Real;
    const uint64_t N = uint64_t(1) << I.n;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += uint64_t(gridDim.x) * blockDim.x)
        arena[I.off + i] = make_amp(rfrom_i<Re>(i == 0 ? 1 : 0), rzero<Re>());
}

}  // namespace
}  // namespace cast

// ------------------------------------------------------------------- host
struct cast_hea {
    int ninst = 0, layers = 0, nparams = 0;
    cast_dtype dt = CAST_C64;
    bool with_grad = false;
    cudaStream_t stream = nullptr;
    std::vector<cast::HeaInst> inst;
    void *psi = nullptr, *lam = nullptr;  // arenas
    cast::HeaInst *d_inst = nullptr;
    void *d_rot = nullptr;
    double *d_params = nullptr, *d_out = nullptr;  // out: [ninst energies][nparams grads]
    double *h_params = nullptr, *h_out = nullptr;  // pinned
    int *d_pass_inst = nullptr;
    uint64_t *d_pass_prefix = nullptr;
    std::vector<int> pass_ninst;            // per group
    std::vector<size_t> pass_inst_off, pass_prefix_off;
    std::vector<uint64_t> pass_tiles;
    std::vector<char> pass_full;            // every tile of the pass is 2^T amplitudes
    int ngroups_max = 0;
    double zz = 0, hx = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};  // [energy][grad]
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    double graph_zz[2] = {0, 0}, graph_hx[2] = {0, 0};
    bool graph_df[2] = {false, false};  // complex128 graph built in double-float arithmetic
    int grid = 0;
};

namespace cast {
namespace {

template <typename R>
cast_status queue_hea(cast_hea *b, bool grad) {
    using T2 = typename HT<R>::Amp;  // 8 or 16 bytes per amplitude in the arena
    constexpr int T = tile_bits<R>();
    cudaStream_t st = b->stream;
    T2 *psi = static_cast<T2 *>(b->psi), *lam = static_cast<T2 *>(b->lam);
    Rot<R> *rot = static_cast<Rot<R> *>(b->d_rot);
    const int G = b->grid;
    auto pass = [&](int layer, int g) {
        PassArgs P;
        P.layer = layer;
        P.group = g;
        P.ninst = b->pass_ninst[g];
        P.inst = b->d_pass_inst + b->pass_inst_off[g];
        P.prefix = b->d_pass_prefix + b->pass_prefix_off[g];
        return P;
    };
    CAST_CUDA(cudaMemcpyAsync(b->d_params, b->h_params, sizeof(double) * b->nparams, cudaMemcpyHostToDevice, st));
    CAST_CUDA(cudaMemsetAsync(b->d_out, 0, sizeof(double) * (b->ninst + (grad ? b->nparams : 0)), st));
    k_hea_prep<R><<<b->ninst, 256, 0, st>>>(b->d_inst, b->ninst, b->layers, b->d_params, rot);
    k_hea_reset<R><<<dim3(64, b->ninst), 256, 0, st>>>(psi, b->d_inst, b->ninst);
    for (int l = 0; l < b->layers; l++)
        for (int g = 0; g < b->ngroups_max; g++) {
            if (b->pass_ninst[g] == 0) continue;
            ProfScope ps(st, std::string("hea_fwd_") + dt_name(b->dt), 2.0 * sizeof(T2) * double(b->pass_tiles[g] << T), 0);
            if (b->pass_full[g]) k_hea_forward<R, true><<<G, kThreads, 0, st>>>(psi, b->d_inst, rot, pass(l, g));
            else k_hea_forward<R, false><<<G, kThreads, 0, st>>>(psi, b->d_inst, rot, pass(l, g));
        }
    for (int g = 0; g < b->ngroups_max; g++) {
        if (b->pass_ninst[g] == 0) continue;
        ProfScope ps(st, std::string("hea_energy_") + dt_name(b->dt), sizeof(T2) * double(b->pass_tiles[g] << T), 0);
        if (b->pass_full[g]) k_hea_energy<R, true><<<G, kThreads, 0, st>>>(psi, b->d_inst, pass(0, g), b->zz, b->hx, b->d_out);
        else k_hea_energy<R, false><<<G, kThreads, 0, st>>>(psi, b->d_inst, pass(0, g), b->zz, b->hx, b->d_out);
    }
    if (grad) {
        constexpr bool SR = bwd_smem_ry<R>();
        CAST_CUDA(cudaFuncSetAttribute(k_hea_backward<R, SR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(2 * sizeof(T2) << T)));
        CAST_CUDA(cudaFuncSetAttribute(k_hea_backward<R, SR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(2 * sizeof(T2) << T)));
        for (int g = 0; g < b->ngroups_max; g++) {
            if (b->pass_ninst[g] == 0) continue;
            if (b->pass_full[g]) k_hea_lambda<R, true><<<G, kThreads, 0, st>>>(psi, lam, b->d_inst, pass(0, g), b->zz, b->hx);
            else k_hea_lambda<R, false><<<G, kThreads, 0, st>>>(psi, lam, b->d_inst, pass(0, g), b->zz, b->hx);
        }
        for (int l = b->layers - 1; l >= 0; l--)
            for (int g = b->ngroups_max - 1; g >= 0; g--) {
                if (b->pass_ninst[g] == 0) continue;
                ProfScope ps(st, std::string("hea_bwd_") + dt_name(b->dt),
                             4.0 * sizeof(T2) * double(b->pass_tiles[g] << T), 0);
                if (b->pass_full[g])
                    k_hea_backward<R, SR, true><<<G, kThreads, 2 * sizeof(T2) << T, st>>>(
                        psi, lam, b->d_inst, rot, pass(l, g), b->d_out + b->ninst);
                else
                    k_hea_backward<R, SR, false><<<G, kThreads, 2 * sizeof(T2) << T, st>>>(
                        psi, lam, b->d_inst, rot, pass(l, g), b->d_out + b->ninst);
            }
    }
    CAST_CUDA(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * (b->ninst + (grad ? b->nparams : 0)),
                              cudaMemcpyDeviceToHost, st));
    CAST_CUDA(cudaGetLastError());
    return CAST_OK;
}

void free_hea(cast_hea *b) {
    for (int i = 0; i < 2; i++) {
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
        if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
    }
    cudaFree(b->psi);
    cudaFree(b->lam);
    cudaFree(b->d_inst);
    cudaFree(b->d_rot);
    cudaFree(b->d_params);
    cudaFree(b->d_out);
    cudaFree(b->d_pass_inst);
    cudaFree(b->d_pass_prefix);
    cudaFreeHost(b->h_params);
    cudaFreeHost(b->h_out);
    delete b;
}

}  // namespace
}  // namespace cast

using namespace cast;

extern "C" {

cast_status cast_hea_create(int n_instances, const int32_t *n_qubits, int layers, cast_dtype dt, int with_grad,
                            void *cuda_stream, cast_hea **out) {
    if (!out) return fail(CAST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (n_instances < 1 || !n_qubits) return fail(CAST_ERR_ARG, "need at least one instance");
    if (layers < 1) return fail(CAST_ERR_ARG, "layers must be >= 1");
    if (dt != CAST_C64 && dt != CAST_C128) return fail(CAST_ERR_ARG, "unknown dtype");
    const int T = dt == CAST_C64 ? tile_bits<float>() : tile_bits<double>();
    cast_hea *b = new cast_hea();
    b->ninst = n_instances;
    b->layers = layers;
    b->dt = dt;
    b->with_grad = with_grad != 0;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t S = amp_bytes(dt);
    uint64_t off = 0;
    int poff = 0, roff = 0;
    for (int i = 0; i < n_instances; i++) {
        const int n = n_qubits[i];
        if (n < 2 || n > 30) {
            delete b;
            return fail(CAST_ERR_ARG, "instance qubit counts must be in 2..30");
        }
        HeaInst I;
        I.off = off;
        I.n = n;
        I.ngroups = group_count(n, T);
        I.param_off = poff;
        I.rot_off = roff;
        b->inst.push_back(I);
        off += (uint64_t(1) << n) + (256 / S);  // keep every state 256-byte aligned
        off = (off + 255) & ~uint64_t(255);
        poff += 2 * n * layers;
        roff += n * layers;
        b->ngroups_max = std::max(b->ngroups_max, I.ngroups);
    }
    if (b->ngroups_max > kMaxGroups) {
        delete b;
        return fail(CAST_ERR_UNSUPPORTED, "too many qubit groups");
    }
    b->nparams = poff;
    // per-group instance lists and tile prefix sums
    std::vector<int> all_inst;
    std::vector<uint64_t> all_prefix;
    b->pass_ninst.assign(b->ngroups_max, 0);
    b->pass_tiles.assign(b->ngroups_max, 0);
    b->pass_full.assign(b->ngroups_max, 1);
    for (int g = 0; g < b->ngroups_max; g++) {
        b->pass_inst_off.push_back(all_inst.size());
        b->pass_prefix_off.push_back(all_prefix.size());
        uint64_t acc = 0;
        for (int i = 0; i < n_instances; i++) {
            if (g >= b->inst[i].ngroups) continue;
            const Geo Gm = geometry(b->inst[i].n, g, T);
            if (Gm.T0 != T) b->pass_full[g] = 0;
            all_inst.push_back(i);
            all_prefix.push_back(acc);
            acc += uint64_t(1) << (b->inst[i].n - Gm.T0);
            b->pass_ninst[g]++;
        }
        all_prefix.push_back(acc);
        b->pass_tiles[g] = acc;
    }
    static_assert(sizeof(Rot<DF>) == sizeof(Rot<double>) && tile_bits<DF>() == tile_bits<double>(),
                  "one complex128 layout for both arithmetics");
    const size_t rot_bytes = (dt == CAST_C64 ? sizeof(Rot<float>) : sizeof(Rot<double>)) * size_t(roff);
    bool ok = cudaMalloc(&b->psi, off * S) == cudaSuccess;
    ok = ok && (!b->with_grad || cudaMalloc(&b->lam, off * S) == cudaSuccess);
    ok = ok && cudaMalloc(&b->d_inst, sizeof(HeaInst) * n_instances) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_rot, rot_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_params, sizeof(double) * b->nparams) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_out, sizeof(double) * (n_instances + b->nparams)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_pass_inst, sizeof(int) * all_inst.size()) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_pass_prefix, sizeof(uint64_t) * all_prefix.size()) == cudaSuccess;
    ok = ok && cudaMallocHost(&b->h_params, sizeof(double) * b->nparams) == cudaSuccess;
    ok = ok && cudaMallocHost(&b->h_out, sizeof(double) * (n_instances + b->nparams)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_hea(b);
        return fail(CAST_ERR_OOM, "batch allocation failed");
    }
    cudaError_t e = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(HeaInst) * n_instances, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pass_inst, all_inst.data(), sizeof(int) * all_inst.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pass_prefix, all_prefix.data(), sizeof(uint64_t) * all_prefix.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_hea(b);
        return cuda_fail(e, "batch upload");
    }
    b->grid = sm_count_cached() * (dt == CAST_C64 ? 6 : 6);
    *out = b;
    return CAST_OK;
}

static cast_status run_hea(cast_hea *b, const double *params, double zz, double hx, double *energies,
                           double *grads, bool grad) {
    if (!b || !params || !energies || (grad && !grads)) return fail(CAST_ERR_ARG, "null argument");
    if (grad && !b->with_grad) return fail(CAST_ERR_ARG, "batch was created without gradient buffers");
    if (!std::isfinite(zz) || !std::isfinite(hx)) return fail(CAST_ERR_ARG, "non-finite coefficient");
    for (int p = 0; p < b->nparams; p++)
        if (!std::isfinite(params[p])) return fail(CAST_ERR_ARG, "non-finite parameter");
    const int gi = grad ? 1 : 0;
    CAST_CUDA(cudaStreamSynchronize(b->stream));  // the pinned buffers are free
    std::memcpy(b->h_params, params, sizeof(double) * b->nparams);
    b->zz = zz;
    b->hx = hx;
    // the graph bakes in zz, hx and the complex128 arithmetic; rebuild it when they change
    const bool use_df = b->dt == CAST_C128 && f64_mode() == CAST_F64_EMULATED;
    if (b->exec[gi] && (b->graph_zz[gi] != zz || b->graph_hx[gi] != hx || b->graph_df[gi] != use_df)) {
        cudaGraphExecDestroy(b->exec[gi]);
        cudaGraphDestroy(b->graph[gi]);
        b->exec[gi] = nullptr;
        b->graph[gi] = nullptr;
    }
    if (!b->exec[gi]) {
        cudaStream_t cap = nullptr;
        CAST_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaStream_t orig = b->stream;
        b->stream = cap;
        cast_status st = CAST_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture");
        } else {
            st = b->dt == CAST_C64 ? queue_hea<float>(b, grad)
                 : use_df          ? queue_hea<DF>(b, grad)
                                   : queue_hea<double>(b, grad);
            cudaGraph_t gph = nullptr;
            cudaError_t e = cudaStreamEndCapture(cap, &gph);
            if (st == CAST_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture");
            if (st == CAST_OK) {
                e = cudaGraphInstantiate(&b->exec[gi], gph, 0);
                if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate");
                b->graph[gi] = gph;
                b->graph_zz[gi] = zz;
                b->graph_hx[gi] = hx;
                b->graph_df[gi] = use_df;
            } else if (gph) {
                cudaGraphDestroy(gph);
            }
        }
        b->stream = orig;
        cudaStreamDestroy(cap);
        if (st != CAST_OK) return st;
    }
    CAST_CUDA(cudaGraphLaunch(b->exec[gi], b->stream));
    CAST_CUDA(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->ninst; i++) energies[i] = b->h_out[i];
    if (grad)
        for (int p = 0; p < b->nparams; p++) grads[p] = b->h_out[b->ninst + p];
    return take_device_error();
}

cast_status cast_hea_energy(cast_hea *b, const double *params, double zz, double hx, double *energies) {
    return run_hea(b, params, zz, hx, energies, nullptr, false);
}

cast_status cast_hea_grad(cast_hea *b, const double *params, double zz, double hx, double *energies,
                          double *grads) {
    return run_hea(b, params, zz, hx, energies, grads, true);
}

cast_status cast_hea_info(const cast_hea *b, int *n_params, int *n_passes_per_layer_max) {
    if (!b) return fail(CAST_ERR_ARG, "null batch");
    if (n_params) *n_params = b->nparams;
    if (n_passes_per_layer_max) *n_passes_per_layer_max = b->ngroups_max;
    return CAST_OK;
}

cast_status cast_hea_destroy(cast_hea *b) {
    if (!b) return CAST_OK;
    cudaStreamSynchronize(b->stream);
    free_hea(b);
    return CAST_OK;
}

}  // extern "C"
