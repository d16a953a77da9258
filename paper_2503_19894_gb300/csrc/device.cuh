// Device-side helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace cast {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

struct Targets {
    int q[CAST_MAX_K];  // sorted ascending
};

// Eq. 4: the base index of slice t is t with a zero bit inserted at each
// (ascending) target position.
template <int K>
__device__ __forceinline__ uint64_t slice_base(uint64_t t, const Targets &tg) {
#pragma unroll
    for (int i = 0; i < K; i++) {
        const int q = tg.q[i];
        const uint64_t low = t & ((uint64_t(1) << q) - 1);
        t = ((t >> q) << (q + 1)) | low;
    }
    return t;
}

// Offset of member j of a slice: 2^q[i] for every set bit i of j.
template <int K>
__device__ __forceinline__ uint64_t member_offset(int j, const Targets &tg) {
    uint64_t off = 0;
#pragma unroll
    for (int i = 0; i < K; i++) off |= uint64_t((j >> i) & 1) << tg.q[i];
    return off;
}

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// FP64-class accumulator.  double: plain FP64.  float: (hi, lo) pair updated
// with Knuth's TwoSum, so the running sum carries ~48 significant bits while
// using only FP32 instructions.
template <typename R> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float s = hi + v;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (v - bb);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in
// thread 0.  Uses 32 doubles of static shared memory.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

}  // namespace cast
