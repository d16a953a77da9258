// Tensor-pipe peak of this GPU, measured: one CTA per SM issues a long run of
// back-to-back tcgen05.mma instructions (M = 128, N = 256, operands in shared
// memory, one fp32 accumulator in TMEM) and the launch is timed with CUDA
// events.  The figure is the denominator of the tensor-core kernels'
// utilisation (executed MMA flops / time / this peak); it is measured rather
// than derived from a nominal ratio between data types.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace cast {
namespace {

constexpr int kPeakM = 128, kPeakN = 256;
constexpr uint32_t kPeakWait = 1u << 26;

__device__ int g_peak_error = 0;

// kind 0: kind::tf32 (K = 8 per instruction), kind 1: kind::f16 with bf16
// operands (K = 16); both read 32 bytes of K per row per instruction.
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_tensor_peak(int iters) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;                          // 128 rows x 128 bytes
    uint8_t *sB = sA + kPeakM * 128;             // 256 rows x 128 bytes
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + kPeakN * 128);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (kPeakM + kPeakN) * 128 / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(sA)[i] = 0u;  // zero operands: the pipe's rate does not depend on values
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, kPeakN);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    bool ok = true;
    if (tid == 0) {
        const uint32_t a = tc::smem_u32(sA), b = tc::smem_u32(sB);
        uint32_t idesc;
        if (KIND == 0) idesc = tc::idesc_tf32(kPeakM, kPeakN);
        else idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kPeakN >> 3) << 17) | (uint32_t(kPeakM >> 4) << 24);
        uint32_t acc = 0;
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint64_t da = tc::smem_desc_sw128(a + 32 * s), db = tc::smem_desc_sw128(b + 32 * s);
                if (KIND == 0) {
                    tc::mma_tf32(taddr, da, db, idesc, acc);
                } else {
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
                acc = 1;
            }
        }
        tc::mma_commit(mbar);
        ok = tc::mbar_wait(mbar, 0, kPeakWait);
        if (!ok) {
            atomicOr(&g_peak_error, 1);
            tc::mbar_wait(mbar, 0, kPeakWait);  // give an MMA in flight time before TMEM is freed
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, kPeakN);
}

template <int KIND>
cast_status time_peak(int iters, double *ms) {
    const size_t smem = 1024 + (kPeakM + kPeakN) * 128 + 64 + 120 * 1024;  // > half of an SM: one CTA each
    CAST_CUDA(cudaFuncSetAttribute(k_tensor_peak<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaStream_t s = nullptr;
    CAST_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sm_count_cached();
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; rep++) {  // the first launch is a warm-up
        cudaEventRecord(e0, s);
        k_tensor_peak<KIND><<<grid, 128, smem, s>>>(iters);
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float t = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) best = std::min(best, t);
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (err != cudaSuccess) return cuda_fail(err, "tensor peak kernel");
    int flag = 0;
    CAST_CUDA(cudaMemcpyFromSymbol(&flag, g_peak_error, sizeof(int)));
    if (flag) {
        const int zero = 0;
        CAST_CUDA(cudaMemcpyToSymbol(g_peak_error, &zero, sizeof(int)));
        return fail(CAST_ERR_TIMEOUT, "tensor peak kernel gave up waiting for its MMAs (bounded wait)");
    }
    *ms = best;
    return CAST_OK;
}

// Issue cost of small MMAs: thread 0 of one CTA per SM issues `iters`
// back-to-back tcgen05.mma kind::f16 (M = 128, K = 16, N = n, bf16 zero
// operands, A from TMEM columns 256..263 or from shared memory, one fp32
// accumulator at column 0) and measures the SM clock from the first issue to
// the commit's completion.
template <bool ATMEM>
__global__ void __launch_bounds__(128, 1) k_mma_issue(int n, int iters, long long *cycles) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;                          // 128 rows x 128 bytes
    uint8_t *sB = sA + kPeakM * 128;             // 256 rows x 128 bytes
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + kPeakN * 128);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (kPeakM + kPeakN) * 128 / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sA)[i] = 0u;
    if (tid == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *tslot;
    if (ATMEM) {  // zero A in TMEM, columns 256..263 of every lane
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        tc::tmem_st<8>(taddr + (uint32_t(32 * warp) << 16) + 256u, z);
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kPeakM >> 4) << 24);
        const uint64_t da = tc::smem_desc_sw128(tc::smem_u32(sA)), db = tc::smem_desc_sw128(tc::smem_u32(sB));
        const long long t0 = clock64();
        for (int it = 0; it < iters; it++) {
            if (ATMEM) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(taddr),
                    "r"(taddr + 256u), "l"(db), "r"(idesc), "r"(1));
            } else {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                    "l"(da), "l"(db), "r"(idesc), "r"(1));
            }
        }
        tc::mma_commit(mbar);
        if (tc::mbar_wait(mbar, 0, kPeakWait)) {
            cycles[blockIdx.x] = clock64() - t0;
        } else {
            atomicOr(&g_peak_error, 1);
            cycles[blockIdx.x] = -1;
            tc::mbar_wait(mbar, 0, kPeakWait);  // give an MMA in flight time before TMEM is freed
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

template <bool ATMEM>
cast_status time_mma_issue(int n, int iters, double *cycles_per_mma) {
    const size_t smem = 1024 + (kPeakM + kPeakN) * 128 + 64 + 120 * 1024;  // > half of an SM: one CTA each
    CAST_CUDA(cudaFuncSetAttribute(k_mma_issue<ATMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = sm_count_cached();
    long long *d = nullptr;
    CAST_CUDA(cudaMalloc(&d, sizeof(long long) * grid));
    std::vector<long long> h(grid, 0);
    cudaError_t err = cudaSuccess;
    double best = 1e300;
    for (int rep = 0; rep < 3 && err == cudaSuccess; rep++) {  // the first launch is a warm-up
        k_mma_issue<ATMEM><<<grid, 128, smem>>>(n, iters, d);
        err = cudaDeviceSynchronize();
        if (err == cudaSuccess) err = cudaMemcpy(h.data(), d, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
        if (err == cudaSuccess && rep > 0) {
            double sum = 0;
            for (long long c : h) sum += double(c);
            best = std::min(best, sum / grid / iters);
        }
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaFree(d);
    if (err != cudaSuccess) return cuda_fail(err, "MMA issue kernel");
    int flag = 0;
    CAST_CUDA(cudaMemcpyFromSymbol(&flag, g_peak_error, sizeof(int)));
    if (flag) {
        const int zero = 0;
        CAST_CUDA(cudaMemcpyToSymbol(g_peak_error, &zero, sizeof(int)));
        return fail(CAST_ERR_TIMEOUT, "MMA issue kernel gave up waiting for its MMAs (bounded wait)");
    }
    *cycles_per_mma = best;
    return CAST_OK;
}

}  // namespace
}  // namespace cast

using namespace cast;

extern "C" cast_status cast_measure_mma_issue(int n_cols, int a_in_tmem, double *cycles_per_mma) {
    if (!cycles_per_mma) return fail(CAST_ERR_ARG, "null output");
    if (n_cols < 16 || n_cols > 256 || n_cols % 16 != 0) return fail(CAST_ERR_ARG, "N must be 16..256, a multiple of 16");
    const int iters = 8192;
    return a_in_tmem ? time_mma_issue<true>(n_cols, iters, cycles_per_mma)
                     : time_mma_issue<false>(n_cols, iters, cycles_per_mma);
}

extern "C" cast_status cast_measure_tensor_peak(int kind, double *tflops) {
    if (!tflops) return fail(CAST_ERR_ARG, "null output");
    if (kind != CAST_PEAK_TF32 && kind != CAST_PEAK_BF16) return fail(CAST_ERR_ARG, "unknown MMA kind");
    const int iters = 8192;  // 32768 MMAs per SM, ~2-5 ms per launch
    double ms = 0;
    cast_status st = kind == CAST_PEAK_TF32 ? time_peak<0>(iters, &ms) : time_peak<1>(iters, &ms);
    if (st != CAST_OK) return st;
    const double kdim = kind == CAST_PEAK_TF32 ? 8.0 : 16.0;
    const double flops = 2.0 * kPeakM * kPeakN * kdim * 4.0 * iters * double(sm_count_cached());
    *tflops = flops / (ms * 1e-3) / 1e12;
    return CAST_OK;
}
