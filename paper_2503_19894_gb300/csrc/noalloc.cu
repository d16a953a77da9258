// cast_expectation_noalloc: the Pauli-sum expectation with its scratch in a
// fixed device array, for callers that cannot allocate memory.
//
// The per-block FP64 partial sums and the final value live in g_noalloc, a
// file-scope __device__ array of CAST_NOALLOC_SCRATCH_DOUBLES doubles that
// every GPU loading this library holds until the process exits.  Host code
// must not pass the symbol itself to a kernel (on the host it names a
// host-side stand-in); the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call there.
// That cached address belongs to the device's primary context: after
// cudaDeviceReset it is stale, and the call must not be used again in the
// process.
//
// Every call on a device shares the array.  Each call writes every partial
// sum it later reads, and the final value, before reading them, so nothing
// has to start at zero; but two calls whose work overlaps on the GPU (for
// example on two streams) race on the array and may return wrong values.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace cast {
namespace {

__device__ __align__(256) double g_noalloc[CAST_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc on device `dev` (which must be current).
cast_status scratch_address(int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(CAST_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc)");
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return CAST_OK;
}

}  // namespace
}  // namespace cast

using namespace cast;

extern "C" cast_status cast_expectation_noalloc(const cast_sv *sv, const cast_pauli_sum *h, double *out) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!out) return fail(CAST_ERR_ARG, "null output");
    cast_status st = check_pauli(h, sv->n);
    if (st != CAST_OK) return st;
    int dev = -1;
    CAST_CUDA(cudaGetDevice(&dev));
    if (dev != sv->device) return fail(CAST_ERR_ARG, "make the state's device current before this call");
    const PauliGroups G = group_terms(h);
    const size_t B = (size_t)reduce_grid_blocks();
    // slot 0: result; then one partial sum per block of every launch, counted
    // by the same helper that sizes cast_expectation's buffer
    const size_t partials = pauli_partials_needed(G);
    const size_t need = 1 + partials;
    if (need > CAST_NOALLOC_SCRATCH_DOUBLES)
        return fail(CAST_ERR_ARG, "Pauli sum needs " + std::to_string(need) + " scratch doubles (" +
                                      std::to_string(partials / B) + " launches x " + std::to_string(B) +
                                      " blocks + 1); the fixed scratch holds " +
                                      std::to_string(CAST_NOALLOC_SCRATCH_DOUBLES));
    if (partials == 0) {
        *out = 0.0;
        return CAST_OK;
    }
    double *base = nullptr;
    if ((st = scratch_address(dev, &base)) != CAST_OK) return st;
    double *part = base + 1;
    size_t used = 0;
    for (size_t g = 0; g < G.xm.size(); g++) {
        int np = 0;
        st = launch_pauli_group(sv, G.xm[g], (int)G.c[g].size(), G.c[g].data(), G.z[g].data(), part + used, &np);
        if (st != CAST_OK) return st;
        used += (size_t)np;
        if (used > partials) return fail(CAST_ERR_CUDA, "Pauli launches wrote more partial sums than counted");
    }
    if ((st = launch_finalize(sv->stream, part, (int)used, 1, base)) != CAST_OK) return st;
    CAST_CUDA(cudaMemcpyAsync(out, base, sizeof(double), cudaMemcpyDeviceToHost, sv->stream));
    CAST_CUDA(cudaStreamSynchronize(sv->stream));
    // a bounded wait that gave up in earlier work on this stream makes the
    // state, and so this value, unreliable: report it as cast_expectation does
    return take_device_error();
}
