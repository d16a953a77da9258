// Launch profiling: a pair of CUDA events recorded on the launch stream around
// every kernel while profiling is on; durations are aggregated per kernel
// family when profiling stops.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>

#include "internal.h"

namespace cast {

namespace {
struct Rec {
    cudaEvent_t a, b;
    std::string fam;
    double bytes, flops;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

ProfScope::ProfScope(cudaStream_t s, const std::string &family, double bytes, double flops) {
    if (!g_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return;
    cudaEventRecord(a, s);
    active_ = true;
    stream_ = s;
    a_ = a;
    b_ = b;
    fam_ = family;
    bytes_ = bytes;
    flops_ = flops;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    cudaEventRecord(b_, stream_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back(Rec{a_, b_, fam_, bytes_, flops_});
}

}  // namespace cast

using namespace cast;

extern "C" {

cast_status cast_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (Rec &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_on = true;
    return CAST_OK;
}

cast_status cast_profile_end(cast_profile_entry *out, int *n_out) {
    if (!n_out) return fail(CAST_ERR_ARG, "null count");
    g_on = false;
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, cast_profile_entry> agg;
    for (Rec &r : g_recs) {
        CAST_CUDA(cudaEventSynchronize(r.b));
        float ms = 0.f;
        CAST_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        cast_profile_entry &e = agg[r.fam];
        std::strncpy(e.name, r.fam.c_str(), sizeof(e.name) - 1);
        e.launches += 1;
        e.ms += ms;
        e.bytes += r.bytes;
        e.flops += r.flops;
    }
    std::vector<cast_profile_entry> v;
    for (auto &kv : agg) v.push_back(kv.second);
    std::sort(v.begin(), v.end(), [](const cast_profile_entry &x, const cast_profile_entry &y) { return x.ms > y.ms; });
    const int cap = *n_out;
    *n_out = (int)v.size();
    if ((int)v.size() > cap) return fail(CAST_ERR_ARG, "profile output capacity too small");
    for (size_t i = 0; i < v.size(); i++) out[i] = v[i];
    return CAST_OK;
}

}  // extern "C"
