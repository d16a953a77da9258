// Autotuner: measured per-gate costs (the GPU counterpart of the paper's
// CostModel, Section IV-C) and the launch widths of the CUDA-core kernels.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace cast {

namespace {
std::mutex g_mu;
cast_cost_table g_tab[2];
bool g_have[2] = {false, false};

// DFT matrix (dense, unitary), a phase diagonal, a cyclic shift with phases
std::vector<cplx> sample_matrix(int k, int cls) {
    const int d = 1 << k;
    std::vector<cplx> m(size_t(d) * d, cplx(0.0, 0.0));
    for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) {
            if (cls == CLS_DENSE) m[size_t(r) * d + c] = std::polar(1.0 / std::sqrt(double(d)), 2 * M_PI * r * c / d);
            else if (cls == CLS_DIAG && r == c) m[size_t(r) * d + c] = std::polar(1.0, 0.7 + r);
            else if (cls == CLS_MONO && c == (r + 1) % d) m[size_t(r) * d + c] = std::polar(1.0, 0.3 + r);
        }
    return m;
}
// unitary with two entries per row: H on local bit 0, identity elsewhere
std::vector<cplx> two_per_row_matrix(int k) {
    const int d = 1 << k;
    std::vector<cplx> m(size_t(d) * d, cplx(0.0, 0.0));
    const double h = 1.0 / std::sqrt(2.0);
    for (int r = 0; r < d; r++) {
        m[size_t(r) * d + (r & ~1)] = cplx(h, 0.0);
        m[size_t(r) * d + (r | 1)] = cplx((r & 1) ? -h : h, 0.0);
    }
    return m;
}

// average ms of one launch of g (two warm-up launches, three timed)
cast_status time_gate(cast_sv *sv, const PreparedGate &g, cudaEvent_t e0, cudaEvent_t e1, double *per) {
    cast_status st = CAST_OK;
    for (int rep = 0; rep < 2 && st == CAST_OK; rep++) st = launch_gate(sv, g);
    if (st != CAST_OK) return st;
    cudaEventRecord(e0, sv->stream);
    const int reps = 3;
    for (int rep = 0; rep < reps && st == CAST_OK; rep++) st = launch_gate(sv, g);
    cudaEventRecord(e1, sv->stream);
    if (st != CAST_OK) return st;
    if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune timing");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    *per = double(ms) / reps;
    return CAST_OK;
}
}  // namespace

int tuned_blocks_per_sm(cast_dtype dt, int k, int cls, int def) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int i = dt == CAST_C64 ? 0 : 1;
    if (!g_have[i] || k < 1 || k > CAST_MAX_K || cls < 0 || cls > 3) return def;
    const int v = g_tab[i].blocks_per_sm[k][cls];
    return v > 0 ? v : def;
}

// cost-table estimate of a block (integer nanoseconds), used by the fusion pass
int64_t table_estimate(const cast_cost_table &t, int k, int cls, int64_t ops) {
    double ms = t.ms[k][cls];
    if (cls != CLS_IDENTITY && !(ms > 0)) ms = t.ms[k][CLS_DENSE];
    if (cls != CLS_IDENTITY && !(ms > 0)) {
        for (int kk = 1; kk <= CAST_MAX_K; kk++)
            for (int c = 1; c < 4; c++) ms = std::max(ms, t.ms[kk][c]);
    }
    if (cls == CLS_DENSE && k >= 3 && t.sparse_floor_ms[k] > 0 && t.sparse_ms_per_op[k] > 0) {
        const double sp = std::max(t.sparse_floor_ms[k], t.sparse_ms_per_op[k] * double(ops));
        ms = std::min(ms, sp);
    }
    return cls == CLS_IDENTITY ? 0 : int64_t(std::llround(ms * 1e6));
}

}  // namespace cast

using namespace cast;

extern "C" {

cast_status cast_set_cost_table(const cast_cost_table *t) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!t) {
        g_have[0] = g_have[1] = false;
        return CAST_OK;
    }
    if (t->dtype != CAST_C64 && t->dtype != CAST_C128) return fail(CAST_ERR_ARG, "cost table has an unknown dtype");
    const int i = t->dtype == CAST_C64 ? 0 : 1;
    g_tab[i] = *t;
    g_have[i] = true;
    return CAST_OK;
}

cast_status cast_autotune(cast_dtype dt, int n, void *stream, cast_cost_table *out) {
    if (!out) return fail(CAST_ERR_ARG, "null output table");
    if (dt != CAST_C64 && dt != CAST_C128) return fail(CAST_ERR_ARG, "unknown dtype");
    if (n < CAST_MAX_K + 1 || n > 30) return fail(CAST_ERR_ARG, "autotune state size must be in 8..30 qubits");
    cast_sv *sv = nullptr;
    cast_status st = cast_sv_create(n, dt, stream, &sv);
    if (st != CAST_OK) return st;
    // time on a state with every amplitude non-zero: the complex128 kernels
    // skip work on zero values (a 2-qubit double-float gate ran 7.7 ms on
    // |0...0> and 13.2 ms on a random 30-qubit state)
    if ((st = launch_fill_random(sv, 0x5eedu)) != CAST_OK) {
        cast_sv_destroy(sv);
        return st;
    }
    std::memset(out, 0, sizeof(*out));
    out->n_qubits = n;
    out->dtype = dt;
    const int ti = dt == CAST_C64 ? 0 : 1;
    cast_cost_table saved_tab;
    bool saved_have;
    {  // the process-wide table is borrowed for the trial widths and restored below
        std::lock_guard<std::mutex> lk(g_mu);
        saved_tab = g_tab[ti];
        saved_have = g_have[ti];
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int widths[4] = {1, 2, 4, 8};
    for (int k = 1; k <= CAST_MAX_K && st == CAST_OK; k++) {
        int qs[CAST_MAX_K];
        for (int i = 0; i < k; i++) qs[i] = k == 1 ? n / 2 : int(std::lround(double(i) * (n - 1) / (k - 1)));
        for (int cls = CLS_DIAG; cls <= CLS_DENSE && st == CAST_OK; cls++) {
            std::vector<cplx> m = sample_matrix(k, cls);
            PreparedGate g;
            if ((st = prepare_gate(n, qs, k, m.data(), 1e-12, &g)) != CAST_OK) break;
            double best = 0;
            int best_w = 0;
            for (int wi = 0; wi < 4 && st == CAST_OK; wi++) {
                {  // try this width through the process-wide table
                    std::lock_guard<std::mutex> lk(g_mu);
                    cast_cost_table t = *out;
                    t.dtype = dt;
                    t.blocks_per_sm[k][cls] = widths[wi];
                    g_tab[ti] = t;
                    g_have[ti] = true;
                }
                for (int rep = 0; rep < 2 && st == CAST_OK; rep++) st = launch_gate(sv, g);  // warm-up
                if (st != CAST_OK) break;
                cudaEventRecord(e0, sv->stream);
                const int reps = 3;
                for (int rep = 0; rep < reps && st == CAST_OK; rep++) st = launch_gate(sv, g);
                cudaEventRecord(e1, sv->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "autotune timing");
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                const double per = double(ms) / reps;
                if (best_w == 0 || per < best) {
                    best = per;
                    best_w = widths[wi];
                }
            }
            out->ms[k][cls] = best;
            out->blocks_per_sm[k][cls] = best_w;
        }
    }
    // the sparse kernel (k = 3..7): its floor with two entries per row, and
    // its time per operation with the dense sample
    const int sparse_saved = cast_get_sparse_mode();
    if (n >= 12) cast_set_sparse_mode(CAST_SPARSE_ALWAYS);
    for (int k = 3; k <= CAST_MAX_K && st == CAST_OK && n >= 12; k++) {
        int qs[CAST_MAX_K];
        for (int i = 0; i < k; i++) qs[i] = int(std::lround(double(i) * (n - 1) / (k - 1)));
        for (int which = 0; which < 2 && st == CAST_OK; which++) {
            std::vector<cplx> m = which == 0 ? two_per_row_matrix(k) : sample_matrix(k, CLS_DENSE);
            PreparedGate g;
            if ((st = prepare_gate(n, qs, k, m.data(), 1e-12, &g)) != CAST_OK) break;
            if (!sparse_preferred(sv, g)) break;  // e.g. complex128 in native FP64 mode
            double per = 0;
            if ((st = time_gate(sv, g, e0, e1, &per)) != CAST_OK) break;
            if (which == 0) out->sparse_floor_ms[k] = per;
            else out->sparse_ms_per_op[k] = per / double(opcount(g.m.data(), k, 0.0));
        }
    }
    cast_set_sparse_mode(sparse_saved);
    {  // leave the process-wide table as it was before the call
        std::lock_guard<std::mutex> lk(g_mu);
        g_tab[ti] = saved_tab;
        g_have[ti] = saved_have;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cast_status st2 = cast_sv_destroy(sv);
    return st != CAST_OK ? st : st2;
}

}  // extern "C"
