// C ABI of the engine: state lifecycle, argument validation, dispatch of
// prepared gates to the kernels, expectation values and the adjoint driver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>

#include "internal.h"

namespace cast {

namespace {
thread_local std::string g_err;

bool valid_dt(cast_dtype dt) { return dt == CAST_C64 || dt == CAST_C128; }

// grow-only device scratch, allocated in stream order
cast_status ensure_dev(cast_sv *sv, DeviceScratch &s, size_t bytes) {
    if (s.bytes >= bytes) return CAST_OK;
    if (s.ptr) {
        CAST_CUDA(cudaFreeAsync(s.ptr, sv->stream));
        s.ptr = nullptr;
        s.bytes = 0;
    }
    cudaError_t e = cudaMallocAsync(&s.ptr, bytes, sv->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s.ptr = nullptr;
        return fail(CAST_ERR_OOM, "device scratch allocation failed");
    }
    s.bytes = bytes;
    return CAST_OK;
}

cast_status ensure_pinned(cast_sv *sv, size_t bytes) {
    if (sv->host_pinned_bytes >= bytes) return CAST_OK;
    if (sv->host_pinned) {
        CAST_CUDA(cudaStreamSynchronize(sv->stream));
        cudaFreeHost(sv->host_pinned);
        sv->host_pinned = nullptr;
        sv->host_pinned_bytes = 0;
    }
    if (cudaMallocHost(&sv->host_pinned, bytes) != cudaSuccess) {
        cudaGetLastError();
        sv->host_pinned = nullptr;
        return fail(CAST_ERR_OOM, "pinned host allocation failed");
    }
    sv->host_pinned_bytes = bytes;
    return CAST_OK;
}

cast_status ensure_gate_buffers(cast_sv *sv, int k) {
    if (k < 6 || sv->mat_dev) return CAST_OK;
    const size_t bytes = kMatSlotBytes * kMatSlots;
    if (cudaMalloc(&sv->mat_dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        sv->mat_dev = nullptr;
        return fail(CAST_ERR_OOM, "matrix ring allocation failed");
    }
    if (cudaMallocHost(&sv->mat_pinned, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sv->mat_dev);
        sv->mat_dev = nullptr;
        sv->mat_pinned = nullptr;
        return fail(CAST_ERR_OOM, "pinned matrix staging allocation failed");
    }
    for (int s = 0; s < kMatSlots; s++) CAST_CUDA(cudaEventCreateWithFlags(&sv->mat_events[s], cudaEventDisableTiming));
    return CAST_OK;
}

cast_status apply_prepared(cast_sv *sv, const PreparedGate &g) {
    cast_status st = ensure_gate_buffers(sv, g.k);
    if (st != CAST_OK) return st;
    return launch_gate(sv, g);
}

}  // namespace

cast_status upload_matrix(cast_sv *sv, const void *host, size_t bytes, const void **dev) {
    if (bytes > kMatSlotBytes) return fail(CAST_ERR_ARG, "matrix larger than a ring slot");
    cast_status st = ensure_gate_buffers(sv, CAST_MAX_K);
    if (st != CAST_OK) return st;
    const int s = sv->mat_next;
    sv->mat_next = (s + 1) % kMatSlots;
    CAST_CUDA(cudaEventSynchronize(sv->mat_events[s]));  // the slot's previous copy has completed
    char *hp = static_cast<char *>(sv->mat_pinned) + size_t(s) * kMatSlotBytes;
    char *dp = static_cast<char *>(sv->mat_dev) + size_t(s) * kMatSlotBytes;
    std::memcpy(hp, host, bytes);
    // stream order puts this copy after every kernel that read the slot before
    CAST_CUDA(cudaMemcpyAsync(dp, hp, bytes, cudaMemcpyHostToDevice, sv->stream));
    CAST_CUDA(cudaEventRecord(sv->mat_events[s], sv->stream));
    *dev = dp;
    return CAST_OK;
}

cast_status ensure_work(cast_sv *sv, size_t bytes, void **ptr) {
    cast_status st = ensure_dev(sv, sv->work, bytes);
    if (st != CAST_OK) return st;
    *ptr = sv->work.ptr;
    return CAST_OK;
}

cast_status check_sv(const cast_sv *sv) {
    if (!sv || !sv->data) return fail(CAST_ERR_ARG, "null state");
    return CAST_OK;
}

cast_status check_circuit(const cast_circuit *c, int n, const double *params) {
    if (!c) return fail(CAST_ERR_ARG, "null circuit");
    if (c->n_qubits != n) return fail(CAST_ERR_ARG, "circuit qubit count differs from the state's");
    if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) return fail(CAST_ERR_ARG, "bad gate list");
    if (c->n_params < 0 || (c->n_params > 0 && !params)) return fail(CAST_ERR_ARG, "missing parameter array");
    for (int g = 0; g < c->n_gates; g++) {
        const cast_gate &gt = c->gates[g];
        if (gt.k < 1 || gt.k > CAST_MAX_K || gt.k > n) return fail(CAST_ERR_ARG, "gate size out of range");
        if (gt.kind != CAST_GATE_MATRIX && gate_table_arity(gt.kind) != gt.k)
            return fail(CAST_ERR_ARG, "gate kind/arity mismatch");
        uint64_t seen = 0;
        for (int i = 0; i < gt.k; i++) {
            const int q = gt.qubits[i];
            if (q < 0 || q >= n) return fail(CAST_ERR_ARG, "qubit index out of range");
            if (seen & (uint64_t(1) << q)) return fail(CAST_ERR_ARG, "duplicate qubit in gate");
            seen |= uint64_t(1) << q;
        }
        if (gt.param_index >= c->n_params) return fail(CAST_ERR_ARG, "param_index outside the parameter array");
    }
    return CAST_OK;
}

cast_status check_pauli(const cast_pauli_sum *h, int n) {
    if (!h || h->n_terms < 0) return fail(CAST_ERR_ARG, "null Pauli sum");
    if (h->n_terms > 0 && (!h->coeffs || !h->x_masks || !h->z_masks))
        return fail(CAST_ERR_ARG, "null Pauli-sum arrays");
    const uint64_t lim = n >= 64 ? ~uint64_t(0) : (uint64_t(1) << n) - 1;
    for (int t = 0; t < h->n_terms; t++) {
        if ((h->x_masks[t] | h->z_masks[t]) & ~lim) return fail(CAST_ERR_ARG, "Pauli mask names a qubit >= n");
        if (!std::isfinite(h->coeffs[t])) return fail(CAST_ERR_ARG, "non-finite Pauli coefficient");
    }
    return CAST_OK;
}

// terms grouped by x_mask, in ascending mask order (deterministic)
PauliGroups group_terms(const cast_pauli_sum *h) {
    std::map<uint64_t, size_t> at;
    PauliGroups G;
    std::vector<uint64_t> keys;
    for (int t = 0; t < h->n_terms; t++) keys.push_back(h->x_masks[t]);
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (uint64_t k : keys) {
        at[k] = G.xm.size();
        G.xm.push_back(k);
        G.c.emplace_back();
        G.z.emplace_back();
    }
    for (int t = 0; t < h->n_terms; t++) {
        size_t g = at[h->x_masks[t]];
        G.c[g].push_back(h->coeffs[t]);
        G.z[g].push_back(h->z_masks[t]);
    }
    return G;
}

namespace {

// The first kResultSlots doubles of the partials buffer hold final results.
constexpr size_t kResultSlots = 16;

// Queue <psi|H|psi> into the first result slot of sv->partials.
cast_status queue_expectation(cast_sv *sv, const cast_pauli_sum *h) {
    PauliGroups G = group_terms(h);
    const size_t need = pauli_partials_needed(G);
    if (need == 0) {
        cast_status st = ensure_dev(sv, sv->partials, 4096 * sizeof(double));
        if (st != CAST_OK) return st;
        CAST_CUDA(cudaMemsetAsync(sv->partials.ptr, 0, sizeof(double), sv->stream));
        return CAST_OK;
    }
    cast_status st = ensure_dev(sv, sv->partials, (need + kResultSlots) * sizeof(double));
    if (st != CAST_OK) return st;
    double *part = reinterpret_cast<double *>(sv->partials.ptr) + kResultSlots;
    size_t used = 0;
    for (size_t g = 0; g < G.xm.size(); g++) {
        int np = 0;
        st = launch_pauli_group(sv, G.xm[g], (int)G.c[g].size(), G.c[g].data(), G.z[g].data(), part + used, &np);
        if (st != CAST_OK) return st;
        used += np;
    }
    return launch_finalize(sv->stream, part, (int)used, 1, reinterpret_cast<double *>(sv->partials.ptr));
}

}  // namespace

void set_error(const std::string &msg) { g_err = msg; }
cast_status fail(cast_status st, const std::string &msg) {
    g_err = msg;
    return st;
}
cast_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CAST_ERR_OOM : CAST_ERR_CUDA;
}

}  // namespace cast

using namespace cast;

extern "C" {

const char *cast_last_error(void) { return g_err.c_str(); }
const char *cast_version(void) { return "cast-gb300 0.1 (sm_103a)"; }

void cast_options_default(cast_options *o) {
    if (!o) return;
    o->fusion = CAST_FUSE_ADAPTIVE;
    o->max_k = 5;
    o->agglomerative = 1;
    o->op_cap = 4096;
    o->zero_tol = 1e-12;
    o->amp_ops_per_pass = 0;
    o->cost = nullptr;
}

int64_t cast_opcount(const double *matrix, int k, double zero_tol) {
    if (!matrix || k < 1 || k > CAST_MAX_K) return -1;
    std::vector<cplx> m(size_t(1) << (2 * k));
    for (size_t i = 0; i < m.size(); i++) m[i] = cplx(matrix[2 * i], matrix[2 * i + 1]);
    return opcount(m.data(), k, zero_tol);
}

cast_status cast_sv_set_basis(cast_sv *sv, uint64_t index) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (index >= (uint64_t(1) << sv->n)) return fail(CAST_ERR_ARG, "basis index >= 2^n");
    CAST_CUDA(cudaMemsetAsync(sv->data, 0, amp_bytes(sv->dt) << sv->n, sv->stream));
    return launch_set_one(sv, index);
}

static cast_status new_handle(int n, cast_dtype dt, void *stream, cast_sv **out) {
    if (!out) return fail(CAST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (n < 1 || n > CAST_MAX_QUBITS) return fail(CAST_ERR_ARG, "n_qubits must be in 1..34");
    if (!valid_dt(dt)) return fail(CAST_ERR_ARG, "unknown dtype");
    cast_sv *sv = new cast_sv();
    sv->n = n;
    sv->dt = dt;
    sv->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&sv->device);
    *out = sv;
    return CAST_OK;
}

cast_status cast_sv_create(int n_qubits, cast_dtype dt, void *cuda_stream, cast_sv **out) {
    cast_status st = new_handle(n_qubits, dt, cuda_stream, out);
    if (st != CAST_OK) return st;
    cast_sv *sv = *out;
    const size_t bytes = amp_bytes(dt) << n_qubits;
    cudaError_t e = cudaMalloc(&sv->data, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        *out = nullptr;
        return fail(CAST_ERR_OOM, "state allocation of " + std::to_string(bytes) + " bytes failed");
    }
    sv->owned = true;
    st = cast_sv_set_basis(sv, 0);
    if (st != CAST_OK) {
        cudaFree(sv->data);
        delete sv;
        *out = nullptr;
    }
    return st;
}

cast_status cast_sv_wrap(void *device_ptr, int n_qubits, cast_dtype dt, void *cuda_stream, cast_sv **out) {
    if (!device_ptr) return fail(CAST_ERR_ARG, "null device pointer");
    if (reinterpret_cast<uintptr_t>(device_ptr) % 256 != 0)
        return fail(CAST_ERR_ARG, "device pointer must be 256-byte aligned");
    cast_status st = new_handle(n_qubits, dt, cuda_stream, out);
    if (st != CAST_OK) return st;
    (*out)->data = device_ptr;
    (*out)->owned = false;
    return CAST_OK;
}

cast_status cast_sv_destroy(cast_sv *sv) {
    if (!sv) return CAST_OK;
    if (sv->partials.ptr) cudaFreeAsync(sv->partials.ptr, sv->stream);
    if (sv->work.ptr) cudaFreeAsync(sv->work.ptr, sv->stream);
    cudaError_t e = cudaStreamSynchronize(sv->stream);
    if (sv->mat_dev) cudaFree(sv->mat_dev);
    if (sv->mat_pinned) cudaFreeHost(sv->mat_pinned);
    for (int s = 0; s < kMatSlots; s++)
        if (sv->mat_events[s]) cudaEventDestroy(sv->mat_events[s]);
    if (sv->host_pinned) cudaFreeHost(sv->host_pinned);
    if (sv->owned && sv->data) cudaFree(sv->data);
    delete sv;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return CAST_OK;
}

cast_status cast_sv_info(const cast_sv *sv, int *n_qubits, cast_dtype *dt, void **device_ptr) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (n_qubits) *n_qubits = sv->n;
    if (dt) *dt = sv->dt;
    if (device_ptr) *device_ptr = sv->data;
    return CAST_OK;
}

cast_status cast_sv_copy_to_host(const cast_sv *sv, void *host) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!host) return fail(CAST_ERR_ARG, "null host buffer");
    CAST_CUDA(cudaMemcpyAsync(host, sv->data, amp_bytes(sv->dt) << sv->n, cudaMemcpyDeviceToHost, sv->stream));
    CAST_CUDA(cudaStreamSynchronize(sv->stream));
    return take_device_error();
}

cast_status cast_sv_copy_from_host(cast_sv *sv, const void *host) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!host) return fail(CAST_ERR_ARG, "null host buffer");
    CAST_CUDA(cudaMemcpyAsync(sv->data, host, amp_bytes(sv->dt) << sv->n, cudaMemcpyHostToDevice, sv->stream));
    CAST_CUDA(cudaStreamSynchronize(sv->stream));
    return CAST_OK;
}

cast_status cast_sv_copy_from_host_async(cast_sv *sv, const void *host) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!host) return fail(CAST_ERR_ARG, "null host buffer");
    CAST_CUDA(cudaMemcpyAsync(sv->data, host, amp_bytes(sv->dt) << sv->n, cudaMemcpyHostToDevice, sv->stream));
    return CAST_OK;
}

static cast_options resolve_options(const cast_options *opt, cast_dtype dt) {
    cast_options o;
    if (opt)
        o = *opt;
    else
        cast_options_default(&o);
    if (o.amp_ops_per_pass == 0) o.amp_ops_per_pass = (int32_t)default_amp_ops_per_pass(dt);
    return o;
}

static cast_status check_options(const cast_options &o) {
    if (o.fusion < CAST_FUSE_NONE || o.fusion > CAST_FUSE_ADAPTIVE) return fail(CAST_ERR_ARG, "unknown fusion mode");
    if (o.max_k < (o.cost ? 0 : 1) || o.max_k > CAST_MAX_K)
        return fail(CAST_ERR_ARG, "max_k must be in 1..7 (0 = chosen from a cost table)");
    if (!(o.zero_tol >= 0.0) || !std::isfinite(o.zero_tol)) return fail(CAST_ERR_ARG, "bad zero_tol");
    if (o.op_cap < 0) return fail(CAST_ERR_ARG, "op_cap must be >= 0");
    if (o.amp_ops_per_pass < 0) return fail(CAST_ERR_ARG, "amp_ops_per_pass must be >= 0 (0 = default)");
    if (o.agglomerative != 0 && o.agglomerative != 1) return fail(CAST_ERR_ARG, "agglomerative must be 0 or 1");
    return CAST_OK;
}

cast_status cast_gate_path(int n_qubits, cast_dtype dt, const int *qubits, int k, const double *matrix,
                           int *path) {
    if (!qubits || !matrix || !path) return fail(CAST_ERR_ARG, "null qubits, matrix or output");
    if (n_qubits < 1 || n_qubits > CAST_MAX_QUBITS) return fail(CAST_ERR_ARG, "n_qubits out of range");
    if (dt != CAST_C64 && dt != CAST_C128) return fail(CAST_ERR_ARG, "unknown dtype");
    if (k < 1 || k > CAST_MAX_K) return fail(CAST_ERR_ARG, "gate size k must be in 1..7");
    std::vector<cplx> m(size_t(1) << (2 * k));
    for (size_t i = 0; i < m.size(); i++) m[i] = cplx(matrix[2 * i], matrix[2 * i + 1]);
    PreparedGate g;
    cast_status st = prepare_gate(n_qubits, qubits, k, m.data(), 1e-12, &g);
    if (st != CAST_OK) return st;
    cast_sv shape;  // only the qubit count and type are read
    shape.n = n_qubits;
    shape.dt = dt;
    *path = choose_path(&shape, g);
    return CAST_OK;
}

cast_status cast_apply_gate(cast_sv *sv, const int *qubits, int k, const double *matrix) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!qubits || !matrix) return fail(CAST_ERR_ARG, "null qubits or matrix");
    if (k < 1 || k > CAST_MAX_K) return fail(CAST_ERR_ARG, "gate size k must be in 1..7");
    std::vector<cplx> m(size_t(1) << (2 * k));
    for (size_t i = 0; i < m.size(); i++) m[i] = cplx(matrix[2 * i], matrix[2 * i + 1]);
    PreparedGate g;
    cast_status st = prepare_gate(sv->n, qubits, k, m.data(), 1e-12, &g);
    if (st != CAST_OK) return st;
    return apply_prepared(sv, g);
}

// fuse (unless disabled) and prepare every gate of a circuit, host only
static cast_status prepare_circuit(const cast_circuit *c, const double *params, const cast_options &o,
                                   std::vector<PreparedGate> *prepared) {
    cast_status st;
    prepared->clear();
    if (o.fusion == CAST_FUSE_NONE) {
        prepared->resize(c->n_gates);
        for (int g = 0; g < c->n_gates; g++) {
            std::vector<cplx> m;
            if ((st = gate_matrix_of(c->gates[g], params, c->n_params, &m)) != CAST_OK) return st;
            if ((st = prepare_gate(c->n_qubits, c->gates[g].qubits, c->gates[g].k, m.data(), o.zero_tol,
                                   &(*prepared)[g])) != CAST_OK)
                return st;
        }
        return CAST_OK;
    }
    std::vector<FusedGate> fused;
    if ((st = fuse_circuit(c, params, &o, &fused)) != CAST_OK) return st;
    prepared->resize(fused.size());
    for (size_t g = 0; g < fused.size(); g++)
        if ((st = prepare_gate(c->n_qubits, fused[g].q, fused[g].k, fused[g].m.data(), o.zero_tol, &(*prepared)[g])) !=
            CAST_OK)
            return st;
    return CAST_OK;
}

static cast_status apply_all(cast_sv *sv, const std::vector<PreparedGate> &gates) {
    int kmax = 1;
    for (const PreparedGate &g : gates) kmax = std::max(kmax, g.k);
    cast_status st = ensure_gate_buffers(sv, kmax);
    if (st != CAST_OK) return st;
    for (const PreparedGate &g : gates)
        if ((st = launch_gate(sv, g)) != CAST_OK) return st;
    return CAST_OK;
}

cast_status cast_apply_circuit(cast_sv *sv, const cast_circuit *c, const double *params, const cast_options *opt) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    cast_status st = check_circuit(c, sv->n, params);
    if (st != CAST_OK) return st;
    const cast_options o = resolve_options(opt, sv->dt);
    if ((st = check_options(o)) != CAST_OK) return st;
    std::vector<PreparedGate> prepared;
    if ((st = prepare_circuit(c, params, o, &prepared)) != CAST_OK) return st;
    return apply_all(sv, prepared);
}

}  // extern "C"

struct cast_plan {
    int n = 0;
    std::vector<cast::PreparedGate> gates;
    int64_t ops = 0;
};

extern "C" {

cast_status cast_plan_create(const cast_circuit *c, const double *params, const cast_options *opt, cast_dtype dt,
                             cast_plan **out) {
    if (!out) return fail(CAST_ERR_ARG, "null output handle");
    *out = nullptr;
    if (!c) return fail(CAST_ERR_ARG, "null circuit");
    if (!valid_dt(dt)) return fail(CAST_ERR_ARG, "unknown dtype");
    if (c->n_qubits < 1 || c->n_qubits > CAST_MAX_QUBITS) return fail(CAST_ERR_ARG, "n_qubits out of range");
    cast_status st = check_circuit(c, c->n_qubits, params);
    if (st != CAST_OK) return st;
    const cast_options o = resolve_options(opt, dt);
    if ((st = check_options(o)) != CAST_OK) return st;
    cast_plan *p = new cast_plan();
    p->n = c->n_qubits;
    if ((st = prepare_circuit(c, params, o, &p->gates)) != CAST_OK) {
        delete p;
        return st;
    }
    for (const PreparedGate &g : p->gates) p->ops += opcount(g.m.data(), g.k, o.zero_tol);
    *out = p;
    return CAST_OK;
}

cast_status cast_plan_apply(cast_sv *sv, const cast_plan *p) {
    if (check_sv(sv) != CAST_OK) return CAST_ERR_ARG;
    if (!p) return fail(CAST_ERR_ARG, "null plan");
    if (p->n != sv->n) return fail(CAST_ERR_ARG, "plan qubit count differs from the state's");
    return apply_all(sv, p->gates);
}

cast_status cast_plan_info(const cast_plan *p, int *n_gates, int64_t *total_ops) {
    if (!p) return fail(CAST_ERR_ARG, "null plan");
    if (n_gates) *n_gates = (int)p->gates.size();
    if (total_ops) *total_ops = p->ops;
    return CAST_OK;
}

cast_status cast_plan_destroy(cast_plan *p) {
    delete p;
    return CAST_OK;
}

cast_status cast_fuse(const cast_circuit *c, const double *params, const cast_options *opt, int *n_out,
                      int *ks_out, int *qubits_out, int64_t *opcount_out, double *matrices_out) {
    if (!c || !n_out) return fail(CAST_ERR_ARG, "null circuit or count");
    cast_status st = check_circuit(c, c->n_qubits, params);
    if (st != CAST_OK) return st;
    if (c->n_qubits < 1 || c->n_qubits > CAST_MAX_QUBITS) return fail(CAST_ERR_ARG, "n_qubits out of range");
    const cast_options o = resolve_options(opt, CAST_C64);
    if ((st = check_options(o)) != CAST_OK) return st;
    std::vector<FusedGate> fused;
    if (o.fusion == CAST_FUSE_NONE) {
        for (int g = 0; g < c->n_gates; g++) {
            std::vector<cplx> m;
            PreparedGate pg;
            if ((st = gate_matrix_of(c->gates[g], params, c->n_params, &m)) != CAST_OK) return st;
            if ((st = prepare_gate(c->n_qubits, c->gates[g].qubits, c->gates[g].k, m.data(), o.zero_tol, &pg)) != CAST_OK)
                return st;
            FusedGate fg;
            fg.k = pg.k;
            for (int i = 0; i < CAST_MAX_K; i++) fg.q[i] = i < pg.k ? pg.q[i] : -1;
            fg.m = pg.m;
            fg.ops = opcount(pg.m.data(), pg.k, o.zero_tol);
            fused.push_back(std::move(fg));
        }
    } else if ((st = fuse_circuit(c, params, &o, &fused)) != CAST_OK) {
        return st;
    }
    const int cap = *n_out;
    *n_out = (int)fused.size();
    if ((int)fused.size() > cap) return fail(CAST_ERR_ARG, "output capacity too small");
    const size_t slot = size_t(1) << (2 * CAST_MAX_K);
    for (size_t g = 0; g < fused.size(); g++) {
        if (ks_out) ks_out[g] = fused[g].k;
        if (qubits_out)
            for (int i = 0; i < CAST_MAX_K; i++) qubits_out[g * CAST_MAX_K + i] = fused[g].q[i];
        if (opcount_out) opcount_out[g] = fused[g].ops;
        if (matrices_out) {
            double *dst = matrices_out + 2 * slot * g;
            for (size_t i = 0; i < fused[g].m.size(); i++) {
                dst[2 * i] = fused[g].m[i].real();
                dst[2 * i + 1] = fused[g].m[i].imag();
            }
        }
    }
    return CAST_OK;
}

cast_status cast_expectation(const cast_sv *csv, const cast_pauli_sum *h, double *out) {
    if (check_sv(csv) != CAST_OK) return CAST_ERR_ARG;
    if (!out) return fail(CAST_ERR_ARG, "null output");
    cast_status st = check_pauli(h, csv->n);
    if (st != CAST_OK) return st;
    cast_sv *sv = const_cast<cast_sv *>(csv);  // scratch buffers only
    if ((st = ensure_pinned(sv, 64)) != CAST_OK) return st;
    if ((st = queue_expectation(sv, h)) != CAST_OK) return st;
    CAST_CUDA(cudaMemcpyAsync(sv->host_pinned, sv->partials.ptr, sizeof(double), cudaMemcpyDeviceToHost, sv->stream));
    CAST_CUDA(cudaStreamSynchronize(sv->stream));
    *out = *reinterpret_cast<double *>(sv->host_pinned);
    return take_device_error();
}

static cast_status same_shape(const cast_sv *a, const cast_sv *b) {
    if (check_sv(a) != CAST_OK || check_sv(b) != CAST_OK) return CAST_ERR_ARG;
    if (a->n != b->n || a->dt != b->dt) return fail(CAST_ERR_ARG, "work states must match psi's size and type");
    if (a == b || a->data == b->data) return fail(CAST_ERR_ARG, "work states must be distinct");
    return CAST_OK;
}

cast_status cast_adjoint_grad(cast_sv *psi, cast_sv *lam, const cast_circuit *c, const double *params,
                              const cast_pauli_sum *h, double *energy_out, double *grad_out) {
    cast_status st;
    if ((st = same_shape(psi, lam)) != CAST_OK) return st;
    if ((st = check_circuit(c, psi->n, params)) != CAST_OK) return st;
    if ((st = check_pauli(h, psi->n)) != CAST_OK) return st;
    if (!energy_out || (c->n_params > 0 && !grad_out)) return fail(CAST_ERR_ARG, "null outputs");
    // every gate's matrix (and its adjoint) is prepared before any launch
    const int G = c->n_gates;
    std::vector<PreparedGate> fwd(G), bwd(G);
    std::vector<int> rot_pauli(G, 0);
    for (int g = 0; g < G; g++) {
        const cast_gate &gt = c->gates[g];
        std::vector<cplx> m;
        if ((st = gate_matrix_of(gt, params, c->n_params, &m)) != CAST_OK) return st;
        if ((st = prepare_gate(psi->n, gt.qubits, gt.k, m.data(), 0.0, &fwd[g])) != CAST_OK) return st;
        if (gt.param_index >= 0) {
            if (gt.kind == CAST_GATE_RX) rot_pauli[g] = 1;
            else if (gt.kind == CAST_GATE_RY) rot_pauli[g] = 2;
            else if (gt.kind == CAST_GATE_RZ) rot_pauli[g] = 3;
            else return fail(CAST_ERR_UNSUPPORTED, "adjoint: only RX, RY, RZ may carry parameters");
            continue;
        }
        const int d = 1 << gt.k;
        std::vector<cplx> mh(m.size());
        for (int r = 0; r < d; r++)
            for (int cc = 0; cc < d; cc++) mh[size_t(r) * d + cc] = std::conj(m[size_t(cc) * d + r]);
        if ((st = prepare_gate(psi->n, gt.qubits, gt.k, mh.data(), 0.0, &bwd[g])) != CAST_OK) return st;
    }
    std::vector<int> rot_gates;
    for (int g = 0; g < G; g++)
        if (rot_pauli[g]) rot_gates.push_back(g);
    const int R = (int)rot_gates.size();
    const int B = reduce_grid_blocks();
    int kmax = 1;
    for (int g = 0; g < G; g++) kmax = std::max(kmax, c->gates[g].k);
    // device scratch (doubles): [2 energy][n_params grads][R gate values][R*B partials]
    const size_t nd = 2 + size_t(c->n_params) + R + size_t(R) * B + 2 * size_t(B);
    if ((st = ensure_dev(psi, psi->partials, nd * sizeof(double) + R * sizeof(int) + 64)) != CAST_OK) return st;
    if ((st = ensure_gate_buffers(psi, kmax)) != CAST_OK) return st;
    if ((st = ensure_gate_buffers(lam, kmax)) != CAST_OK) return st;
    const size_t pinned = (2 + size_t(c->n_params)) * sizeof(double) + R * sizeof(int) + 64;
    if ((st = ensure_pinned(psi, std::max<size_t>(pinned, psi->host_pinned_bytes))) != CAST_OK) return st;
    double *d_energy = reinterpret_cast<double *>(psi->partials.ptr);
    double *d_grad = d_energy + 2;
    double *gate_vals = d_grad + c->n_params;
    double *part = gate_vals + R;
    int *d_pidx = reinterpret_cast<int *>(part + size_t(R) * B + 2 * size_t(B));

    // lam's earlier work is ordered before this call, and all of this call's
    // work runs on psi's stream; lam's stream waits for it at the end.
    cudaStream_t lam_stream = lam->stream;
    if (lam_stream != psi->stream) {
        cudaEvent_t ev;
        CAST_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, lam_stream);
        cudaStreamWaitEvent(psi->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    lam->stream = psi->stream;
    struct Restore {
        cast_sv *s;
        cudaStream_t orig, work;
        ~Restore() {
            s->stream = orig;
            if (orig != work) {
                cudaEvent_t ev;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                    cudaEventRecord(ev, work);
                    cudaStreamWaitEvent(orig, ev, 0);
                    cudaEventDestroy(ev);
                }
            }
        }
    } restore{lam, lam_stream, psi->stream};

    // forward: psi <- U psi
    for (int g = 0; g < G; g++)
        if ((st = launch_gate(psi, fwd[g])) != CAST_OK) return st;
    // lam <- H psi, grouped by x mask;  E = Re <psi|lam>
    PauliGroups PG = group_terms(h);
    if (PG.xm.empty()) CAST_CUDA(cudaMemsetAsync(lam->data, 0, amp_bytes(psi->dt) << psi->n, psi->stream));
    for (size_t g = 0; g < PG.xm.size(); g++)
        if ((st = launch_pauli_apply(psi, lam, PG.xm[g], (int)PG.c[g].size(), PG.c[g].data(), PG.z[g].data(),
                                     g > 0)) != CAST_OK)
            return st;
    if ((st = launch_inner(psi, lam, part, part + B)) != CAST_OK) return st;
    if ((st = launch_finalize(psi->stream, part, B, 2, d_energy)) != CAST_OK) return st;
    // backward sweep: uncompute psi and lam together
    int slot = R;
    for (int g = G - 1; g >= 0; g--) {
        const cast_gate &gt = c->gates[g];
        if (rot_pauli[g]) {
            slot--;
            const double theta = params[gt.param_index];
            if ((st = launch_adjoint_rotation(psi, lam, fwd[g].q[0], rot_pauli[g], theta, part + size_t(slot) * B)) !=
                CAST_OK)
                return st;
        } else {
            if ((st = launch_gate(psi, bwd[g])) != CAST_OK) return st;
            if ((st = launch_gate(lam, bwd[g])) != CAST_OK) return st;
        }
    }
    char *hp = reinterpret_cast<char *>(psi->host_pinned);
    if (R > 0) {
        if ((st = launch_finalize(psi->stream, part, B, R, gate_vals)) != CAST_OK) return st;
        int *hpidx = reinterpret_cast<int *>(hp + (2 + size_t(c->n_params)) * sizeof(double));
        for (int i = 0; i < R; i++) hpidx[i] = c->gates[rot_gates[i]].param_index;
        CAST_CUDA(cudaMemcpyAsync(d_pidx, hpidx, R * sizeof(int), cudaMemcpyHostToDevice, psi->stream));
        if ((st = launch_param_sum(psi->stream, gate_vals, d_pidx, R, d_grad, c->n_params)) != CAST_OK) return st;
    } else if (c->n_params > 0) {
        CAST_CUDA(cudaMemsetAsync(d_grad, 0, c->n_params * sizeof(double), psi->stream));
    }
    CAST_CUDA(cudaMemcpyAsync(hp, d_energy, (c->n_params + 2) * sizeof(double), cudaMemcpyDeviceToHost, psi->stream));
    CAST_CUDA(cudaStreamSynchronize(psi->stream));
    const double *hd = reinterpret_cast<const double *>(hp);
    *energy_out = hd[0];
    for (int p = 0; p < c->n_params; p++) grad_out[p] = hd[2 + p];
    return take_device_error();
}

}  // extern "C"
