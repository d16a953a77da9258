// Internal declarations shared by the host side (capi.cpp, fusion.cpp,
// gates.cpp) and the CUDA kernels (apply.cu, reduce.cu, adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cast.h"

namespace cast {

using cplx = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
cast_status fail(cast_status st, const std::string &msg);
cast_status cuda_fail(cudaError_t e, const char *what);
#define CAST_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------------ state handle
struct DeviceScratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace cast

struct cast_sv {
    void *data = nullptr;    // 2^n amplitudes
    int n = 0;
    cast_dtype dt = CAST_C128;
    cudaStream_t stream = nullptr;
    bool owned = false;
    int device = 0;
    // per-state device scratch: FP64 partial sums of reductions
    cast::DeviceScratch partials;
    // per-state device scratch of kernels that hold results back (grow-only)
    cast::DeviceScratch work;
    // ring of device slots for matrices too large for launch parameters,
    // filled from pinned staging slots; slot i is reused after its last copy
    // completed (mat_events[i])
    void *mat_dev = nullptr;
    void *mat_pinned = nullptr;
    cudaEvent_t mat_events[16] = {nullptr};
    int mat_next = 0;
    // pinned host buffer for results
    void *host_pinned = nullptr;
    size_t host_pinned_bytes = 0;
};

namespace cast {

inline size_t amp_bytes(cast_dtype dt) { return dt == CAST_C128 ? 16 : 8; }

// ------------------------------------------------------------- profiling
// Records CUDA events around one launch on stream s while profiling is on.
class ProfScope {
  public:
    ProfScope(cudaStream_t s, const std::string &family, double bytes, double flops);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    bool active_ = false;
    cudaStream_t stream_ = nullptr;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    std::string fam_;
    double bytes_ = 0, flops_ = 0;
};
inline const char *dt_name(cast_dtype dt) { return dt == CAST_C64 ? "c64" : "c128"; }

// ---------------------------------------------------------- prepared gates
enum GateClass { CLS_IDENTITY = 0, CLS_DIAG = 1, CLS_MONO = 2, CLS_DENSE = 3 };

// A gate ready for a kernel: qubits sorted ascending, matrix permuted to that
// order, entries below the zero tolerance set to exactly zero.
struct PreparedGate {
    int k = 0;
    int q[CAST_MAX_K] = {0};
    int cls = CLS_DENSE;
    std::vector<cplx> m;        // 4^k, row-major, sorted-qubit order
    std::vector<cplx> diag;     // CLS_DIAG: 2^k diagonal entries
    std::vector<int> perm;      // CLS_MONO: row r reads column perm[r]
    std::vector<cplx> phase;    // CLS_MONO: value of the non-zero in row r
    bool unit_phases = false;   // CLS_MONO: every phase is exactly 1
    bool unitary = false;       // max |U^dag U - I| <= 1e-9
};

// Validate + sort + classify.  Returns CAST_OK or CAST_ERR_ARG.
cast_status prepare_gate(int n, const int *qubits, int k, const cplx *matrix, double zero_tol,
                         PreparedGate *out);
int64_t opcount(const cplx *m, int k, double zero_tol);

// Matrix of a table gate (kind != MATRIX) with the given angles.
cast_status gate_table_matrix(int kind, int k, const double *params, std::vector<cplx> *out);
int gate_table_arity(int kind);
// Matrix of any cast_gate (table gate, parametrised rotation or explicit).
cast_status gate_matrix_of(const cast_gate &g, const double *params, int n_params,
                           std::vector<cplx> *out);
int64_t default_amp_ops_per_pass(cast_dtype dt);

// ------------------------------------------------------- shared validation
cast_status check_sv(const cast_sv *sv);
cast_status check_pauli(const cast_pauli_sum *h, int n);
// Pauli terms grouped by x_mask, ascending mask order
struct PauliGroups {
    std::vector<uint64_t> xm;
    std::vector<std::vector<double>> c;
    std::vector<std::vector<uint64_t>> z;
};
PauliGroups group_terms(const cast_pauli_sum *h);

// ------------------------------------------------------------ fusion pass
struct FusedGate {
    int k;
    int q[CAST_MAX_K];         // sorted ascending
    std::vector<cplx> m;       // 4^k row-major over q
    int64_t ops;
};
cast_status fuse_circuit(const cast_circuit *c, const double *params, const cast_options *opt,
                         std::vector<FusedGate> *out);

// --------------------------------------------------------------- kernels
// Matrix ring: kMatSlots slots of kMatSlotBytes (a 7-qubit complex128 matrix,
// the entry list of a dense 7-qubit complex128 gate for the sparse kernel, or
// the 896 KiB digit image of a dense 7-qubit complex128 gate).
constexpr int kMatSlots = 16;
constexpr size_t kMatSlotBytes = size_t(1) << 20;
// Copy `bytes` (<= kMatSlotBytes) of host data to a device slot, in stream
// order on sv's stream; *dev receives the slot's device address.
cast_status upload_matrix(cast_sv *sv, const void *host, size_t bytes, const void **dev);
// sv->work grown to at least `bytes` (in stream order); *ptr its device address.
cast_status ensure_work(cast_sv *sv, size_t bytes, void **ptr);

// Queue one prepared gate on sv's stream.
// Staging geometry of a warp's "cube": 32 consecutive slices (rows) x the
// members spanned by the first mb = min(k, 4) targets (mb member bits), i.e.
// 5 + mb index bits: the 5 lowest non-target bits and q0..q_{mb-1}.  Address
// bits 0..4 always belong to it, so the cube is made of runs of at least 32
// contiguous amplitudes and a warp moves it with coalesced 16-byte chunks.
// In shared memory cube element c sits in slot c ^ X(c >> 4): X maps the row
// bits that land above bit 3 onto free slot bits 1..3, so 16-byte chunk
// accesses (8 lanes per phase) never conflict and 8-byte row accesses
// (16 lanes per phase) conflict at most 2-way (only when qubit 0 is a
// target; then 16-byte row accesses of member pairs are conflict-free).  Offsets and slots are additive over disjoint bit fields: an
// element is addressed by one per-lane entry combined with one per-round or
// per-member entry.  Built on the host per gate (csrc/cube.cpp).
struct CubeTables {
    uint64_t g_lane[32];  // global offset (amplitudes) of cube element 2 * lane, from the cube base
    uint64_t g_j[8];      // offset of element 64 * j (chunk round j; 2^(mb-1) rounds)
    uint16_t s_lane[32];  // slot of element 2 * lane
    uint16_t s_j[8];      // slot of element 64 * j
    uint16_t s_row[32];   // slot of (row r = lane, member 0)
    uint16_t s_mem[16];   // slot of (row 0, member m), m < 2^mb
    uint32_t pair;        // q0 == 0: members 2m and 2m+1 of a row share one 16-byte chunk,
                          // so rows move as 16-byte pairs (conflict-free, half the accesses)
};
CubeTables make_cube_tables(const int *q, int k);
// the same with the cube's member bits given: the first mb targets (mb <= min(k, 4))
CubeTables make_cube_tables(const int *q, int k, int mb);

// Bit layout of a list-kernel super-tile (apply_sparse.cu): 4096 amplitudes
// whose 12 varying address bits are the 12 - k lowest non-target positions
// and the k targets.  Cube position b (ascending address bit pos[b]) is
// either bit role[b] < 16 of the slice row within the super-tile or target
// bit role[b] - 16 of the member index.  Built on the host per gate
// (csrc/cube.cpp); needs n >= 12.
struct SpTile {
    uint8_t pos[12];
    uint8_t role[12];
};
SpTile make_tile_layout(const int *q, int k);

cast_status launch_gate(cast_sv *sv, const PreparedGate &g);
// The kernel family launch_gate takes for a prepared gate, from the state's
// qubit count and type and the process-wide mode settings only (host, no
// CUDA call); values as the CAST_PATH_* constants of cast.h.
int choose_path(const cast_sv *sv, const PreparedGate &g);
// Tensor-core path for dense complex64 gates (apply_tc.cu).
bool tc_eligible(const cast_sv *sv, const PreparedGate &g);
cast_status launch_gate_tc(cast_sv *sv, const PreparedGate &g);
bool tcc_eligible(const cast_sv *sv, const PreparedGate &g);  // dense k = 6, 7, K-chunked (apply_tcc.cu)
cast_status launch_gate_tcc(cast_sv *sv, const PreparedGate &g);
int tcc_error_flag_take();          // the chunked kernel's bounded-wait error flag, cleared
bool tensor_cores_on();             // cast_set_tensor_mode other than CAST_TC_OFF in effect
uint32_t take_inject_limit();       // cast_debug_inject_timeout's pending limit, cleared (0: none)
// Autotuned launch width (blocks per SM) of a CUDA-core kernel, or def.
int tuned_blocks_per_sm(cast_dtype dt, int k, int cls, int def);
// Cost-table estimate of one gate of size k, class cls and operation count
// ops, in integer ns.
int64_t table_estimate(const cast_cost_table &t, int k, int cls, int64_t ops);
// Class of a 2^k x 2^k matrix (identity / diagonal / monomial / dense).
int classify_matrix(const cplx *m, int k, double zero_tol);

// Sparsity-specialised kernels (apply_sparse.cu): per-row entry lists, k = 3..7.
bool sparse_preferred(const cast_sv *sv, const PreparedGate &g);
cast_status launch_gate_sparse(cast_sv *sv, const PreparedGate &g);
int64_t dense_opcount(int k);
int sparse_mode();  // CAST_SPARSE_AUTO / OFF / ALWAYS

// Tensor-core complex128 path for dense k = 4..7 (apply_oz.cu): exact
// products of 7-bit digits.
bool oz_eligible(const cast_sv *sv, const PreparedGate &g);
cast_status launch_gate_oz(cast_sv *sv, const PreparedGate &g);
int oz_error_flag_take();

// Double-float path for complex128 gates (apply_df.cu).
bool df_eligible(const cast_sv *sv, const PreparedGate &g);
cast_status launch_gate_df(cast_sv *sv, const PreparedGate &g);
int f64_mode();
// CAST_ERR_TIMEOUT (and clears the flag) if a kernel's bounded wait gave up.
cast_status take_device_error();
// Queue sum_t coeff_t <psi|P_t|psi> terms sharing one x_mask; partial sums
// of FP64 go to sv->partials; returns the number of partials written.
cast_status launch_pauli_group(const cast_sv *sv, uint64_t x_mask, int n_terms,
                               const double *coeffs, const uint64_t *z_masks, double *d_out,
                               int *n_partials);
int reduce_grid_blocks();
// Partial sums launch_pauli_group writes for all groups of G: one launch per
// kMaxTerms terms of a group, reduce_grid_blocks() partials per launch.
size_t pauli_partials_needed(const PauliGroups &G);
int sm_count_cached();
cast_status launch_set_one(cast_sv *sv, uint64_t index);
// Pseudo-random amplitudes of magnitude ~2^(-n/2) in every entry (timing probes).
cast_status launch_fill_random(cast_sv *sv, uint64_t seed);
cast_status launch_param_sum(cudaStream_t st, const double *gate_vals, const int *gate_pidx, int ngates,
                             double *grad, int nparams);
cast_status launch_finalize(cudaStream_t st, const double *d_partials, int per_slot, int nslots,
                            double *d_out);
cast_status launch_inner(const cast_sv *a, const cast_sv *b, double *d_partials_re,
                         double *d_partials_im);
// out = (or +=) sum over terms sharing x_mask of c_t P_t psi
cast_status launch_pauli_apply(const cast_sv *psi, cast_sv *out, uint64_t x_mask, int n_terms,
                               const double *coeffs, const uint64_t *z_masks, bool accumulate);
// Adjoint step for a rotation exp(-i theta P / 2) on qubit q (P = 1:X, 2:Y, 3:Z):
// partial sums of Im<lam|P_q|psi> into d_partials (reduce_grid_blocks() values),
// then psi <- U^dag psi and lam <- U^dag lam.
cast_status launch_adjoint_rotation(cast_sv *psi, cast_sv *lam, int q, int pauli, double theta,
                                    double *d_partials);

}  // namespace cast
