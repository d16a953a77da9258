/*
 * cast.h -- C ABI of the GB300 state-vector gate engine.
 *
 * The engine applies a stream of k-qubit unitaries (k = 1..7) to a 2^n
 * amplitude complex state vector held in GPU memory (Section II-A of the
 * paper, Eq. 1-3), optionally after the paper's agglomerative, sparsity-aware
 * gate fusion (Section IV, Algorithm 1), and computes expectation values and
 * adjoint gradients of parametrised circuits on the same state.
 *
 * Conventions shared by every call
 *   - Qubit q is bit q of the amplitude index (Eq. 1: U on qubit q is
 *     I^(n-q-1) (x) U (x) I^q, little-endian).
 *   - Amplitudes are interleaved (re, im): complex64 = 2 x float,
 *     complex128 = 2 x double.  The buffer is 2^n * S bytes, S = 8 or 16.
 *   - Gate matrices are given in complex128, row-major, interleaved, 2^k x 2^k;
 *     bit i of a row/column index belongs to qubits[i] (caller's order).
 *   - Every pointer argument is borrowed for the duration of the call only;
 *     the library copies what it needs before returning.
 *   - Work on a state is queued on the CUDA stream given when the state was
 *     created or wrapped, and is asynchronous with respect to the host, except
 *     for calls that return host values (copy_to_host, expectation,
 *     adjoint_grad, fuse) which wait for their own results.
 *   - Every call validates its arguments before any GPU work is queued and
 *     returns a cast_status; on failure nothing has been queued and
 *     cast_last_error() describes the problem.  No call aborts the process.
 *
 * Thread safety: distinct states may be used from distinct host threads;
 * one state must not be used by two threads at once.
 */
#ifndef CAST_H
#define CAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CAST_MAX_QUBITS 34 /* 2^34 complex64 = 128 GiB */
#define CAST_MAX_K 7       /* largest gate the kernels accept */

typedef enum { CAST_C64 = 0, CAST_C128 = 1 } cast_dtype;

typedef enum {
    CAST_OK = 0,
    CAST_ERR_ARG = 1,         /* invalid argument (nothing queued) */
    CAST_ERR_OOM = 2,         /* device or pinned-host allocation failed */
    CAST_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    CAST_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    CAST_ERR_UNSUPPORTED = 5  /* valid request the library does not serve */
} cast_status;

/* Opaque state-vector handle. */
typedef struct cast_sv cast_sv;

/* ------------------------------------------------------------------------
 * State vectors
 * ---------------------------------------------------------------------- */

/* Allocate a 2^n_qubits state of type dt on the current CUDA device, set to
 * |0...0>, bound to `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream).  1 <= n_qubits <= CAST_MAX_QUBITS.  The library owns the memory
 * until cast_sv_destroy.  CAST_ERR_OOM if the device allocation fails. */
cast_status cast_sv_create(int n_qubits, cast_dtype dt, void *cuda_stream, cast_sv **out);

/* Wrap caller-owned device memory (2^n_qubits amplitudes of type dt, 256-byte
 * aligned) without copying it; the contents are used as they are.  The
 * caller keeps ownership and must keep the memory alive until
 * cast_sv_destroy(*out).  CAST_ERR_ARG for a NULL or misaligned pointer or
 * n_qubits outside 1..CAST_MAX_QUBITS. */
cast_status cast_sv_wrap(void *device_ptr, int n_qubits, cast_dtype dt, void *cuda_stream,
                         cast_sv **out);

/* Release the handle (and the amplitudes if the library allocated them).
 * Waits for the state's queued work first.  NULL is accepted. */
cast_status cast_sv_destroy(cast_sv *sv);

/* Size and location of a state. Any out-pointer may be NULL. */
cast_status cast_sv_info(const cast_sv *sv, int *n_qubits, cast_dtype *dt, void **device_ptr);

/* Set the state to the computational basis state |index>, index < 2^n.
 * CAST_ERR_ARG for a NULL state or index >= 2^n. */
cast_status cast_sv_set_basis(cast_sv *sv, uint64_t index);

/* Copy all 2^n amplitudes to / from host memory (2^n * S bytes, interleaved).
 * Both wait for completion before returning.  CAST_ERR_ARG for a NULL state
 * or buffer; copy_to_host also reports a bounded device wait that gave up in
 * earlier work on the stream (CAST_ERR_TIMEOUT). */
cast_status cast_sv_copy_to_host(const cast_sv *sv, void *host);
cast_status cast_sv_copy_from_host(cast_sv *sv, const void *host);

/* Queue the copy of all 2^n amplitudes from host memory on the state's stream
 * and return without waiting, so that a caller with two states on two
 * streams can stream one state's next input in while the other computes.
 * The copy is asynchronous only when `host` is page-locked (cudaHostAlloc or
 * a pinned torch tensor); the buffer must stay valid and unchanged until the
 * state's stream has passed the copy (e.g. until a later call on this state
 * that waits, such as cast_expectation). */
cast_status cast_sv_copy_from_host_async(cast_sv *sv, const void *host);

/* ------------------------------------------------------------------------
 * Single gates (Eq. 3)
 * ---------------------------------------------------------------------- */

/* Apply one k-qubit gate, 1 <= k <= min(CAST_MAX_K, n): for every t in
 * [0, 2^(n-k)) gather the 2^k amplitudes whose indices differ only in the
 * target bits, multiply by the 2^k x 2^k matrix, scatter back (Eq. 3).
 * qubits: k distinct values in [0, n).  matrix: 4^k complex128 entries.
 * Entries with |re|, |im| <= zero_tol (1e-12) are treated as zero when the
 * library picks a diagonal, monomial or dense kernel for the matrix.
 * CAST_ERR_ARG for a NULL argument, k out of range, a repeated or
 * out-of-range qubit or a non-finite entry. */
cast_status cast_apply_gate(cast_sv *sv, const int *qubits, int k, const double *matrix);

/* Host only (no CUDA call): the kernel family cast_apply_gate takes for this
 * gate on a state of n_qubits qubits and type dt under the current mode
 * settings (cast_set_tensor_mode, cast_set_f64_mode,
 * cast_set_c128_tensor_mode, cast_set_sparse_mode):
 *   CAST_PATH_DIGIT            complex128 dense-class k = 3..7 as digit
 *                              products on the tensor cores;
 *   CAST_PATH_LIST             the sparsity-specialised list kernel (per-row
 *                              lists of tagged non-zero entries, Section V-A);
 *   CAST_PATH_TENSOR_CHUNKED   complex64 dense unitary k = 6, 7 on the tensor
 *                              cores, K fed in chunks;
 *   CAST_PATH_TENSOR           complex64 dense unitary k = 4, 5 on the tensor
 *                              cores;
 *   CAST_PATH_DOUBLE_FLOAT     complex128 k <= 5 in double-float arithmetic
 *                              on the CUDA cores;
 *   CAST_PATH_CUDA_CORE        the FP32 / FP64 CUDA-core kernels (identity,
 *                              diagonal, monomial, dense, cube, tile).
 * Same arguments and CAST_ERR_ARG cases as cast_apply_gate, plus
 * n_qubits outside 1..CAST_MAX_QUBITS or an unknown dt. */
#define CAST_PATH_DIGIT 0
#define CAST_PATH_LIST 1
#define CAST_PATH_TENSOR_CHUNKED 2
#define CAST_PATH_TENSOR 3
#define CAST_PATH_DOUBLE_FLOAT 4
#define CAST_PATH_CUDA_CORE 5
cast_status cast_gate_path(int n_qubits, cast_dtype dt, const int *qubits, int k, const double *matrix,
                           int *path);

/* Arithmetic for dense, unitary complex64 gates with k = 4..7 on states of
 * at least k + 7 qubits (process-wide setting):
 *   CAST_TC_TF32X3 (default): tcgen05 tensor cores, each operand split into
 *     two tf32 parts, three products accumulated in fp32, and each slice's
 *     norm restored to its input norm (fp32-class accuracy, unbiased);
 *   CAST_TC_BF16X6: as CAST_TC_TF32X3, but k = 4, 5 gates split each operand
 *     into three bf16 parts (the first two truncated, so the remainders are
 *     exact, the last rounded) and accumulate the six products of weight
 *     above 2^-24 (kind::f16); k = 6, 7 stay on 3xTF32;
 *   CAST_TC_OFF: fp32 FMA on the CUDA cores for every gate.
 * Other gates are unaffected.  CAST_ERR_ARG for an unknown mode. */
#define CAST_TC_OFF 0
#define CAST_TC_TF32X3 1
#define CAST_TC_BF16X6 2
cast_status cast_set_tensor_mode(int mode);
int cast_get_tensor_mode(void);

/* complex128 dense gates on the tensor cores (process-wide setting):
 *   CAST_C128_TC_OFF: double-float arithmetic on the FP32 pipe;
 *   CAST_C128_TC_OZAKI (default): dense-class gates of k = 3..7 on states of
 *     n >= k + 7 qubits (in CAST_F64_EMULATED mode) as exact products of
 *     7-bit digits on tcgen05 (kind::f16, bf16 operands, fp32 accumulation
 *     that never rounds for the five leading digit-weight sums): each slice
 *     row and each row of the gate's real form is scaled by a power of two
 *     and cut to 49 fractional bits (rounded), the digit-pair products with
 *     i + j <= 7 are accumulated by weight, and the result is assembled with
 *     integer operations; error ~2^-48 of the slice's largest amplitude.
 *     Gates below about 33 / 17 / 11 / 10 / 5% of the dense operation count
 *     (k = 3..7), where the list kernel is faster, stay on it.  The paper has
 *     no tensor-core path; this is the complex128 form of Eq. 3's matvec on
 *     GB300's tensor cores.
 * CAST_ERR_ARG for an unknown mode. */
#define CAST_C128_TC_OFF 0
#define CAST_C128_TC_OZAKI 1
cast_status cast_set_c128_tensor_mode(int mode);
int cast_get_c128_tensor_mode(void);

/* Sparsity-specialised kernels (Section V-A: generated kernels skip zero
 * entries and specialise real and unit ones; Section IV-C: the cost of a gate
 * follows its operation count).  A dense-class gate of k = 3..7 qubits may
 * run through a per-row list of its non-zero entries, each tagged general
 * complex (4 multiply-adds), real or imaginary (2), or +-1 / +-i (2
 * additions); entries within 1e-14 of +-1 or +-i count as exactly that value
 * (the paper's one tolerance).  Process-wide setting:
 *   CAST_SPARSE_AUTO (default): complex128 (double-float mode) gates of
 *     k = 3..7 that the tensor-core digit kernels leave (every one with
 *     CAST_C128_TC_OFF); complex64 dense-class gates that the tensor cores do not take
 *     (non-unitary, or tensor cores off) of k = 4 with at most 24
 *     operations per amplitude, k = 5 with at most 80% and k = 6, 7 with at
 *     most 40% of the dense operation count;
 *   CAST_SPARSE_OFF: never;  CAST_SPARSE_ALWAYS: every dense-class gate of
 *     k = 3..7 (complex128 only in double-float mode).
 * States need n >= 12.  CAST_ERR_ARG for an unknown mode. */
#define CAST_SPARSE_AUTO 0
#define CAST_SPARSE_OFF 1
#define CAST_SPARSE_ALWAYS 2
cast_status cast_set_sparse_mode(int mode);
int cast_get_sparse_mode(void);

/* Measured tensor-pipe peak of the current GPU, in dense TFLOP/s: one CTA per
 * SM issues 32768 back-to-back tcgen05.mma instructions (M = 128, N = 256,
 * operands in shared memory, fp32 accumulation in tensor memory) and the best
 * of three timed launches is kept.  kind: CAST_PEAK_TF32 (kind::tf32) or
 * CAST_PEAK_BF16 (kind::f16 with bf16 operands).  The paper has no
 * counterpart: this is the denominator of the tensor-core kernels'
 * utilisation.  Waits; runs on its own stream; allocates nothing on the
 * device.  CAST_ERR_ARG for an unknown kind, CAST_ERR_TIMEOUT if the MMAs
 * did not complete within the bounded wait. */
#define CAST_PEAK_TF32 0
#define CAST_PEAK_BF16 1
cast_status cast_measure_tensor_peak(int kind, double *tflops);

/* Issue cost of one small tensor-core MMA on the current GPU, in SM clock
 * cycles: one CTA per SM issues 8192 back-to-back tcgen05.mma kind::f16
 * instructions (M = 128, K = 16, N = n_cols, bf16 zero operands, A from tensor
 * memory if a_in_tmem else from shared memory, one fp32 accumulator) and the
 * SM's clock64 is read from the first issue to the completion of their
 * commit; *cycles_per_mma is the mean over SMs, best of two timed launches.
 * It is the measurement behind the complex128 digit kernels' operand layout
 * (one MMA over stacked digit blocks instead of many narrow ones).
 * CAST_ERR_ARG unless n_cols is 16..256 and a multiple of 16. */
cast_status cast_measure_mma_issue(int n_cols, int a_in_tmem, double *cycles_per_mma);

/* Failure-detection test hook.  The next tensor-core gate launch (complex64
 * k = 4..7, complex128 digit products k = 3..5; a complex128 gate of k = 6,
 * 7 leaves the hook pending) waits on an
 * MMA completion that never comes (its issuing thread skips the MMAs), with
 * the barrier wait bounded to wait_limit polls instead of the default 2^26:
 * every CTA gives up, frees its tensor memory and returns; the error is
 * reported as CAST_ERR_TIMEOUT by the next call that synchronises with the
 * state (copy_to_host, expectation, adjoint_grad).  The state's contents are
 * then unspecified; the CUDA context stays usable.  Nothing traps or hangs. */
cast_status cast_debug_inject_timeout(uint32_t wait_limit);

/* Arithmetic for complex128 gates (process-wide setting):
 *   CAST_F64_EMULATED (default): dense (k <= 5), diagonal and phased
 *     monomial gates in double-float arithmetic on the FP32 pipe (pairs of
 *     floats, error-free TwoSum / TwoProduct, ~2^-46 relative error), with the
 *     FP64 <-> float-pair conversions done by integer bit manipulation;
 *     magnitudes must stay below 2^120;
 *   CAST_F64_NATIVE: IEEE FP64 on the FP64 pipe (about 1/67 of the FP32 rate
 *     on this GPU).
 * CAST_ERR_ARG for an unknown mode. */
#define CAST_F64_EMULATED 0
#define CAST_F64_NATIVE 1
cast_status cast_set_f64_mode(int mode);
int cast_get_f64_mode(void);

/* ------------------------------------------------------------------------
 * Circuits and gate fusion (Section IV)
 * ---------------------------------------------------------------------- */

typedef enum {
    CAST_GATE_MATRIX = 0, /* explicit matrix in cast_gate.matrix */
    CAST_GATE_H = 1, CAST_GATE_X = 2, CAST_GATE_Y = 3, CAST_GATE_Z = 4,
    CAST_GATE_S = 5, CAST_GATE_T = 6,
    CAST_GATE_RX = 7, CAST_GATE_RY = 8, CAST_GATE_RZ = 9, /* exp(-i theta P / 2) */
    CAST_GATE_U3 = 10,   /* params (theta, phi, lambda) */
    CAST_GATE_CX = 11, CAST_GATE_CZ = 12,
    CAST_GATE_CP = 13,   /* diag(1, 1, 1, e^{i phi}) */
    CAST_GATE_SWAP = 14
} cast_gate_kind;

/* One gate.  For CX / CZ / CP qubits[0] is the control.  A rotation (RX, RY,
 * RZ, CP) with param_index >= 0 takes its angle from the params array given
 * to the call instead of params[0]. */
typedef struct {
    int32_t kind;          /* cast_gate_kind */
    int32_t k;             /* number of qubits (1..CAST_MAX_K) */
    int32_t qubits[CAST_MAX_K];
    int32_t param_index;   /* -1 = fixed angles in params[] */
    double params[3];
    const double *matrix;  /* CAST_GATE_MATRIX only: 4^k complex128 */
} cast_gate;

/* n_params: length of the angle array passed with the circuit; every
 * param_index must be below it.  Only RX, RY, RZ and CP may be parametrised. */
typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    const cast_gate *gates;
    int32_t n_params;
} cast_circuit;

typedef enum {
    CAST_FUSE_NONE = 0,     /* apply the gates as given */
    CAST_FUSE_SIZE = 1,     /* fuse while the fused block has <= max_k qubits */
    CAST_FUSE_ADAPTIVE = 2  /* size test plus the cost-model test (Section IV-C) */
} cast_fusion_mode;

/* Measured cost of one gate per size and class on a state of n_qubits
 * qubits: the GPU counterpart of the paper's CostModel (Section IV-C), which
 * records gate times for varying size and sparsity and launch shapes.
 * class index: 0 identity, 1 diagonal, 2 monomial, 3 dense.
 * The sparse kernel's cost grows with the operation count: a dense-class
 * gate of k = 3..7 qubits with operation count c is estimated at
 *   min(ms[k][3], max(sparse_floor_ms[k], sparse_ms_per_op[k] * c))
 * when both sparse entries of k are measured (> 0), else at ms[k][3]. */
typedef struct {
    int32_t n_qubits;
    int32_t dtype;                                 /* cast_dtype */
    double ms[CAST_MAX_K + 1][4];                  /* average ms per gate; 0 = not measured */
    int32_t blocks_per_sm[CAST_MAX_K + 1][4];      /* best CUDA-core launch width, 0 = default */
    double sparse_floor_ms[CAST_MAX_K + 1];        /* sparse kernel, two entries per row */
    double sparse_ms_per_op[CAST_MAX_K + 1];       /* sparse kernel, dense matrix time / its count */
} cast_cost_table;

typedef struct {
    int32_t fusion;        /* cast_fusion_mode, default CAST_FUSE_ADAPTIVE */
    int32_t max_k;         /* largest fused gate, 1..CAST_MAX_K, default 5 */
    int32_t agglomerative; /* 1: raise the allowed size 2..max_k (Section IV-B), default 1 */
    int32_t op_cap;        /* adaptive: largest operation count of a fused gate, default 4096 */
    double zero_tol;       /* |real scalar| <= zero_tol counts as zero, default 1e-12 */
    int32_t amp_ops_per_pass; /* adaptive cost model: operations per amplitude that take as
                                 long as one pass over the state; 0 = measured default for
                                 the state type (complex64: 82; complex128: 64 in the
                                 emulated mode, 2 with native FP64) */
    const cast_cost_table *cost; /* adaptive: estimate a block by the measured time of its
                                    (size, class) instead of the operation-count model;
                                    with max_k = 0 the plan also picks the fusion width
                                    2..CAST_MAX_K of least estimated time.  NULL = model */
} cast_options;
/* Every call taking options returns CAST_ERR_ARG, before any other work, for
 * an unknown fusion mode, max_k outside 1..CAST_MAX_K (0 only with a cost
 * table), agglomerative other than 0 or 1, a negative or non-finite
 * zero_tol, a negative op_cap or a negative amp_ops_per_pass. */

/* Measure the cost table on a scratch state of n_qubits (allocated and
 * freed here, filled with seeded pseudo-random amplitudes so that kernels
 * which skip work on zero values are timed as on a state in use) on
 * cuda_stream: one gate of every size 1..CAST_MAX_K and class
 * (diagonal, monomial, dense), for the CUDA-core kernels at launch widths of
 * 1, 2, 4 and 8 blocks per SM keeping the fastest; then, for k = 3..7 and
 * n_qubits >= 12, the sparse kernel on a matrix with two entries per row
 * (its floor) and on the dense one (its time per operation).  Waits for the
 * results. */
cast_status cast_autotune(cast_dtype dt, int n_qubits, void *cuda_stream, cast_cost_table *out);

/* Use a table's launch widths for every later launch in this process (per
 * state type; NULL restores the built-in widths for both types). */
cast_status cast_set_cost_table(const cast_cost_table *t);

/* Fill *o with the defaults listed above. */
void cast_options_default(cast_options *o);

/* Apply a whole circuit: fuse on the host (unless opt->fusion is NONE),
 * classify each resulting gate, upload all matrices once, and queue one
 * kernel per gate.  params: angles for gates with param_index >= 0 (may be
 * NULL if there are none).  opt NULL = defaults.
 * c->n_qubits must equal the state's qubit count. */
cast_status cast_apply_circuit(cast_sv *sv, const cast_circuit *c, const double *params,
                               const cast_options *opt);

/* Host only (no GPU work): run the fusion pass and report its output.
 * On entry *n_out is the capacity of the output arrays (in gates); on return
 * it is the number of fused gates.  ks_out[g]: size of fused gate g;
 * qubits_out: CAST_MAX_K entries per gate, sorted ascending, unused = -1;
 * opcount_out[g]: operation count (Section IV-C: 2 per non-zero real scalar);
 * matrices_out (may be NULL): 4^CAST_MAX_K complex128 entries per gate, each
 * gate's 2^k x 2^k matrix stored row-major at the start of its slot, local
 * bit i <-> qubits_out[g*CAST_MAX_K + i].  CAST_ERR_ARG if the capacity is
 * too small (then *n_out is the required count).  With amp_ops_per_pass = 0
 * the complex64 default is used. */
cast_status cast_fuse(const cast_circuit *c, const double *params, const cast_options *opt,
                      int *n_out, int *ks_out, int *qubits_out, int64_t *opcount_out,
                      double *matrices_out);

/* Host only: operation count of a 2^k x 2^k complex128 matrix, i.e. 2 x the
 * number of real scalars with magnitude > zero_tol (Section IV-C). */
int64_t cast_opcount(const double *matrix, int k, double zero_tol);

/* ------------------------------------------------------------------------
 * Plans: a circuit fused and prepared once, applied many times
 * ---------------------------------------------------------------------- */

typedef struct cast_plan cast_plan;

/* Fuse (per *opt, NULL = defaults) and classify the circuit's gates on the
 * host and keep the result.  dt selects the cost-model default when
 * opt->amp_ops_per_pass is 0.  No GPU work.  The plan can be applied to any
 * state with c->n_qubits qubits, of either type. */
cast_status cast_plan_create(const cast_circuit *c, const double *params, const cast_options *opt,
                             cast_dtype dt, cast_plan **out);

/* Queue the plan's gates on the state's stream (one kernel per gate, or none
 * for gates that are the identity within the zero tolerance). */
cast_status cast_plan_apply(cast_sv *sv, const cast_plan *p);

/* Number of gates after fusion, and their total operation count (either
 * out-pointer may be NULL). */
cast_status cast_plan_info(const cast_plan *p, int *n_gates, int64_t *total_ops);

/* Free a plan (host memory only; work already queued from it is unaffected).
 * NULL is accepted. */
cast_status cast_plan_destroy(cast_plan *p);

/* ------------------------------------------------------------------------
 * Profiling: CUDA events around every kernel launch, on its own stream
 * ---------------------------------------------------------------------- */

typedef struct {
    char name[32];      /* kernel family, e.g. "dense_k5_c64" */
    int64_t launches;
    double ms;          /* sum of event-measured launch durations */
    double bytes;       /* sum of algorithmic bytes: the amplitudes the
                           method must read and write (2 N S per full pass) */
    double flops;       /* sum of algorithmic floating-point operations */
} cast_profile_entry;

/* Start recording (clears earlier records).  Adds two event records per
 * launch; meant for measurement runs. */
cast_status cast_profile_begin(void);

/* Stop recording, wait for the recorded events and return one entry per
 * kernel family, largest total time first.  *n_out: in = capacity of out,
 * out = number of families (CAST_ERR_ARG if the capacity is too small). */
cast_status cast_profile_end(cast_profile_entry *out, int *n_out);

/* ------------------------------------------------------------------------
 * Observables and gradients
 * ---------------------------------------------------------------------- */

/* A sum of Pauli strings, each c_t * P_t with P_t given by two bit masks:
 * bit q of x_mask set = X or Y on qubit q; bit q of z_mask set = Z or Y on
 * qubit q (both set = Y).  Coefficients are real, so H is Hermitian. */
typedef struct {
    int32_t n_terms;
    const double *coeffs;
    const uint64_t *x_masks;
    const uint64_t *z_masks;
} cast_pauli_sum;

/* *out = <psi|H|psi> accumulated in FP64.  Waits for the result. */
cast_status cast_expectation(const cast_sv *sv, const cast_pauli_sum *h, double *out);

/* Scratch size of cast_expectation_noalloc, in doubles (512 KiB). */
#define CAST_NOALLOC_SCRATCH_DOUBLES 65536

/* The value of cast_expectation, computed without allocating any memory.
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate: a process whose state vector already fills the GPU's
 * memory (a 33-qubit complex128 state takes 128 GiB), code running under a
 * memory manager that owns every device allocation, or a loop that must not
 * stall on the device-wide synchronisation that cudaMalloc and cudaFree can
 * cause.  cast_expectation allocates its partial-sum buffer and a pinned
 * result buffer on first use; this call instead keeps its scratch in one
 * fixed array of CAST_NOALLOC_SCRATCH_DOUBLES doubles that every GPU which
 * loads the library holds until the process exits, and copies the result
 * straight into *out.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The state's device must be current.  The
 *     address is kept for the process's life: after cudaDeviceReset it is
 *     stale, and this call must not be used again.
 *   - A Pauli sum needs 1 + (launches x blocks) doubles, one launch per
 *     32 terms sharing an x_mask and 4 blocks per SM (608 on a 152-SM GB300,
 *     so up to 107 launches); larger sums get CAST_ERR_ARG, with the launch
 *     and block counts in the message.
 *   - Like cast_expectation it returns CAST_ERR_TIMEOUT when earlier work on
 *     the state's stream gave up a bounded wait (the value is then void).
 *   - All calls share the array and it keeps the last call's contents; each
 *     call writes every value it reads, so nothing needs clearing, but calls
 *     whose GPU work overlaps (e.g. on two streams) race and may return wrong
 *     values.
 * Waits for the result. */
cast_status cast_expectation_noalloc(const cast_sv *sv, const cast_pauli_sum *h, double *out);

/* Adjoint differentiation of E(theta) = <psi0|U(theta)^dag H U(theta)|psi0>
 * for a circuit whose parametrised gates are RX/RY/RZ (exp(-i theta P / 2))
 * with param_index >= 0; fixed gates may be of any kind.
 *   psi   : on entry the initial state psi0; on return psi0 recomputed by
 *           uncomputation (equal to the input up to rounding)
 *   lam   : work state of the same size and type (contents ignored); its
 *           stream waits for psi's stream around the call
 *   params: the circuit's c->n_params angles; grad_out[p] for
 *           p < c->n_params receives dE/dtheta_p; energy_out receives E.
 * Uses two state vectors in total, independent of the circuit depth:
 * the forward pass, lam = H psi, then one backward sweep that applies
 * U_j^dag to psi and lam and, at each rotation, forms Im<lam|P|psi> (the
 * derivative of exp(-i theta P / 2)) with FP64-class accumulation.
 * Waits for the result. */
cast_status cast_adjoint_grad(cast_sv *psi, cast_sv *lam, const cast_circuit *c, const double *params,
                              const cast_pauli_sum *h, double *energy_out, double *grad_out);

/* ------------------------------------------------------------------------
 * Batched variational circuits: the hardware-efficient ansatz
 * ---------------------------------------------------------------------- */

/* A batch of instances of the hardware-efficient ansatz, each with its own
 * qubit count n_i (2..30) and parameters: per layer RY(theta) on every qubit,
 * RZ(phi) on every qubit, then CZ(i, i+1) for i < n_i - 1, starting from
 * |0...0>.  Instance i's 2 n_i L parameters are, per layer l, the n_i RY
 * angles then the n_i RZ angles (index 2 n_i l + q and 2 n_i l + n_i + q);
 * the batch's parameter array concatenates the instances in order.
 * Energies are of H = zz sum_{i<n-1} Z_i Z_{i+1} + hx sum_i X_i (open
 * boundary), accumulated in FP64.  These are the training forms of the same
 * gate arithmetic (Eq. 3); the paper's VQA motivation is in Section I.
 *
 * The gates of a group of up to T - 5 qubits are applied while a tile of 2^T
 * amplitudes is resident in shared memory (T = 12 complex64, 11
 * complex128), so a layer costs ~n/(T-5) passes over the states instead of
 * 3n - 1; all instances share each launch, and the launch sequence is
 * captured once in a CUDA graph and replayed for every parameter set.
 * with_grad allocates the second state arena that adjoint gradients need.
 * A CAST_C128 batch computes in the arithmetic cast_set_f64_mode selects when
 * a call builds its graph (double-float by default: the arenas then hold
 * (hi, lo) float pairs, 16 bytes per amplitude like complex128); a later
 * mode change rebuilds the graph at the next call. */
typedef struct cast_hea cast_hea;

/* CAST_ERR_ARG for no instances, a qubit count outside 2..30, layers < 1,
 * an unknown dtype or a NULL output; CAST_ERR_OOM if the arenas do not fit. */
cast_status cast_hea_create(int n_instances, const int32_t *n_qubits, int layers, cast_dtype dt,
                            int with_grad, void *cuda_stream, cast_hea **out);

/* energies[i] = <psi_i|H|psi_i>.  params: all instances' parameters.
 * Waits for the result. */
cast_status cast_hea_energy(cast_hea *b, const double *params, double zz, double hx, double *energies);

/* Energies plus adjoint gradients (same layout as params): forward sweep,
 * lambda = H psi, then a backward sweep that un-applies the gates from psi
 * and lambda and forms Im<lambda|P|psi> for every rotation (two state
 * vectors per instance).  CAST_ERR_ARG if the batch was created without
 * with_grad.  Waits for the result. */
cast_status cast_hea_grad(cast_hea *b, const double *params, double zz, double hx, double *energies,
                          double *grads);

/* Total parameter count and the largest number of passes per layer. */
cast_status cast_hea_info(const cast_hea *b, int *n_params, int *n_passes_per_layer_max);

/* Wait for the batch's stream, then free its arenas and graphs.  NULL is
 * accepted. */
cast_status cast_hea_destroy(cast_hea *b);

/* ------------------------------------------------------------------------
 * Batched variational circuits of any shape
 * ---------------------------------------------------------------------- */

/* A batch of circuit instances that need not share a shape: instance i has
 * its own qubit count (1..30), gate list (1- and 2-qubit gates of any kind;
 * RX, RY, RZ may carry a parameter: exp(-i theta P / 2)) and Pauli sum, and
 * reads its parameters from the batch's parameter array starting at
 * param_offsets[i] (NULL: instances' parameters stored one after the other;
 * offsets may overlap to share parameters).  All states live in one arena,
 * each starting at |0...0>.  Gate step s applies the s-th gate of every
 * instance that has one in a single launch; rotation matrices are formed on
 * the device from the parameters at every call, so the launch sequence is
 * captured once into a CUDA graph and replayed for each parameter set.  The
 * hardware-efficient ansatz has the faster tile executor (cast_hea_*); this is
 * the general form.  Gradients use the adjoint method (two state vectors per
 * instance, with_grad).  complex64 in FP32; complex128 in double-float
 * arithmetic; energies and gradients accumulate in FP64.  The circuits and
 * Pauli sums are copied; nothing the caller passed is kept. */
typedef struct cast_batch cast_batch;

/* CAST_ERR_ARG for no instances, a qubit count outside 1..30, an invalid gate
 * (qubits, arity, parameter index, non-finite matrix), a negative parameter
 * offset, an unknown dtype or a NULL output; CAST_ERR_UNSUPPORTED for a gate
 * of three or more qubits; CAST_ERR_OOM if the arenas do not fit. */
cast_status cast_batch_create(int n_instances, const cast_circuit *circuits, const int32_t *param_offsets,
                              const cast_pauli_sum *hamiltonians, cast_dtype dt, int with_grad,
                              void *cuda_stream, cast_batch **out);

/* energies[i] = <psi_i|H_i|psi_i> for the given parameters.  Waits. */
cast_status cast_batch_energy(cast_batch *b, const double *params, double *energies);

/* Energies plus dE_i/dparams (summed over the instances that read a
 * parameter), by the adjoint method.  CAST_ERR_ARG without with_grad.  Waits. */
cast_status cast_batch_grad(cast_batch *b, const double *params, double *energies, double *grads);

/* Parameter array length and number of gate steps (the longest gate list). */
cast_status cast_batch_info(const cast_batch *b, int *n_params, int *n_steps);

/* Free the batch's arenas and graphs (its calls have already waited for
 * their results).  NULL is accepted. */
cast_status cast_batch_destroy(cast_batch *b);

/* Thread-local description of the last failure on this host thread. */
const char *cast_last_error(void);

/* Version string of the library. */
const char *cast_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CAST_H */
