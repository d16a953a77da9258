"""ctypes binding of include/cast.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
simulation work of its own: it converts Python / numpy / torch arguments to the
C structs, calls libcast.so, and raises CastError when the call fails.  The
library must have been built (paper_2503_19894_gb300.build.build()); there is
no fallback of any kind when it is missing.
"""
import ctypes
import os

import numpy as np

from . import build as _build

CAST_MAX_K = 7
CAST_MAX_QUBITS = 34
CAST_C64, CAST_C128 = 0, 1
CAST_FUSE_NONE, CAST_FUSE_SIZE, CAST_FUSE_ADAPTIVE = 0, 1, 2
STATUS = {0: "CAST_OK", 1: "CAST_ERR_ARG", 2: "CAST_ERR_OOM", 3: "CAST_ERR_CUDA",
          4: "CAST_ERR_TIMEOUT", 5: "CAST_ERR_UNSUPPORTED"}
GATE_KIND = {"U": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "T": 6, "RX": 7, "RY": 8,
             "RZ": 9, "U3": 10, "CX": 11, "CZ": 12, "CP": 13, "SWAP": 14}
DTYPES = {"c64": CAST_C64, "complex64": CAST_C64, "c128": CAST_C128, "complex128": CAST_C128}


class CastError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class cast_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("qubits", ctypes.c_int32 * CAST_MAX_K), ("param_index", ctypes.c_int32),
                ("params", ctypes.c_double * 3), ("matrix", ctypes.c_void_p)]


class cast_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32),
                ("gates", ctypes.POINTER(cast_gate)), ("n_params", ctypes.c_int32)]


class cast_cost_table(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("ms", (ctypes.c_double * 4) * (CAST_MAX_K + 1)),
                ("blocks_per_sm", (ctypes.c_int32 * 4) * (CAST_MAX_K + 1)),
                ("sparse_floor_ms", ctypes.c_double * (CAST_MAX_K + 1)),
                ("sparse_ms_per_op", ctypes.c_double * (CAST_MAX_K + 1))]


class cast_options(ctypes.Structure):
    _fields_ = [("fusion", ctypes.c_int32), ("max_k", ctypes.c_int32),
                ("agglomerative", ctypes.c_int32), ("op_cap", ctypes.c_int32),
                ("zero_tol", ctypes.c_double), ("amp_ops_per_pass", ctypes.c_int32),
                ("cost", ctypes.POINTER(cast_cost_table))]


class cast_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class cast_pauli_sum(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int32), ("coeffs", ctypes.c_void_p),
                ("x_masks", ctypes.c_void_p), ("z_masks", ctypes.c_void_p)]


EXPORTS = ("cast_sv_create", "cast_sv_wrap", "cast_sv_destroy", "cast_sv_info",
           "cast_sv_set_basis", "cast_sv_copy_to_host", "cast_sv_copy_from_host", "cast_sv_copy_from_host_async",
           "cast_apply_gate", "cast_options_default", "cast_apply_circuit", "cast_fuse",
           "cast_opcount", "cast_expectation", "cast_adjoint_grad", "cast_last_error",
           "cast_version", "cast_plan_create", "cast_plan_apply", "cast_plan_info",
           "cast_plan_destroy", "cast_profile_begin", "cast_profile_end",
           "cast_expectation_noalloc", "cast_set_tensor_mode", "cast_get_tensor_mode",
           "cast_hea_create", "cast_hea_energy", "cast_hea_grad", "cast_hea_info", "cast_hea_destroy",
           "cast_set_f64_mode", "cast_get_f64_mode", "cast_autotune", "cast_set_cost_table",
           "cast_debug_inject_timeout", "cast_measure_tensor_peak", "cast_set_sparse_mode",
           "cast_get_sparse_mode", "cast_set_c128_tensor_mode", "cast_get_c128_tensor_mode",
           "cast_batch_create", "cast_batch_energy", "cast_batch_grad", "cast_batch_info", "cast_batch_destroy",
           "cast_measure_mma_issue")

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libcast.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libcast.so not found at {path}; run paper_2503_19894_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "cast_sv_create": (I, [I, I, P, PP]),
        "cast_sv_wrap": (I, [P, I, I, P, PP]),
        "cast_sv_destroy": (I, [P]),
        "cast_sv_info": (I, [P, P, P, P]),
        "cast_sv_set_basis": (I, [P, U64]),
        "cast_sv_copy_to_host": (I, [P, P]),
        "cast_sv_copy_from_host": (I, [P, P]),
        "cast_sv_copy_from_host_async": (I, [P, P]),
        "cast_apply_gate": (I, [P, P, I, P]),
        "cast_options_default": (None, [P]),
        "cast_apply_circuit": (I, [P, P, P, P]),
        "cast_fuse": (I, [P, P, P, P, P, P, P, P]),
        "cast_opcount": (ctypes.c_int64, [P, I, D]),
        "cast_expectation": (I, [P, P, P]),
        "cast_adjoint_grad": (I, [P, P, P, P, P, P, P]),
        "cast_last_error": (ctypes.c_char_p, []),
        "cast_version": (ctypes.c_char_p, []),
        "cast_plan_create": (I, [P, P, P, I, PP]),
        "cast_plan_apply": (I, [P, P]),
        "cast_plan_info": (I, [P, P, P]),
        "cast_plan_destroy": (I, [P]),
        "cast_profile_begin": (I, []),
        "cast_profile_end": (I, [P, P]),
        "cast_expectation_noalloc": (I, [P, P, P]),
        "cast_set_tensor_mode": (I, [I]),
        "cast_get_tensor_mode": (I, []),
        "cast_hea_create": (I, [I, P, I, I, I, P, PP]),
        "cast_hea_energy": (I, [P, P, D, D, P]),
        "cast_hea_grad": (I, [P, P, D, D, P, P]),
        "cast_hea_info": (I, [P, P, P]),
        "cast_hea_destroy": (I, [P]),
        "cast_set_f64_mode": (I, [I]),
        "cast_get_f64_mode": (I, []),
        "cast_autotune": (I, [I, I, P, P]),
        "cast_set_cost_table": (I, [P]),
        "cast_debug_inject_timeout": (I, [ctypes.c_uint32]),
        "cast_measure_tensor_peak": (I, [I, P]),
        "cast_measure_mma_issue": (I, [I, I, P]),
        "cast_set_sparse_mode": (I, [I]),
        "cast_get_sparse_mode": (I, []),
        "cast_set_c128_tensor_mode": (I, [I]),
        "cast_get_c128_tensor_mode": (I, []),
        "cast_batch_create": (I, [I, P, P, P, I, I, P, PP]),
        "cast_batch_energy": (I, [P, P, P]),
        "cast_batch_grad": (I, [P, P, P, P]),
        "cast_batch_info": (I, [P, P, P]),
        "cast_batch_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise CastError(status, load().cast_last_error().decode())


def _dt(dtype):
    if isinstance(dtype, int):
        return dtype
    return DTYPES[str(dtype).replace("torch.", "")]


def _amp_np(dt):
    return np.complex64 if dt == CAST_C64 else np.complex128


# ----------------------------------------------------------------- states

def cast_sv_create(n_qubits, dtype, stream=0):
    h = ctypes.c_void_p()
    _check(load().cast_sv_create(n_qubits, _dt(dtype), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def cast_sv_wrap(device_ptr, n_qubits, dtype, stream=0):
    h = ctypes.c_void_p()
    _check(load().cast_sv_wrap(ctypes.c_void_p(device_ptr), n_qubits, _dt(dtype),
                               ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def cast_sv_destroy(sv):
    _check(load().cast_sv_destroy(ctypes.c_void_p(sv)))


def cast_sv_info(sv):
    n, dt, ptr = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(load().cast_sv_info(ctypes.c_void_p(sv), ctypes.byref(n), ctypes.byref(dt), ctypes.byref(ptr)))
    return n.value, dt.value, ptr.value


def cast_sv_set_basis(sv, index):
    _check(load().cast_sv_set_basis(ctypes.c_void_p(sv), ctypes.c_uint64(index)))


def cast_sv_copy_to_host(sv, out=None):
    n, dt, _ = cast_sv_info(sv)
    if out is None:
        out = np.empty(1 << n, dtype=_amp_np(dt))
    if out.dtype != _amp_np(dt) or out.size != (1 << n) or not out.flags.c_contiguous:
        raise ValueError("host buffer must be a contiguous array of the state's size and type")
    _check(load().cast_sv_copy_to_host(ctypes.c_void_p(sv), ctypes.c_void_p(out.ctypes.data)))
    return out


def cast_sv_copy_from_host(sv, host):
    n, dt, _ = cast_sv_info(sv)
    arr = np.ascontiguousarray(host, dtype=_amp_np(dt))
    if arr.size != (1 << n):
        raise ValueError("host buffer size differs from the state's")
    _check(load().cast_sv_copy_from_host(ctypes.c_void_p(sv), ctypes.c_void_p(arr.ctypes.data)))


def cast_sv_copy_from_host_async(sv, host):
    """Queue the host-to-device copy on the state's stream and return.  `host`
    must already be a contiguous array of the state's amplitude type (no
    temporary copy is made: the buffer must outlive the queued copy), and
    page-locked for the copy to run asynchronously."""
    n, dt, _ = cast_sv_info(sv)
    if not isinstance(host, np.ndarray) or host.dtype != _amp_np(dt) or not host.flags["C_CONTIGUOUS"]:
        raise ValueError("host must be a contiguous numpy array of the state's amplitude type")
    if host.size != (1 << n):
        raise ValueError("host buffer size differs from the state's")
    _check(load().cast_sv_copy_from_host_async(ctypes.c_void_p(sv), ctypes.c_void_p(host.ctypes.data)))


# ------------------------------------------------------------------ gates

def cast_apply_gate(sv, qubits, matrix):
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    m = np.ascontiguousarray(matrix, dtype=np.complex128)
    _check(load().cast_apply_gate(ctypes.c_void_p(sv), ctypes.c_void_p(q.ctypes.data), int(q.size),
                                  ctypes.c_void_p(m.ctypes.data)))


class _Circuit:
    """Keeps the ctypes arrays of a marshalled circuit alive."""

    def __init__(self, n, gates, n_params):
        self.gates = (cast_gate * max(1, len(gates)))()
        self.mats = []
        for i, g in enumerate(gates):
            cg = self.gates[i]
            cg.kind = GATE_KIND[g.name]
            cg.k = len(g.qubits)
            for j in range(CAST_MAX_K):
                cg.qubits[j] = g.qubits[j] if j < len(g.qubits) else 0
            cg.param_index = int(g.pidx)
            for j in range(3):
                cg.params[j] = g.params[j] if j < len(g.params) else 0.0
            if g.name == "U":
                m = np.ascontiguousarray(g.matrix, dtype=np.complex128)
                self.mats.append(m)
                cg.matrix = m.ctypes.data
            else:
                cg.matrix = None
        self.c = cast_circuit(n, len(gates), self.gates, n_params)


def options(fusion="adaptive", max_k=5, agglomerative=True, op_cap=4096, zero_tol=1e-12,
            amp_ops_per_pass=0, cost=None):
    """cost: a cast_cost_table (from cast_autotune or cost_table()); the
    options object keeps it alive."""
    o = cast_options()
    load().cast_options_default(ctypes.byref(o))
    o.fusion = {"none": 0, "size": 1, "adaptive": 2}[fusion] if isinstance(fusion, str) else fusion
    o.max_k, o.agglomerative, o.op_cap = max_k, int(bool(agglomerative)), op_cap
    o.zero_tol, o.amp_ops_per_pass = zero_tol, amp_ops_per_pass
    if cost is not None:
        o._cost_ref = cost
        o.cost = ctypes.pointer(cost)
    return o


def cost_table(ms, dtype="c64", n_qubits=0, blocks_per_sm=None, sparse_floor_ms=None, sparse_ms_per_op=None):
    """A cast_cost_table from nested lists ms[k][class] (k = 0..7; class 0
    identity, 1 diagonal, 2 monomial, 3 dense) and, optionally, the sparse
    kernel's per-k floor and time per operation."""
    t = cast_cost_table()
    t.n_qubits, t.dtype = n_qubits, _dt(dtype)
    for k in range(CAST_MAX_K + 1):
        for c in range(4):
            t.ms[k][c] = float(ms[k][c])
            t.blocks_per_sm[k][c] = int(blocks_per_sm[k][c]) if blocks_per_sm is not None else 0
        t.sparse_floor_ms[k] = float(sparse_floor_ms[k]) if sparse_floor_ms is not None else 0.0
        t.sparse_ms_per_op[k] = float(sparse_ms_per_op[k]) if sparse_ms_per_op is not None else 0.0
    return t


def cost_table_dict(t):
    """The table as plain lists (the form oracle.fusion takes)."""
    return {"ms": [[t.ms[k][c] for c in range(4)] for k in range(CAST_MAX_K + 1)],
            "sparse_floor_ms": [t.sparse_floor_ms[k] for k in range(CAST_MAX_K + 1)],
            "sparse_ms_per_op": [t.sparse_ms_per_op[k] for k in range(CAST_MAX_K + 1)]}


def cast_autotune(dtype, n_qubits, stream=0):
    t = cast_cost_table()
    _check(load().cast_autotune(_dt(dtype), int(n_qubits), ctypes.c_void_p(stream), ctypes.byref(t)))
    return t


def cast_set_cost_table(table):
    _check(load().cast_set_cost_table(ctypes.byref(table) if table is not None else None))


def _params_arr(params):
    if params is None:
        return None, 0
    p = np.ascontiguousarray(params, dtype=np.float64)
    return p, int(p.size)


def cast_apply_circuit(sv, n, gates, params=None, opts=None):
    p, npar = _params_arr(params)
    circ = _Circuit(n, gates, npar)
    o = opts if opts is not None else options()
    _check(load().cast_apply_circuit(ctypes.c_void_p(sv), ctypes.byref(circ.c),
                                     ctypes.c_void_p(p.ctypes.data if p is not None else None),
                                     ctypes.byref(o)))


def cast_fuse(n, gates, params=None, opts=None):
    """Run the host fusion pass; returns a list of (qubits, matrix, opcount)."""
    p, npar = _params_arr(params)
    circ = _Circuit(n, gates, npar)
    o = opts if opts is not None else options()
    cap = max(1, len(gates))
    ks = np.zeros(cap, dtype=np.int32)
    qs = np.zeros(cap * CAST_MAX_K, dtype=np.int32)
    ops = np.zeros(cap, dtype=np.int64)
    slot = 1 << (2 * CAST_MAX_K)
    mats = np.zeros(cap * slot, dtype=np.complex128)
    nout = ctypes.c_int(cap)
    _check(load().cast_fuse(ctypes.byref(circ.c), ctypes.c_void_p(p.ctypes.data if p is not None else None),
                            ctypes.byref(o), ctypes.byref(nout), ctypes.c_void_p(ks.ctypes.data),
                            ctypes.c_void_p(qs.ctypes.data), ctypes.c_void_p(ops.ctypes.data),
                            ctypes.c_void_p(mats.ctypes.data)))
    out = []
    for g in range(nout.value):
        k = int(ks[g])
        d = 1 << k
        out.append((tuple(int(x) for x in qs[g * CAST_MAX_K:g * CAST_MAX_K + k]),
                    mats[g * slot:g * slot + d * d].reshape(d, d).copy(), int(ops[g])))
    return out


def cast_plan_create(n, gates, params=None, opts=None, dtype="c64"):
    p, npar = _params_arr(params)
    circ = _Circuit(n, gates, npar)
    o = opts if opts is not None else options()
    h = ctypes.c_void_p()
    _check(load().cast_plan_create(ctypes.byref(circ.c),
                                   ctypes.c_void_p(p.ctypes.data if p is not None else None),
                                   ctypes.byref(o), _dt(dtype), ctypes.byref(h)))
    return h.value


def cast_plan_apply(sv, plan):
    _check(load().cast_plan_apply(ctypes.c_void_p(sv), ctypes.c_void_p(plan)))


def cast_plan_info(plan):
    n, ops = ctypes.c_int(), ctypes.c_int64()
    _check(load().cast_plan_info(ctypes.c_void_p(plan), ctypes.byref(n), ctypes.byref(ops)))
    return n.value, ops.value


def cast_plan_destroy(plan):
    _check(load().cast_plan_destroy(ctypes.c_void_p(plan)))


def cast_profile_begin():
    _check(load().cast_profile_begin())


def cast_profile_end(capacity=256):
    """Returns [{name, launches, ms, bytes, flops}], largest total time first."""
    arr = (cast_profile_entry * capacity)()
    n = ctypes.c_int(capacity)
    _check(load().cast_profile_end(arr, ctypes.byref(n)))
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, ms=arr[i].ms,
                 bytes=arr[i].bytes, flops=arr[i].flops) for i in range(n.value)]


CAST_PATH_DIGIT, CAST_PATH_LIST, CAST_PATH_TENSOR_CHUNKED, CAST_PATH_TENSOR, CAST_PATH_DOUBLE_FLOAT, \
    CAST_PATH_CUDA_CORE = range(6)


def cast_gate_path(n, dtype, qubits, matrix):
    """The kernel family (CAST_PATH_*) cast_apply_gate takes for this gate on
    an n-qubit state of the given type under the current modes; host only."""
    m = np.ascontiguousarray(matrix, dtype=np.complex128)
    k = len(qubits)
    q = (ctypes.c_int * k)(*[int(x) for x in qubits])
    out = ctypes.c_int()
    _check(load().cast_gate_path(int(n), _dt(dtype), q, k, ctypes.c_void_p(m.ctypes.data), ctypes.byref(out)))
    return out.value


def cast_opcount(matrix, zero_tol=0.0):
    m = np.ascontiguousarray(matrix, dtype=np.complex128)
    k = int(m.shape[0]).bit_length() - 1
    return int(load().cast_opcount(ctypes.c_void_p(m.ctypes.data), k, zero_tol))


# ---------------------------------------------------------- observables

_PAULI_BITS = {"X": (1, 0), "Y": (1, 1), "Z": (0, 1)}


class _Pauli:
    def __init__(self, terms):
        self.coeffs = np.array([t.coeff for t in terms], dtype=np.float64)
        xm, zm = [], []
        for t in terms:
            x = z = 0
            for p, q in zip(t.paulis, t.qubits):
                bx, bz = _PAULI_BITS[p]
                x |= bx << q
                z |= bz << q
            xm.append(x)
            zm.append(z)
        self.x = np.array(xm, dtype=np.uint64)
        self.z = np.array(zm, dtype=np.uint64)
        self.s = cast_pauli_sum(len(terms), self.coeffs.ctypes.data if len(terms) else None,
                                self.x.ctypes.data if len(terms) else None,
                                self.z.ctypes.data if len(terms) else None)


def cast_expectation(sv, terms):
    h = _Pauli(terms)
    out = ctypes.c_double()
    _check(load().cast_expectation(ctypes.c_void_p(sv), ctypes.byref(h.s), ctypes.byref(out)))
    return out.value


def cast_expectation_noalloc(sv, terms):
    """<psi|H|psi> with the scratch in the library's fixed device array (no
    allocation; see cast.h)."""
    h = _Pauli(terms)
    out = ctypes.c_double()
    _check(load().cast_expectation_noalloc(ctypes.c_void_p(sv), ctypes.byref(h.s), ctypes.byref(out)))
    return out.value


def cast_adjoint_grad(psi, lam, n, gates, params, terms):
    """Returns (energy, gradient array)."""
    p, npar = _params_arr(params)
    circ = _Circuit(n, gates, npar)
    h = _Pauli(terms)
    energy = ctypes.c_double()
    grad = np.zeros(max(1, npar), dtype=np.float64)
    _check(load().cast_adjoint_grad(ctypes.c_void_p(psi), ctypes.c_void_p(lam), ctypes.byref(circ.c),
                                    ctypes.c_void_p(p.ctypes.data if p is not None else None),
                                    ctypes.byref(h.s), ctypes.byref(energy),
                                    ctypes.c_void_p(grad.ctypes.data)))
    return energy.value, grad[:npar]


CAST_TC_OFF, CAST_TC_TF32X3, CAST_TC_BF16X6 = 0, 1, 2
CAST_F64_EMULATED, CAST_F64_NATIVE = 0, 1


def cast_set_f64_mode(mode):
    _check(load().cast_set_f64_mode(int(mode)))


def cast_get_f64_mode():
    return int(load().cast_get_f64_mode())


def cast_set_tensor_mode(mode):
    _check(load().cast_set_tensor_mode(int(mode)))


def cast_get_tensor_mode():
    return int(load().cast_get_tensor_mode())


CAST_PEAK_TF32, CAST_PEAK_BF16 = 0, 1
CAST_SPARSE_AUTO, CAST_SPARSE_OFF, CAST_SPARSE_ALWAYS = 0, 1, 2


def cast_set_sparse_mode(mode):
    _check(load().cast_set_sparse_mode(int(mode)))


def cast_get_sparse_mode():
    return int(load().cast_get_sparse_mode())


CAST_C128_TC_OFF, CAST_C128_TC_OZAKI = 0, 1


def cast_set_c128_tensor_mode(mode):
    _check(load().cast_set_c128_tensor_mode(int(mode)))


def cast_get_c128_tensor_mode():
    return int(load().cast_get_c128_tensor_mode())


def cast_measure_tensor_peak(kind=CAST_PEAK_TF32):
    """Measured dense tensor-pipe TFLOP/s of the current GPU (kind::tf32 or bf16)."""
    v = ctypes.c_double()
    _check(load().cast_measure_tensor_peak(int(kind), ctypes.byref(v)))
    return float(v.value)


def cast_measure_mma_issue(n_cols, a_in_tmem=True):
    """SM clock cycles per back-to-back kind::f16 MMA of M = 128, K = 16, N = n_cols."""
    v = ctypes.c_double()
    _check(load().cast_measure_mma_issue(int(n_cols), int(bool(a_in_tmem)), ctypes.byref(v)))
    return float(v.value)


# --------------------------------------------- batched hardware-efficient ansatz

def cast_hea_create(n_qubits, layers, dtype="c64", with_grad=False, stream=0):
    n = np.ascontiguousarray(n_qubits, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().cast_hea_create(int(n.size), ctypes.c_void_p(n.ctypes.data), int(layers), _dt(dtype),
                                  int(bool(with_grad)), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def cast_hea_info(b):
    npar, npass = ctypes.c_int(), ctypes.c_int()
    _check(load().cast_hea_info(ctypes.c_void_p(b), ctypes.byref(npar), ctypes.byref(npass)))
    return npar.value, npass.value


def cast_hea_energy(b, params, zz, hx, n_instances):
    p = np.ascontiguousarray(params, dtype=np.float64)
    e = np.zeros(n_instances, dtype=np.float64)
    _check(load().cast_hea_energy(ctypes.c_void_p(b), ctypes.c_void_p(p.ctypes.data), float(zz), float(hx),
                                  ctypes.c_void_p(e.ctypes.data)))
    return e


def cast_hea_grad(b, params, zz, hx, n_instances):
    p = np.ascontiguousarray(params, dtype=np.float64)
    e = np.zeros(n_instances, dtype=np.float64)
    g = np.zeros(p.size, dtype=np.float64)
    _check(load().cast_hea_grad(ctypes.c_void_p(b), ctypes.c_void_p(p.ctypes.data), float(zz), float(hx),
                                ctypes.c_void_p(e.ctypes.data), ctypes.c_void_p(g.ctypes.data)))
    return e, g


def cast_hea_destroy(b):
    _check(load().cast_hea_destroy(ctypes.c_void_p(b)))


def cast_debug_inject_timeout(wait_limit):
    _check(load().cast_debug_inject_timeout(int(wait_limit)))


def cast_last_error():
    return load().cast_last_error().decode()


def cast_version():
    return load().cast_version().decode()


# ------------------------------------------- batched circuits of any shape

class Batch:
    """A cast_batch: instances = [(n_qubits, gates, n_params, terms)], each
    instance's parameters one after the other in the parameter array (or at
    param_offsets)."""

    def __init__(self, instances, dtype="c64", with_grad=False, param_offsets=None, stream=0):
        self._circs = [_Circuit(n, gates, npar) for n, gates, npar, _ in instances]
        self._hams = [_Pauli(terms) for _, _, _, terms in instances]
        circ_arr = (cast_circuit * len(instances))(*[c.c for c in self._circs])
        ham_arr = (cast_pauli_sum * len(instances))(*[h.s for h in self._hams])
        offs = None
        if param_offsets is not None:
            self._offs = np.ascontiguousarray(param_offsets, dtype=np.int32)
            offs = ctypes.c_void_p(self._offs.ctypes.data)
        h = ctypes.c_void_p()
        _check(load().cast_batch_create(len(instances), ctypes.byref(circ_arr), offs, ctypes.byref(ham_arr),
                                        _dt(dtype), int(bool(with_grad)), ctypes.c_void_p(stream), ctypes.byref(h)))
        self.handle = h.value
        self.n_instances = len(instances)
        npar, nsteps = ctypes.c_int(), ctypes.c_int()
        _check(load().cast_batch_info(ctypes.c_void_p(self.handle), ctypes.byref(npar), ctypes.byref(nsteps)))
        self.n_params, self.n_steps = npar.value, nsteps.value

    def energy(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        e = np.zeros(self.n_instances)
        _check(load().cast_batch_energy(ctypes.c_void_p(self.handle), ctypes.c_void_p(p.ctypes.data if p.size else None),
                                        ctypes.c_void_p(e.ctypes.data)))
        return e

    def grad(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        e = np.zeros(self.n_instances)
        g = np.zeros(max(1, self.n_params))
        _check(load().cast_batch_grad(ctypes.c_void_p(self.handle), ctypes.c_void_p(p.ctypes.data if p.size else None),
                                      ctypes.c_void_p(e.ctypes.data), ctypes.c_void_p(g.ctypes.data)))
        return e, g[:self.n_params]

    def close(self):
        if self.handle:
            _check(load().cast_batch_destroy(ctypes.c_void_p(self.handle)))
            self.handle = None
