"""The oracle: a plain, slow, obviously correct FP64 CPU state-vector simulator.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__ and
bench.py's CPU-baseline leg (and its reference arm) may import this package.
It shares no code with the CUDA library in paper_2503_19894_gb300/ and never
imports it; the two meet only in the seeded generators of `workloads`.

What each function follows:
  apply_gate / simulate   Eq. 1-3 (Section II-A): a k-qubit gate is 2^(n-k)
                          matrix-vector products on gathered amplitudes; the
                          gathering is the naive enumeration in sv_oracle.c
  expectation             <psi|H|psi> for a Pauli sum, by applying each Pauli
                          string to a copy of psi and taking the inner product
  grad_param_shift        exact gradient of E(theta) for rotations
                          exp(-i theta P / 2): [E(t + pi/2) - E(t - pi/2)] / 2
  grad_finite_diff        central differences [E(t + h) - E(t - h)] / (2 h)

Every gate is applied unfused, one at a time, in FP64.  Pins that hold this
code to the paper and to mathematics rather than to itself are in
tests/test_oracle.py; fusion (Section IV, Algorithm 1) has its own reference in
oracle/fusion.py.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import gates as G

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force=False):
    """Compile sv_oracle.c with gcc (OpenMP when the compiler supports it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_apply_gate.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
        lib.orc_apply_gate.restype = ctypes.c_int
        lib.orc_apply_gates.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
        lib.orc_apply_gates.restype = ctypes.c_int
        lib.orc_inner.argtypes = [P, P, ctypes.c_int, P, P]
        lib.orc_inner.restype = None
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads():
    return _load().orc_num_threads()


def _nqubits(psi):
    n = int(psi.size).bit_length() - 1
    if psi.dtype != np.complex128 or (1 << n) != psi.size or not psi.flags.c_contiguous:
        raise ValueError("state must be a contiguous complex128 array of length 2^n")
    return n


def basis_state(n, index=0):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def apply_gate(psi, qubits, mat):
    """Apply one gate in place (Eq. 3).  Bit i of the matrix index <-> qubits[i]."""
    n = _nqubits(psi)
    k = len(qubits)
    m = np.ascontiguousarray(mat, dtype=np.complex128)
    if m.shape != (1 << k, 1 << k):
        raise ValueError("matrix shape does not match the number of qubits")
    q = np.asarray(qubits, dtype=np.int32)
    rc = _load().orc_apply_gate(psi.ctypes.data, n, q.ctypes.data, k, m.ctypes.data)
    if rc != 0:
        raise ValueError(f"bad gate on qubits {tuple(qubits)} for n={n}")
    return psi


def gate_matrix(g, theta=None):
    """Matrix of a workloads.Gate; parametrised rotations read theta[g.pidx]."""
    if g.pidx >= 0:
        return G.matrix(g.name, (float(theta[g.pidx]),))
    return G.matrix(g.name, tuple(g.params), g.matrix)


def apply_circuit(psi, gates, theta=None):
    """Apply every gate of a workloads gate list, unfused, in order."""
    n = _nqubits(psi)
    if not gates:
        return psi
    ks = np.array([len(g.qubits) for g in gates], dtype=np.int32)
    qs = np.array([q for g in gates for q in g.qubits], dtype=np.int32)
    mats = np.concatenate([gate_matrix(g, theta).ravel() for g in gates])
    mats = np.ascontiguousarray(mats, dtype=np.complex128)
    rc = _load().orc_apply_gates(psi.ctypes.data, n, len(gates), ks.ctypes.data,
                                 qs.ctypes.data, mats.ctypes.data)
    if rc != 0:
        raise ValueError(f"bad gate #{-rc - 1}")
    return psi


def simulate(n, gates, init_index=0, theta=None):
    """|psi> = U_G ... U_1 |init_index>."""
    return apply_circuit(basis_state(n, init_index), gates, theta)


def inner(a, b):
    """<a|b> in FP64."""
    n = _nqubits(a)
    _nqubits(b)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_inner(a.ctypes.data, b.ctypes.data, n, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def apply_pauli(psi, paulis, qubits):
    """P|psi> for a Pauli string, as a new array (one 2x2 gate per factor)."""
    out = psi.copy()
    for p, q in zip(paulis, qubits):
        apply_gate(out, (q,), G.matrix(p))
    return out


def expectation(psi, terms):
    """<psi|H|psi> = sum_t c_t <psi|P_t|psi> (real for Hermitian H)."""
    total = 0.0
    for t in terms:
        total += t.coeff * inner(psi, apply_pauli(psi, t.paulis, t.qubits)).real
    return total


def z_string_partial(chunk, offset, qubits):
    """The part of <psi|Z_q1 ... Z_qm|psi> carried by the amplitudes
    psi[offset : offset + len(chunk)]:
        sum_x |psi_x|^2 prod_q (1 - 2 bit_q(x)),
    in FP64.  A Z string is diagonal, so the full value is the sum of these
    parts over any split of the index range: states too large to hold twice
    on the host are checked a slice at a time (<Z_0> of a 30-qubit state)."""
    c = np.asarray(chunk).astype(np.complex128)
    x = np.arange(offset, offset + c.size, dtype=np.int64)
    sign = np.ones(c.size, dtype=np.float64)
    for q in qubits:
        sign *= 1.0 - 2.0 * ((x >> q) & 1)
    return float(np.sum((c.real * c.real + c.imag * c.imag) * sign))


def energy(n, gates, theta, terms):
    return expectation(simulate(n, gates, theta=theta), terms)


def grad_param_shift(n, gates, theta, terms, indices=None):
    """dE/dtheta_p = [E(theta_p + pi/2) - E(theta_p - pi/2)] / 2, exact for
    gates exp(-i theta P / 2) when each parameter drives one gate."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = list(range(theta.size)) if indices is None else list(indices)
    g = np.zeros(len(idx))
    for j, p in enumerate(idx):
        tp = theta.copy(); tp[p] += np.pi / 2
        tm = theta.copy(); tm[p] -= np.pi / 2
        g[j] = 0.5 * (energy(n, gates, tp, terms) - energy(n, gates, tm, terms))
    return g


def grad_finite_diff(n, gates, theta, terms, h=1e-6, indices=None):
    """Central differences [E(theta_p + h) - E(theta_p - h)] / (2 h)."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = list(range(theta.size)) if indices is None else list(indices)
    g = np.zeros(len(idx))
    for j, p in enumerate(idx):
        tp = theta.copy(); tp[p] += h
        tm = theta.copy(); tm[p] -= h
        g[j] = (energy(n, gates, tp, terms) - energy(n, gates, tm, terms)) / (2 * h)
    return g
