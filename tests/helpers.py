"""Test-only brute-force references (numpy), independent of oracle/ and of the
CUDA library."""
import numpy as np


def lift(n, qubits, u):
    """Full 2^n x 2^n operator of a gate on `qubits` from the definition of an
    operator on a subsystem: <r|U|c> = u[loc(r), loc(c)] if r, c agree off the
    targets, else 0 (bit i of loc(x) = bit qubits[i] of x)."""
    N = 1 << n
    idx = np.arange(N)
    tmask = sum(1 << q for q in qubits)
    loc = np.zeros(N, dtype=np.int64)
    for i, q in enumerate(qubits):
        loc |= ((idx >> q) & 1) << i
    same = ((idx[:, None] ^ idx[None, :]) & ~tmask) == 0
    return np.where(same, u[loc[:, None], loc[None, :]], 0)


def circuit_unitary(n, gate_mats):
    """Product of lifted gates; gate_mats = [(qubits, matrix), ...] in time order."""
    U = np.eye(1 << n, dtype=np.complex128)
    for qs, m in gate_mats:
        U = lift(n, qs, np.asarray(m)) @ U
    return U


def sorted_gate(qubits, m):
    """Re-express a gate with its qubits in ascending order."""
    k = len(qubits)
    order = sorted(range(k), key=lambda i: qubits[i])
    d = 1 << k
    old = np.array([sum(((j >> i) & 1) << order[i] for i in range(k)) for j in range(d)])
    return tuple(sorted(qubits)), np.asarray(m)[old[:, None], old[None, :]]


def rel_err(got, ref):
    """||got - ref||_2 / ||ref||_2: the error relative to the state's size,
    which stays meaningful when amplitudes are small (large n)."""
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


# Relative error bounds beside the absolute ones (complex128 1e-12, complex64
# 1e-5): complex128 results stay at the FP64 / double-float level, complex64
# results at a few FP32 units in the last place per gate, accumulated as a
# random walk over the circuit.
REL = {"c128": 1e-12, "c64": 2e-5}
