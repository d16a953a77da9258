"""Textbook gate matrices for the oracle (FP64 complex).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.

The paper names its gates (H, U3 in the single-gate table of Section VI-C; the
QFT, random and Hamiltonian-evolution benchmark families of Section VI-A) but
prints no matrix, so the standard textbook forms are used:

  H  = [[1, 1], [1, -1]] / sqrt(2)
  X, Y, Z Pauli matrices;  S = diag(1, i);  T = diag(1, e^{i pi/4})
  RX(t) = exp(-i t X / 2),  RY(t) = exp(-i t Y / 2),  RZ(t) = exp(-i t Z / 2)
  U3(t, p, l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]]
  CX, CZ, CP(phi) = diag(1, 1, 1, e^{i phi}), SWAP

Local index convention (matches Eq. 1's little-endian qubit order): bit i of a
matrix row/column index belongs to the gate's i-th listed qubit.  For the
controlled gates the FIRST listed qubit is the control, so CX(c, t) flips the
target bit (local bit 1) of the states whose control bit (local bit 0) is 1.
"""
import math

import numpy as np

_SQ2 = 1.0 / math.sqrt(2.0)


def H():
    return np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=np.complex128)


def X():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def Y():
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def Z():
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def S():
    return np.array([[1, 0], [0, 1j]], dtype=np.complex128)


def T():
    return np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)


def RX(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def RY(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def RZ(t):
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)


def U3(t, p, l):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -np.exp(1j * l) * s],
                     [np.exp(1j * p) * s, np.exp(1j * (p + l)) * c]], dtype=np.complex128)


def CX():
    # local index j = b0 + 2*b1, b0 = control, b1 = target: swaps |01> <-> |11>
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[2, 2] = 1
    m[1, 3] = m[3, 1] = 1
    return m


def CZ():
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def CP(phi):
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def SWAP():
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[3, 3] = 1
    m[1, 2] = m[2, 1] = 1
    return m


_TABLE = {
    "H": (1, 0, H), "X": (1, 0, X), "Y": (1, 0, Y), "Z": (1, 0, Z),
    "S": (1, 0, S), "T": (1, 0, T),
    "RX": (1, 1, RX), "RY": (1, 1, RY), "RZ": (1, 1, RZ), "U3": (1, 3, U3),
    "CX": (2, 0, CX), "CZ": (2, 0, CZ), "CP": (2, 1, CP), "SWAP": (2, 0, SWAP),
}

# Generators of the rotation gates: R_P(t) = exp(-i t P / 2), used by the
# analytic-gradient references.
GENERATOR = {"RX": X, "RY": Y, "RZ": Z}


def arity(name):
    return _TABLE[name][0]


def matrix(name, params=(), explicit=None):
    """The 2^k x 2^k matrix of gate `name` (or `explicit` for name "U")."""
    if name == "U":
        return np.asarray(explicit, dtype=np.complex128)
    k, npar, fn = _TABLE[name]
    if len(params) != npar:
        raise ValueError(f"{name} takes {npar} parameters, got {len(params)}")
    return fn(*params)
