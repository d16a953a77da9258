"""Seeded synthetic workloads: circuit descriptions, parameters, Hamiltonians.

This module is shared by the oracle and the GPU library's callers.  It holds no
state-vector arithmetic: it only draws random numbers and writes down gate
lists (names, qubits, angles) and Pauli sums.  Each side turns a gate name into
a matrix with its own gate table.

Workload shapes follow the paper's benchmark families (Section VI-A: QFT,
random quantum circuits, ...) and the single-gate table (Section VI-C); the
exact instances are not published, so seeded stand-ins are generated here:

  random_circuit   per layer one gate per qubit drawn from {H, X, RX, RY, RZ}
                   (angles U(0, 2 pi)), then CX on a random perfect matching
  qft_circuit      H plus controlled-phase pi/2^(j-m) on every pair, then swaps
  haar_unitary     2^k x 2^k Haar-random unitary (QR of a complex Ginibre
                   matrix with the phase fix of Mezzadri, 2007)
  gate_sweep       dense k-qubit Haar gates on low / high / mixed targets
  hea_ansatz       hardware-efficient ansatz: RY on all, RZ on all, CZ ladder
  tfim_hamiltonian sum Z_i Z_{i+1} + h sum X_i (open boundary)
  vqa_batch        many ansatz instances of uneven qubit counts
  ala_circuit      alternating layered ansatz: U3 on every qubit, then CZ on
                   the even or odd neighbour pairs, alternating by layer
  qvc_circuit      quantum-volume-shaped circuit: per layer a random pairing,
                   each pair a random two-qubit block of the generic
                   three-CX shape (four U3 layers around three CX)
  iqp_circuit      instantaneous quantum polynomial: H on all, diagonal
                   rounds (RZ on all, CP on a random matching), H on all
  hes_circuit      first-order Trotter steps of the 1-D Heisenberg chain
                   sum (XX + YY + ZZ) + h sum Z, each bond term as basis
                   change + CX + RZ + CX
  benchmark_family one of the six families of the paper by name

The paper names the six families (QFT, ALA, RQC, QVC, IQP, HES) and splits
them into a sparse class (QFT, RQC, IQP, HES) and a dense class (ALA, QVC,
mostly dense single-qubit gates) but gives no instance; the shapes above are
the cited constructions written as gate lists.
"""
import math
from typing import NamedTuple, Optional

import numpy as np


class Gate(NamedTuple):
    """One gate of a circuit description.

    name   : "H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "U3", "CX", "CZ",
             "CP", "SWAP", or "U" (explicit matrix in `matrix`)
    qubits : tuple of qubit indices; bit i of the matrix index <-> qubits[i];
             for CX / CZ / CP the first qubit is the control
    params : fixed angles (RX/RY/RZ/CP: one, U3: three)
    pidx   : index into a parameter vector for a parametrised rotation
             (then `params` is empty), or -1
    matrix : explicit 2^k x 2^k complex128 matrix for name "U"
    """
    name: str
    qubits: tuple
    params: tuple = ()
    pidx: int = -1
    matrix: Optional[np.ndarray] = None


class PauliTerm(NamedTuple):
    """coeff * prod_i P_i on qubits[i], P_i in {"X", "Y", "Z"}."""
    coeff: float
    paulis: str
    qubits: tuple


ONE_QUBIT_CHOICES = ("H", "X", "RX", "RY", "RZ")


def random_circuit(n, layers, seed):
    """Random layered circuit: per layer a uniform pick from {H, X, RX, RY, RZ}
    on every qubit (rotation angles U(0, 2 pi)), then CX on a random perfect
    matching of the qubits (pairs (p[2i], p[2i+1]) of a random permutation p,
    control first; with odd n one qubit is left out)."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(layers):
        picks = rng.integers(0, len(ONE_QUBIT_CHOICES), size=n)
        angles = rng.uniform(0.0, 2.0 * math.pi, size=n)
        for q in range(n):
            name = ONE_QUBIT_CHOICES[picks[q]]
            params = (float(angles[q]),) if name.startswith("R") else ()
            gates.append(Gate(name, (q,), params))
        perm = rng.permutation(n)
        for i in range(n // 2):
            gates.append(Gate("CX", (int(perm[2 * i]), int(perm[2 * i + 1]))))
    return gates


def qft_circuit(n):
    """Quantum Fourier transform on n qubits (qubit 0 = least significant).

    For j = n-1 down to 0: H on j, then CP(pi / 2^(j-m)) on (m, j) for
    m = j-1 down to 0; finally SWAP(i, n-1-i).  Maps |x> to
    2^(-n/2) sum_y exp(+2 pi i x y / 2^n) |y>."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("H", (j,)))
        for m in range(j - 1, -1, -1):
            gates.append(Gate("CP", (m, j), (math.pi / float(1 << (j - m)),)))
    for i in range(n // 2):
        gates.append(Gate("SWAP", (i, n - 1 - i)))
    return gates


def random_basis_index(n, seed):
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, 1 << n))


def haar_unitary(k, rng):
    """2^k x 2^k Haar-random unitary: QR of a complex Ginibre matrix, then
    multiply column j of Q by r_jj / |r_jj| (Mezzadri 2007, Section 5)."""
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :])


def sweep_targets(n, k, placement, rng):
    """Target set for the dense-gate sweep: 'low' = 0..k-1, 'high' = the top k
    qubits, 'mixed' = a random k-subset in random order."""
    if placement == "low":
        return tuple(range(k))
    if placement == "high":
        return tuple(range(n - k, n))
    if placement == "mixed":
        return tuple(int(x) for x in rng.choice(n, size=k, replace=False))
    raise ValueError(placement)


def gate_sweep(n, k, placement, count, seed):
    """`count` Haar-random k-qubit gates on `placement` targets."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        qs = sweep_targets(n, k, placement, rng)
        out.append(Gate("U", qs, matrix=haar_unitary(k, rng)))
    return out


def hea_ansatz(n, layers):
    """Hardware-efficient ansatz.  Layer l: RY(theta[2nl + q]) on every qubit q,
    RZ(theta[2nl + n + q]) on every qubit q, then CZ(i, i+1) for i < n-1.
    Returns (gates, number of parameters = 2 n layers)."""
    gates = []
    for l in range(layers):
        for q in range(n):
            gates.append(Gate("RY", (q,), pidx=2 * n * l + q))
        for q in range(n):
            gates.append(Gate("RZ", (q,), pidx=2 * n * l + n + q))
        for i in range(n - 1):
            gates.append(Gate("CZ", (i, i + 1)))
    return gates, 2 * n * layers


def uniform_params(count, low, high, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=count)


def tfim_hamiltonian(n, hx):
    """Transverse-field Ising model, open boundary:
    H = sum_{i<n-1} Z_i Z_{i+1} + hx * sum_i X_i."""
    terms = [PauliTerm(1.0, "ZZ", (i, i + 1)) for i in range(n - 1)]
    terms += [PauliTerm(float(hx), "X", (i,)) for i in range(n)]
    return terms


def z0_observable():
    return [PauliTerm(1.0, "Z", (0,))]


def vqa_batch(count, n_min, n_max, layers, seed):
    """`count` ansatz instances with qubit counts U{n_min..n_max}; parameters
    U(-pi, pi).  Returns a list of (n, gates, params)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_min, n_max + 1, size=count)
    out = []
    for n in ns:
        gates, npar = hea_ansatz(int(n), layers)
        params = rng.uniform(-math.pi, math.pi, size=npar)
        out.append((int(n), gates, params))
    return out


def random_state(n, seed):
    """Normalised complex Gaussian state (interleaved complex128)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def random_state_device(n, dtype, seed):
    """Normalised complex Gaussian state of 2^n amplitudes drawn directly on
    the current CUDA device with torch's seeded generator (for states too
    large to draw on the host).  dtype: "c64" or "c128"."""
    import torch
    real = torch.float32 if dtype == "c64" else torch.float64
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    re = torch.randn(1 << n, generator=g, device="cuda", dtype=real)
    im = torch.randn(1 << n, generator=g, device="cuda", dtype=real)
    psi = torch.complex(re, im)
    del re, im
    psi /= torch.linalg.vector_norm(psi)
    return psi


def _u3_angles(rng, count):
    return rng.uniform(0.0, 2.0 * math.pi, size=(count, 3))


def ala_circuit(n, layers, seed):
    """Alternating layered ansatz (Cerezo et al. 2021, the ALA family): layer
    l applies U3(theta, phi, lambda) with angles U(0, 2 pi) to every qubit,
    then CZ(i, i+1) for every i with i = l (mod 2), i + 1 < n: two-qubit
    blocks in a brick pattern whose offset alternates between layers."""
    rng = np.random.default_rng(seed)
    gates = []
    for l in range(layers):
        ang = _u3_angles(rng, n)
        for q in range(n):
            gates.append(Gate("U3", (q,), tuple(float(a) for a in ang[q])))
        for i in range(l % 2, n - 1, 2):
            gates.append(Gate("CZ", (i, i + 1)))
    return gates


def qvc_circuit(n, layers, seed):
    """Quantum-volume-shaped circuit (Cross et al. 2019, the QVC family): per
    layer a random permutation p pairs the qubits (p[2i], p[2i+1]); each pair
    gets a random two-qubit block of the generic shape
        U3 x U3, CX(a, b), U3 x U3, CX(b, a), U3 x U3, CX(a, b), U3 x U3
    with U3 angles U(0, 2 pi) (random blocks of the three-CX form rather than
    Haar-distributed SU(4), so the circuit is mostly dense 1-qubit gates)."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(layers):
        perm = rng.permutation(n)
        for i in range(n // 2):
            a, b = int(perm[2 * i]), int(perm[2 * i + 1])
            ang = _u3_angles(rng, 8)
            for r in range(4):
                gates.append(Gate("U3", (a,), tuple(float(v) for v in ang[2 * r])))
                gates.append(Gate("U3", (b,), tuple(float(v) for v in ang[2 * r + 1])))
                if r < 3:
                    gates.append(Gate("CX", (a, b) if r != 1 else (b, a)))
    return gates


def iqp_circuit(n, layers, seed, zero_phases=False):
    """Instantaneous quantum polynomial circuit (Bremner, Montanaro and
    Shepherd 2017, the IQP family): H on every qubit, then `layers` diagonal
    rounds, each RZ(theta) on every qubit and CP(phi) on a random perfect
    matching (angles U(0, 2 pi)), then H on every qubit.  With zero_phases
    every angle is 0 and the circuit is the identity."""
    rng = np.random.default_rng(seed)
    gates = [Gate("H", (q,)) for q in range(n)]
    for _ in range(layers):
        th = rng.uniform(0.0, 2.0 * math.pi, size=n)
        for q in range(n):
            gates.append(Gate("RZ", (q,), (0.0 if zero_phases else float(th[q]),)))
        perm = rng.permutation(n)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=n // 2)
        for i in range(n // 2):
            gates.append(Gate("CP", (int(perm[2 * i]), int(perm[2 * i + 1])), (0.0 if zero_phases else float(ph[i]),)))
    gates += [Gate("H", (q,)) for q in range(n)]
    return gates


def hes_bond(a, b, pauli, angle):
    """exp(-i (angle / 2) P_a P_b) for P in {X, Y, Z} as a gate list: a basis
    change to Z (H for X; RX(pi/2) for Y), CX(a, b), RZ(angle) on b, CX(a, b),
    and the basis change undone."""
    pre, post = [], []
    if pauli == "X":
        pre = [Gate("H", (a,)), Gate("H", (b,))]
        post = list(pre)
    elif pauli == "Y":
        pre = [Gate("RX", (a,), (math.pi / 2,)), Gate("RX", (b,), (math.pi / 2,))]
        post = [Gate("RX", (a,), (-math.pi / 2,)), Gate("RX", (b,), (-math.pi / 2,))]
    core = [Gate("CX", (a, b)), Gate("RZ", (b,), (float(angle),)), Gate("CX", (a, b))]
    return pre + core + post


def hes_circuit(n, steps, dt=0.1, field=0.5, paulis="XYZ"):
    """Hamiltonian evolution simulation (Low and Chuang 2017, the HES family)
    as first-order Trotter steps of the open 1-D Heisenberg chain
        H = sum_i (X_i X_{i+1} + Y_i Y_{i+1} + Z_i Z_{i+1}) + field sum_i Z_i:
    per step, for every bond (i, i+1) and P in `paulis`, exp(-i dt P_i P_{i+1})
    (hes_bond with angle 2 dt), then RZ(2 dt field) on every qubit, i.e.
    exp(-i dt field Z_i).  The initial state is the caller's."""
    gates = []
    for _ in range(steps):
        for i in range(n - 1):
            for p in paulis:
                gates += hes_bond(i, i + 1, p, 2.0 * dt)
        if field:
            gates += [Gate("RZ", (q,), (2.0 * dt * field,)) for q in range(n)]
    return gates


# name -> (generator(n, seed), class): the six benchmark families at the
# sizes the fusion ablation runs (layers chosen so every family has a few
# hundred to two thousand gates at 30 qubits)
FAMILIES = {
    "QFT": (lambda n, seed: qft_circuit(n), "sparse"),
    "RQC": (lambda n, seed: random_circuit(n, 30, seed), "sparse"),
    "IQP": (lambda n, seed: iqp_circuit(n, 10, seed), "sparse"),
    "HES": (lambda n, seed: hes_circuit(n, 2), "sparse"),
    "ALA": (lambda n, seed: ala_circuit(n, 10, seed), "dense"),
    "QVC": (lambda n, seed: qvc_circuit(n, 10, seed), "dense"),
}


def benchmark_family(name, n, seed=1):
    """Gate list of one of the paper's six benchmark families."""
    return FAMILIES[name][0](n, seed)
