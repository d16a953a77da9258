"""The six benchmark families of Section VI-A as gate lists (workloads), run
through the oracle and pinned to things other than the oracle: brute-force
Kronecker products at n <= 6, the Walsh-Hadamard closed form of an IQP
circuit, exact exponentials of the Heisenberg bond terms (scipy's expm, a
library routine) and the first-order Trotter error of the HES family."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W
from oracle import gates as G
from tests.helpers import circuit_unitary

FAMS = sorted(W.FAMILIES)


@pytest.mark.parametrize("fam", FAMS)
def test_family_brute_force_small(fam):
    n = 6
    gates = W.benchmark_family(fam, n, seed=3)
    if len(gates) > 400:  # keep the dense products cheap
        gates = gates[:400]
    U = circuit_unitary(n, [(g.qubits, oracle.gate_matrix(g)) for g in gates])
    x = 5
    want = U[:, x]
    got = oracle.simulate(n, gates, init_index=x)
    assert np.max(np.abs(got - want)) < 1e-12


def test_family_classes_follow_the_paper():
    assert {f for f, (_, c) in W.FAMILIES.items() if c == "sparse"} == {"QFT", "RQC", "IQP", "HES"}
    assert {f for f, (_, c) in W.FAMILIES.items() if c == "dense"} == {"ALA", "QVC"}
    # the dense class is mostly dense single-qubit gates, the sparse class is not
    def dense1q_share(gs):
        return sum(1 for g in gs if g.name in ("U3", "H", "RX", "RY")) / len(gs)
    for f in ("ALA", "QVC"):
        assert dense1q_share(W.benchmark_family(f, 30)) > 0.6
    for f in ("IQP", "HES"):
        gs = W.benchmark_family(f, 30)
        assert sum(1 for g in gs if g.name in ("RZ", "CP", "CZ", "CX")) / len(gs) > 0.5


def test_ala_brick_pattern():
    n, layers = 7, 4
    gates = W.ala_circuit(n, layers, 0)
    cz = [g.qubits for g in gates if g.name == "CZ"]
    assert cz == [(0, 1), (2, 3), (4, 5), (1, 2), (3, 4), (5, 6)] * 2
    assert sum(1 for g in gates if g.name == "U3") == n * layers


def test_qvc_blocks_pair_every_qubit_once_per_layer():
    n = 8
    gates = W.qvc_circuit(n, 3, 4)
    per_layer = len(gates) // 3
    assert per_layer == (n // 2) * 11
    for l in range(3):
        layer = gates[l * per_layer:(l + 1) * per_layer]
        touched = [q for g in layer if g.name == "CX" for q in g.qubits]
        assert sorted(set(touched)) == list(range(n))
        assert len([g for g in layer if g.name == "CX"]) == 3 * (n // 2)


def _iqp_diagonal(n, gates):
    """d(x) of the diagonal part of an IQP gate list, from its angles."""
    x = np.arange(1 << n)
    d = np.ones(1 << n, dtype=np.complex128)
    for g in gates:
        if g.name == "RZ":
            b = (x >> g.qubits[0]) & 1
            d *= np.exp(1j * g.params[0] * (b - 0.5))
        elif g.name == "CP":
            b = ((x >> g.qubits[0]) & 1) & ((x >> g.qubits[1]) & 1)
            d *= np.where(b == 1, np.exp(1j * g.params[0]), 1.0)
    return d


@pytest.mark.parametrize("n,layers,seed", [(5, 1, 0), (7, 3, 1), (8, 2, 2)])
def test_iqp_walsh_hadamard_closed_form(n, layers, seed):
    """H^n D H^n |0>: psi(y) = 2^-n sum_x (-1)^{x.y} d(x)."""
    gates = W.iqp_circuit(n, layers, seed)
    d = _iqp_diagonal(n, gates)
    want = scipy.linalg.hadamard(1 << n) @ d / (1 << n)
    got = oracle.simulate(n, gates)
    assert np.max(np.abs(got - want)) < 1e-13


def test_iqp_zero_phases_is_identity():
    n = 9
    got = oracle.simulate(n, W.iqp_circuit(n, 3, 5, zero_phases=True), init_index=0)
    assert abs(got[0] - 1) < 1e-13 and np.max(np.abs(got[1:])) < 1e-13


def _pauli(p):
    return {"X": G.X(), "Y": G.Y(), "Z": G.Z()}[p]


@pytest.mark.parametrize("p", ["X", "Y", "Z"])
def test_hes_bond_is_the_exact_exponential(p):
    """The bond gate list equals exp(-i (angle/2) P (x) P) (both orders of the
    pair), from scipy's matrix exponential."""
    ang = 0.37
    for a, b in ((0, 1), (1, 0)):
        U = circuit_unitary(2, [(g.qubits, oracle.gate_matrix(g)) for g in W.hes_bond(a, b, p, ang)])
        PP = np.kron(_pauli(p), _pauli(p))
        assert np.max(np.abs(U - scipy.linalg.expm(-0.5j * ang * PP))) < 1e-14


def _heisenberg(n, field, paulis="XYZ"):
    N = 1 << n
    H = np.zeros((N, N), dtype=np.complex128)

    def op(ps):
        m = np.eye(1, dtype=np.complex128)
        for q in reversed(range(n)):  # bit q of the index <-> qubit q (Eq. 1)
            m = np.kron(m, ps.get(q, np.eye(2)))
        return m
    for i in range(n - 1):
        for p in paulis:
            H += op({i: _pauli(p), i + 1: _pauli(p)})
    for i in range(n):
        H += field * op({i: G.Z()})
    return H


def test_hes_commuting_terms_are_exact_in_one_step():
    """ZZ bonds and Z fields commute: one Trotter step is exp(-i dt H) exactly."""
    n, dt, field = 5, 0.3, 0.7
    psi0 = W.random_state(n, 2)
    got = oracle.apply_circuit(psi0.copy(), W.hes_circuit(n, 1, dt, field, paulis="Z"))
    want = scipy.linalg.expm(-1j * dt * _heisenberg(n, field, "Z")) @ psi0
    assert np.max(np.abs(got - want)) < 1e-13


def test_hes_trotter_error_is_first_order():
    """Full XYZ chain: the Trotter error at fixed t shrinks like 1/steps, and
    stays inside the first-order bound t^2 / (2 r) sum_{a<b} ||[H_a, H_b]||
    (crudely bounded by t^2 / (2 r) * (2 * terms^2), every ||H_a|| <= 1)."""
    n, t, field = 4, 0.8, 0.5
    psi0 = W.random_state(n, 6)
    want = scipy.linalg.expm(-1j * t * _heisenberg(n, field)) @ psi0
    errs = []
    for r in (20, 40, 80):
        got = oracle.apply_circuit(psi0.copy(), W.hes_circuit(n, r, t / r, field))
        errs.append(np.linalg.norm(got - want))
    terms = 3 * (n - 1) + n
    assert errs[0] <= t * t / (2 * 20) * 2 * terms * terms
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


def test_families_at_benchmark_size_have_expected_counts():
    counts = {f: len(W.benchmark_family(f, 30)) for f in FAMS}
    assert counts == {"ALA": 445, "HES": 1046, "IQP": 510, "QFT": 480, "QVC": 1650, "RQC": 1350}
