"""Pins for the oracle: closed forms, invariants and brute force (CPU only).

None of these re-types the oracle's own loop.  The brute-force references
build the full 2^n x 2^n operator either literally as Eq. 1's Kronecker product
(numpy.kron) or from the textbook definition of an operator acting on a
subsystem, and multiply it into the state with a dense matmul.
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import gates as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- references

def kron_lift_1q(n, q, u):
    """Eq. 1 literally: I^(n-q-1) (x) U (x) I^q."""
    return np.kron(np.kron(np.eye(1 << (n - q - 1)), u), np.eye(1 << q))


def lift(n, qubits, u):
    """Full operator of a k-qubit gate from the definition of a subsystem
    operator: <r|U_full|c> = U[loc(r), loc(c)] when r and c agree on every
    non-target bit, else 0; loc(x) collects bit qubits[i] of x into bit i."""
    N = 1 << n
    idx = np.arange(N)
    tmask = sum(1 << q for q in qubits)
    loc = np.zeros(N, dtype=np.int64)
    for i, q in enumerate(qubits):
        loc |= ((idx >> q) & 1) << i
    same = ((idx[:, None] ^ idx[None, :]) & ~tmask) == 0
    return np.where(same, u[loc[:, None], loc[None, :]], 0)


def brute_force(n, gates, init=0, theta=None):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[init] = 1
    for g in gates:
        psi = lift(n, g.qubits, oracle.gate_matrix(g, theta)) @ psi
    return psi


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [1, 2, 5, 10, 14])
def test_hadamard_all_uniform(n):
    psi = oracle.simulate(n, [W.Gate("H", (q,)) for q in range(n)])
    assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_ghz(n):
    gates = [W.Gate("H", (0,))] + [W.Gate("CX", (0, i)) for i in range(1, n)]
    psi = oracle.simulate(n, gates)
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


def qft_closed_form(n, x):
    """QFT|x> = 2^(-n/2) sum_y exp(2 pi i ((x y) mod 2^n) / 2^n) |y>, with the
    product reduced modulo 2^n in exact integer arithmetic."""
    y = np.arange(1 << n, dtype=np.int64)
    ph = ((x * y) % (1 << n)).astype(np.float64) / float(1 << n)
    return np.exp(2j * np.pi * ph) / math.sqrt(1 << n)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (8, 4), (11, 5)])
def test_qft_of_basis_state(n, seed):
    x = W.random_basis_index(n, seed)
    psi = oracle.simulate(n, W.qft_circuit(n), init_index=x)
    assert np.max(np.abs(psi - qft_closed_form(n, x))) < 1e-13


def test_qft_gate_count():
    n = 30
    c = W.qft_circuit(n)
    assert sum(g.name == "H" for g in c) == 30
    assert sum(g.name == "CP" for g in c) == 435
    assert sum(g.name == "SWAP" for g in c) == 15


# ----------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 3, 6])
def test_eq1_kron_single_qubit(n):
    rng = np.random.default_rng(n)
    for q in range(n):
        u = W.haar_unitary(1, rng)
        psi0 = W.random_state(n, 10 + q)
        ref = kron_lift_1q(n, q, u) @ psi0
        out = oracle.apply_gate(psi0.copy(), (q,), u)
        assert np.max(np.abs(out - ref)) < 1e-14


def test_eq1_kron_adjacent_two_qubit():
    """Eq. 1 extended to adjacent qubits (q, q+1): I (x) U (x) I^q with bit 0 of
    U's index on qubit q; this fixes the local-bit order of two-qubit gates."""
    n = 5
    rng = np.random.default_rng(7)
    for q in range(n - 1):
        u = W.haar_unitary(2, rng)
        full = np.kron(np.kron(np.eye(1 << (n - q - 2)), u), np.eye(1 << q))
        psi0 = W.random_state(n, q)
        out = oracle.apply_gate(psi0.copy(), (q, q + 1), u)
        assert np.max(np.abs(out - full @ psi0)) < 1e-14


@pytest.mark.parametrize("n,layers,seed", [(4, 6, 0), (6, 5, 1), (8, 3, 2), (7, 4, 3)])
def test_random_circuit_brute_force(n, layers, seed):
    gates = W.random_circuit(n, layers, seed)
    assert np.max(np.abs(oracle.simulate(n, gates) - brute_force(n, gates))) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_haar_gate_arbitrary_targets_brute_force(k):
    n = 8
    rng = np.random.default_rng(100 + k)
    for placement in ("low", "high", "mixed"):
        qs = W.sweep_targets(n, k, placement, rng)
        u = W.haar_unitary(k, rng)
        psi0 = W.random_state(n, k)
        out = oracle.apply_gate(psi0.copy(), qs, u)
        assert np.max(np.abs(out - lift(n, qs, u) @ psi0)) < 1e-13


def test_textbook_gates_against_definitions():
    """Rotation gates equal exp(-i t P / 2) = cos(t/2) I - i sin(t/2) P; U3 at
    special angles reduces to H and X up to known phases."""
    t = 0.7315
    for name, P in (("RX", G.X()), ("RY", G.Y()), ("RZ", G.Z())):
        ref = math.cos(t / 2) * np.eye(2) - 1j * math.sin(t / 2) * P
        assert np.max(np.abs(G.matrix(name, (t,)) - ref)) < 1e-15
    assert np.max(np.abs(G.U3(math.pi / 2, 0, math.pi) - G.H())) < 1e-15
    assert np.max(np.abs(G.U3(math.pi, 0, math.pi) - G.X())) < 1e-15
    for m in (G.H(), G.CX(), G.CZ(), G.SWAP(), G.CP(0.3), G.U3(0.1, 0.2, 0.3)):
        assert np.max(np.abs(m.conj().T @ m - np.eye(m.shape[0]))) < 1e-15


def test_cx_control_is_first_qubit():
    # |control=1, target=0> = index 1 (qubit 0 is control) -> |11> = index 3
    psi = oracle.simulate(2, [W.Gate("X", (0,)), W.Gate("CX", (0, 1))])
    assert abs(psi[3] - 1) < 1e-15
    psi = oracle.simulate(2, [W.Gate("X", (1,)), W.Gate("CX", (0, 1))])
    assert abs(psi[2] - 1) < 1e-15  # control 0: target untouched


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("k", [1, 3, 5, 7])
def test_norm_preserved(k):
    n = 12
    rng = np.random.default_rng(k)
    psi = W.random_state(n, 5)
    for _ in range(6):
        qs = W.sweep_targets(n, k, "mixed", rng)
        oracle.apply_gate(psi, qs, W.haar_unitary(k, rng))
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13


def test_circuit_then_inverse_returns():
    n = 10
    gates = W.random_circuit(n, 8, 11)
    psi = oracle.simulate(n, gates, init_index=37)
    inv = [W.Gate("U", g.qubits, matrix=oracle.gate_matrix(g).conj().T) for g in reversed(gates)]
    oracle.apply_circuit(psi, inv)
    ref = oracle.basis_state(n, 37)
    assert np.max(np.abs(psi - ref)) < 1e-13


def test_qubit_order_of_matrix_respected():
    """Listing the same targets in another order with the matching permuted
    matrix gives the same result."""
    n = 6
    rng = np.random.default_rng(3)
    u = W.haar_unitary(3, rng)
    qs = (4, 1, 3)
    # reorder the qubits to (1, 3, 4): new local bit i <- old local bit perm[i]
    perm = [1, 2, 0]
    d = 8
    src = np.array([sum(((j >> i) & 1) << perm[i] for i in range(3)) for j in range(d)])
    u2 = u[src[:, None], src[None, :]]
    a = oracle.apply_gate(W.random_state(n, 1), qs, u)
    b = oracle.apply_gate(W.random_state(n, 1), (1, 3, 4), u2)
    assert np.max(np.abs(a - b)) < 1e-14


# --------------------------------------------------------- expectations

def test_z0_after_hadamard_is_zero():
    psi = oracle.simulate(4, [W.Gate("H", (0,))])
    assert abs(oracle.expectation(psi, W.z0_observable())) < 1e-15


def test_z0_closed_form_ry():
    for t in (0.0, 0.3, 1.9, -2.5):
        psi = oracle.simulate(3, [W.Gate("RY", (0,), (t,))])
        assert abs(oracle.expectation(psi, W.z0_observable()) - math.cos(t)) < 1e-15


@pytest.mark.parametrize("n,hx", [(5, 0.5), (8, 0.7)])
def test_tfim_special_states(n, hx):
    H = W.tfim_hamiltonian(n, hx)
    zero = oracle.basis_state(n)
    assert abs(oracle.expectation(zero, H) - (n - 1)) < 1e-14
    plus = oracle.simulate(n, [W.Gate("H", (q,)) for q in range(n)])
    assert abs(oracle.expectation(plus, H) - hx * n) < 1e-13


def test_z_string_partial_sums_to_expectation():
    """Split over three index ranges, the parts add up to <psi|Z..Z|psi> of the
    Pauli-string expectation (which applies Z factors as gates), and <Z_0>
    after H(0) on |0..0> is 0 while <Z_0> of |0..0> is 1."""
    n = 9
    psi = W.random_state(n, 4)
    for qs in ((0,), (3,), (0, 8), (1, 2, 7)):
        want = oracle.expectation(psi, [W.PauliTerm(1.0, "Z" * len(qs), qs)])
        cuts = [0, 100, 301, 1 << n]
        got = sum(oracle.z_string_partial(psi[a:b], a, qs) for a, b in zip(cuts[:-1], cuts[1:]))
        assert abs(got - want) < 1e-14
    plus = oracle.simulate(n, [W.Gate("H", (0,))])
    assert abs(oracle.z_string_partial(plus, 0, (0,))) < 1e-15
    assert oracle.z_string_partial(oracle.basis_state(n), 0, (0,)) == 1.0
    # a planted sign error (bit q counted as +1) is caught
    odd = oracle.basis_state(n, 1)
    assert oracle.z_string_partial(odd, 0, (0,)) == -1.0


def test_y_expectation_sign():
    # S H |0> = (|0> + i|1>)/sqrt2 is the +1 eigenstate of Y
    psi = oracle.simulate(1, [W.Gate("H", (0,)), W.Gate("S", (0,))])
    assert abs(oracle.expectation(psi, [W.PauliTerm(1.0, "Y", (0,))]) - 1.0) < 1e-15


def test_expectation_matches_dense_operator():
    n = 5
    psi = W.random_state(n, 9)
    terms = [W.PauliTerm(0.3, "XZ", (0, 3)), W.PauliTerm(-1.1, "YY", (1, 4)),
             W.PauliTerm(0.7, "ZXY", (2, 0, 4))]
    Hm = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t in terms:
        op = np.eye(1 << n, dtype=np.complex128)
        for p, q in zip(t.paulis, t.qubits):
            op = kron_lift_1q(n, q, G.matrix(p)) @ op
        Hm += t.coeff * op
    ref = np.vdot(psi, Hm @ psi).real
    assert abs(oracle.expectation(psi, terms) - ref) < 1e-14


# ------------------------------------------------------------- gradients

def test_gradient_closed_form_single_rotation():
    # E(t) = <0|RY(t)^dag Z RY(t)|0> = cos t
    gates = [W.Gate("RY", (0,), pidx=0)]
    for t in (0.4, 2.2):
        g = oracle.grad_param_shift(1, gates, np.array([t]), W.z0_observable())
        assert abs(g[0] + math.sin(t)) < 1e-15


def test_gradient_closed_form_two_parameters():
    # RY(a) then RX(b) on |0>: <Z> = cos a cos b
    gates = [W.Gate("RY", (0,), pidx=0), W.Gate("RX", (0,), pidx=1)]
    a, b = 0.7, -1.3
    g = oracle.grad_param_shift(1, gates, np.array([a, b]), W.z0_observable())
    assert abs(g[0] + math.sin(a) * math.cos(b)) < 1e-15
    assert abs(g[1] + math.cos(a) * math.sin(b)) < 1e-15


def test_param_shift_agrees_with_finite_differences():
    n, layers = 5, 2
    gates, npar = W.hea_ansatz(n, layers)
    theta = W.uniform_params(npar, -math.pi, math.pi, 4)
    H = W.tfim_hamiltonian(n, 0.7)
    idx = [0, 3, 7, 12, 19]
    ps = oracle.grad_param_shift(n, gates, theta, H, indices=idx)
    fd = oracle.grad_finite_diff(n, gates, theta, H, h=1e-6, indices=idx)
    assert np.max(np.abs(ps - fd)) < 1e-8


def test_hea_parameter_count():
    gates, npar = W.hea_ansatz(26, 20)
    assert npar == 1040
    assert len(gates) == 20 * (2 * 26 + 25)


# ---------------------------------------------------- paper's stated numbers

def opcount(mat, tol=0.0):
    """Operation count of Section IV-C: 2 x (number of non-zero real scalars)."""
    m = np.asarray(mat)
    return 2 * int(np.sum(np.abs(m.real) > tol) + np.sum(np.abs(m.imag) > tol))


def test_paper_operation_counts():
    with open(os.path.join(GOLDEN, "paper_opcounts.json")) as f:
        gold = json.load(f)
    for p in ("X", "Y", "Z"):
        assert opcount(G.matrix(p)) // 2 == gold["nonzero_scalars"][p]
    rng = np.random.default_rng(0)
    assert opcount(W.haar_unitary(1, rng)) // 2 == gold["nonzero_scalars"]["dense_1q"]
    for k in range(1, 8):
        assert opcount(W.haar_unitary(k, rng)) == gold["opcount_dense"][str(k)]
    assert gold["opcount_dense"]["5"] == gold["opcount_cap_example"]


# --------------------------------------- planted mistakes must be caught

def test_planted_transposed_matrix_is_caught(monkeypatch):
    """A transposed gate matrix inside the oracle must fail the brute force."""
    real = oracle.apply_gate

    def transposed(psi, qubits, mat):
        return real(psi, qubits, np.asarray(mat).T.copy())

    n, gates = 5, W.random_circuit(5, 4, 21)
    ref = brute_force(n, gates)
    psi = oracle.basis_state(n)
    for g in gates:
        transposed(psi, g.qubits, oracle.gate_matrix(g))
    assert np.max(np.abs(psi - ref)) > 1e-3


def test_planted_reversed_qubit_order_is_caught():
    n, rng = 6, np.random.default_rng(5)
    qs, u = (0, 4, 2), W.haar_unitary(3, rng)
    psi0 = W.random_state(n, 2)
    wrong = oracle.apply_gate(psi0.copy(), tuple(reversed(qs)), u)
    assert np.max(np.abs(wrong - lift(n, qs, u) @ psi0)) > 1e-3


def test_planted_wrong_qft_sign_is_caught():
    n, x = 6, 45
    gates = [W.Gate(g.name, g.qubits, tuple(-p for p in g.params)) for g in W.qft_circuit(n)]
    psi = oracle.simulate(n, gates, init_index=x)
    assert np.max(np.abs(psi - qft_closed_form(n, x))) > 1e-3


def test_oracle_rejects_bad_arguments():
    psi = oracle.basis_state(3)
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, (0, 0), np.eye(4))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, (3,), np.eye(2))
