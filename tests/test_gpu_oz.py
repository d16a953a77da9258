"""complex128 dense gates on the tensor cores (7-bit digits, exact integer
products; CAST_C128_TC_OZAKI) against the FP64 oracle: every target
placement for k = 3..7 (k = 6, 7 on the K-chunked kernel), rows whose
amplitudes span many orders of magnitude, digits at their largest, long gate
sequences, fused circuits, full-size 30-qubit gates, and the kernel choice
(profiled kernel families)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture
def oz_mode():
    old = capi.cast_get_c128_tensor_mode()
    capi.cast_set_c128_tensor_mode(capi.CAST_C128_TC_OZAKI)
    yield capi
    capi.cast_set_c128_tensor_mode(old)


def run_gate(n, psi0, qubits, m):
    sv = pkg.StateVector(n, "c128", init_index=None)
    sv.from_numpy(psi0)
    capi.cast_profile_begin()
    sv.apply_gate(qubits, m)
    prof = capi.cast_profile_end()
    out = sv.to_numpy()
    sv.close()
    return out, [p["name"] for p in prof]


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7])
def test_oz_gate_every_placement(k, oz_mode):
    rng = np.random.default_rng(300 + k)
    for n in (k + 7, k + 8, 16):
        psi0 = W.random_state(n, n * k)
        for placement in ("low", "high", "mixed", "mixed"):
            qs = W.sweep_targets(n, k, placement, rng)
            u = W.haar_unitary(k, rng)
            got, fams = run_gate(n, psi0, qs, u)
            ref = oracle.apply_gate(psi0.copy(), qs, u)
            assert fams == [f"ozdense_k{k}_c128"], fams
            assert np.max(np.abs(got - ref)) <= TOL, f"n={n} {qs}"
            assert rel_err(got, ref) <= 1e-13


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7])
def test_oz_rows_of_widely_spread_magnitudes(k, oz_mode):
    """Amplitudes from 1e-9 to 1 in one slice: the row exponent follows the
    largest, and the smallest still come out within the absolute bound."""
    n = k + 8
    rng = np.random.default_rng(11)
    mag = 10.0 ** rng.uniform(-9, 0, 1 << n)
    psi0 = mag * np.exp(2j * np.pi * rng.uniform(size=1 << n))
    psi0[rng.integers(0, 1 << n, 64)] = 0.0  # exact zeros too
    qs = W.sweep_targets(n, k, "mixed", rng)
    u = W.haar_unitary(k, rng)
    got, _ = run_gate(n, psi0, qs, u)
    ref = oracle.apply_gate(psi0.copy(), qs, u)
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(psi0)) * 10


@pytest.mark.parametrize("k,qs", [(4, (0, 5, 9, 12)), (7, (0, 2, 5, 8, 9, 12, 14))])
def test_oz_non_unitary_and_scaled_matrix(k, qs, oz_mode):
    """The split needs no unitarity: dense matrices with entries from 1e-6
    to 10."""
    n = 15
    rng = np.random.default_rng(5 + k)
    d = 1 << k
    m = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) * 10.0 ** rng.uniform(-6, 1, (d, d))
    psi0 = W.random_state(n, 8)
    got, fams = run_gate(n, psi0, qs, m)
    ref = oracle.apply_gate(psi0.copy(), qs, m)
    assert fams == [f"ozdense_k{k}_c128"]
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref)) * 10


def test_oz_k7_digits_at_their_largest(oz_mode):
    """Every digit of every input and entry at 127 with one sign (inputs and
    entries 1 - 2^-49 times a power of two): the products of weight 2^-28
    sum past 2^24 over K = 256, the one place where an accumulator can round
    (at most 2^-44 of sum |x w|); the result stays within 1e-12 of the
    largest output."""
    k, n = 7, 14
    d = 1 << k
    big = 1.0 - 2.0 ** -49
    m = np.full((d, d), big * 0.5 + 0.5j * big, dtype=np.complex128)
    psi0 = np.full(1 << n, big * 0.25 * (1 + 1j), dtype=np.complex128)
    qs = (1, 3, 4, 6, 9, 10, 13)
    got, fams = run_gate(n, psi0, qs, m)
    ref = oracle.apply_gate(psi0.copy(), qs, m)
    assert fams == ["ozdense_k7_c128"]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_oz_long_sequence(oz_mode):
    """300 Haar gates of k = 3..5 on 14 qubits (k = 3 on the CUDA cores):
    errors stay at the FP64 level and the norm does not drift."""
    n = 14
    rng = np.random.default_rng(21)
    gates = [W.Gate("U", W.sweep_targets(n, k, ("low", "high", "mixed")[i % 3], rng),
                    matrix=W.haar_unitary(k, rng)) for i, k in enumerate(rng.integers(3, 6, 300))]
    psi0 = W.random_state(n, 2)
    ref = oracle.apply_circuit(psi0.copy(), gates)
    sv = pkg.StateVector(n, "c128", init_index=None)
    sv.from_numpy(psi0)
    sv.apply_circuit(gates, fusion="none")
    norm = sv.expectation([W.PauliTerm(1.0, "", ())])
    got = sv.to_numpy()
    sv.close()
    assert np.max(np.abs(got - ref)) <= TOL
    assert rel_err(got, ref) <= 1e-12
    assert abs(norm - 1.0) <= 1e-12


def test_oz_long_sequence_k6_k7(oz_mode):
    """80 Haar gates of k = 6, 7 on 15 qubits: errors stay at the FP64 level
    and the norm does not drift."""
    n = 15
    rng = np.random.default_rng(23)
    gates = [W.Gate("U", W.sweep_targets(n, k, ("low", "high", "mixed")[i % 3], rng),
                    matrix=W.haar_unitary(k, rng)) for i, k in enumerate(rng.integers(6, 8, 80))]
    psi0 = W.random_state(n, 3)
    ref = oracle.apply_circuit(psi0.copy(), gates)
    sv = pkg.StateVector(n, "c128", init_index=None)
    sv.from_numpy(psi0)
    capi.cast_profile_begin()
    sv.apply_circuit(gates, fusion="none")
    fams = {p["name"] for p in capi.cast_profile_end()}
    norm = sv.expectation([W.PauliTerm(1.0, "", ())])
    got = sv.to_numpy()
    sv.close()
    assert fams == {"ozdense_k6_c128", "ozdense_k7_c128"}, fams
    assert np.max(np.abs(got - ref)) <= TOL
    assert rel_err(got, ref) <= 1e-12
    assert abs(norm - 1.0) <= 1e-12


@pytest.mark.parametrize("fam", ["RQC", "QVC", "QFT"])
@pytest.mark.parametrize("fusion,max_k", [("adaptive", 5), ("size", 7)])
def test_oz_fused_circuits(fam, fusion, max_k, oz_mode):
    n = 16
    gates = W.benchmark_family(fam, n, seed=3)[:500]
    ref = oracle.simulate(n, gates, init_index=7)
    sv = pkg.StateVector(n, "c128", init_index=7)
    sv.apply_circuit(gates, fusion=fusion, max_k=max_k)
    got = sv.to_numpy()
    sv.close()
    assert np.max(np.abs(got - ref)) <= TOL
    assert rel_err(got, ref) <= 1e-12


def test_oz_sparse_gates_stay_on_the_sparse_kernel(oz_mode):
    k, n = 5, 13  # two entries per row: 3% of the dense count, below the 11% crossover (5% for k = 7)
    d = 1 << k
    m = np.zeros((d, d), dtype=np.complex128)
    for r in range(d):
        m[r, r] = 0.6
        m[r, (r + 5) % d] = 0.8j
    psi0 = W.random_state(n, 4)
    got, fams = run_gate(n, psi0, (1, 3, 6, 8, 11), m)
    assert fams == ["sparse_k5_c128"]
    assert np.max(np.abs(got - oracle.apply_gate(psi0.copy(), (1, 3, 6, 8, 11), m))) <= TOL
    k, d = 7, 128
    m = np.zeros((d, d), dtype=np.complex128)
    for r in range(d):
        m[r, r] = 0.6
        m[r, (r + 37) % d] = 0.8j
    qs = (0, 2, 4, 5, 7, 10, 12)
    psi0 = W.random_state(14, 6)
    got, fams = run_gate(14, psi0, qs, m)
    assert fams == ["sparse_k7_c128"]
    assert np.max(np.abs(got - oracle.apply_gate(psi0.copy(), qs, m))) <= TOL


@pytest.mark.parametrize("k", [5, 7])
def test_oz_full_size_basis_column(k, oz_mode):
    """30 qubits (16 GiB): a Haar gate on |x> reproduces the matrix column,
    and its adjoint restores |x>."""
    n = 30
    rng = np.random.default_rng(77 + k)
    qs = W.sweep_targets(n, k, "mixed", rng)
    u = W.haar_unitary(k, rng)
    x = int(rng.integers(0, 1 << n))
    sv = pkg.StateVector(n, "c128", init_index=x)
    sv.apply_gate(qs, u)
    jx = sum(((x >> q) & 1) << i for i, q in enumerate(qs))
    base = x & ~sum(1 << q for q in qs)
    idx = np.array([base | sum(((j >> i) & 1) << q for i, q in enumerate(qs)) for j in range(1 << k)])
    t = torch.as_tensor(idx, dtype=torch.int64, device=sv.tensor.device)
    got = sv.tensor.index_select(0, t).cpu().numpy()
    assert np.max(np.abs(got - u[:, jx])) <= TOL
    sv.apply_gate(qs, u.conj().T)
    back = sv.tensor.index_select(0, torch.as_tensor([x], device=sv.tensor.device)).cpu().numpy()
    assert abs(back[0] - 1.0) <= 10 * TOL
    sv.close()
    torch.cuda.empty_cache()


def test_oz_mode_validation():
    with pytest.raises(capi.CastError):
        capi.cast_set_c128_tensor_mode(5)
