"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on seeded inputs.

Tolerances (maximum |delta amplitude|): 1e-12 for complex128 and 1e-5 for
complex64, fused or unfused.  Expectation values are compared within the same
bounds scaled by the sum of |coefficients|; adjoint gradients within 1e-10
(complex128) of the exact parameter-shift gradient.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import REL, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}
NP = {"c128": np.complex128, "c64": np.complex64}


def run_gate(n, dtype, psi0, qubits, m):
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(psi0.astype(NP[dtype]))
    sv.apply_gate(qubits, m)
    out = sv.to_numpy().astype(np.complex128)
    sv.close()
    return out


def oracle_gate(psi0, dtype, qubits, m):
    # the oracle starts from the same (rounded) input the GPU received
    return oracle.apply_gate(psi0.astype(NP[dtype]).astype(np.complex128), qubits, m)


def random_diag(k, rng):
    return np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k)))


def random_monomial(k, rng, unit=False):
    d = 1 << k
    perm = rng.permutation(d)
    m = np.zeros((d, d), dtype=np.complex128)
    ph = np.ones(d) if unit else np.exp(1j * rng.uniform(0, 2 * np.pi, d))
    m[np.arange(d), perm] = ph
    return m


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_dense_gate_all_placements(dtype, k):
    rng = np.random.default_rng(10 + k)
    for n in sorted({k, k + 1, k + 3, 13}):
        psi0 = W.random_state(n, n)
        for placement in ("low", "high", "mixed"):
            qs = W.sweep_targets(n, k, placement, rng)
            u = W.haar_unitary(k, rng)
            got = run_gate(n, dtype, psi0, qs, u)
            ref = oracle_gate(psi0, dtype, qs, u)
            err = np.max(np.abs(got - ref))
            assert err <= TOL[dtype], f"n={n} k={k} {placement} {qs}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("kind", ["diag", "mono", "mono_unit"])
def test_sparse_gate_classes(dtype, k, kind):
    rng = np.random.default_rng(100 * k + len(kind))
    n = max(k + 2, 11)
    psi0 = W.random_state(n, 3)
    for placement in ("low", "high", "mixed"):
        qs = W.sweep_targets(n, k, placement, rng)
        m = random_diag(k, rng) if kind == "diag" else random_monomial(k, rng, kind == "mono_unit")
        got = run_gate(n, dtype, psi0, qs, m)
        ref = oracle_gate(psi0, dtype, qs, m)
        assert np.max(np.abs(got - ref)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_diag_with_unit_entries_and_identity(dtype):
    n = 10
    psi0 = W.random_state(n, 4)
    for m, qs in ((oracle.gates.CP(0.3), (7, 2)), (oracle.gates.CZ(), (0, 9)),
                  (np.eye(4), (3, 4)), (oracle.gates.T(), (5,)), (oracle.gates.Z(), (0,))):
        got = run_gate(n, dtype, psi0, qs, m)
        assert np.max(np.abs(got - oracle_gate(psi0, dtype, qs, m))) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_diag_partial_identity_all_placements(dtype, k):
    """Diagonal gates with a random subset of identity entries: the kernel that
    enumerates only the non-identity amplitudes (lowest target >= 2) and the
    vector kernel (lowest target 0 or 1), small and multi-block states."""
    rng = np.random.default_rng(700 + k)
    for n in (k + 3, 12, 18):
        psi0 = W.random_state(n, n)
        for trial in range(4):
            low = [0, 1, 2, 3][trial]  # lowest target
            if low + k > n:
                continue
            rest = rng.choice(np.arange(low + 1, n), size=k - 1, replace=False) if k > 1 else []
            qs = tuple(int(q) for q in rng.permutation([low] + list(rest)))
            d = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k))
            keep = rng.random(1 << k) < 0.5
            keep[rng.integers(0, 1 << k)] = False  # at least one identity entry
            keep[rng.integers(0, 1 << k)] = True   # at least one phase
            d = np.where(keep, d, 1.0)
            got = run_gate(n, dtype, psi0, qs, np.diag(d))
            ref = oracle_gate(psi0, dtype, qs, np.diag(d))
            assert np.max(np.abs(got - ref)) <= TOL[dtype], (n, qs)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_config0_random_circuit_unfused(dtype):
    """12-qubit random circuit, 20 layers, from |0...0>, no fusion: full state
    and <Z_0>."""
    n = 12
    gates = W.random_circuit(n, 20, seed=0)
    ref = oracle.simulate(n, gates)
    sv = pkg.StateVector(n, dtype)
    sv.apply_circuit(gates, fusion="none")
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    z0 = sv.expectation(W.z0_observable())
    assert abs(z0 - oracle.expectation(ref, W.z0_observable())) <= TOL[dtype]
    sv.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode,max_k,agg", [("size", 2, True), ("size", 5, True), ("adaptive", 5, True),
                                            ("size", 7, False), ("adaptive", 7, True)])
def test_fused_random_circuit(dtype, mode, max_k, agg):
    n = 14
    gates = W.random_circuit(n, 12, seed=7)
    ref = oracle.simulate(n, gates)
    sv = pkg.StateVector(n, dtype)
    sv.apply_circuit(gates, fusion=mode, max_k=max_k, agglomerative=agg)
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    sv.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fused_qft_matches_closed_form(dtype):
    n = 16
    x = W.random_basis_index(n, 3)
    gates = W.qft_circuit(n)
    ref = oracle.simulate(n, gates, init_index=x)
    sv = pkg.StateVector(n, dtype, init_index=x)
    sv.apply_circuit(gates, fusion="adaptive", max_k=5)
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    sv.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_pauli_sums(dtype):
    n = 12
    psi0 = W.random_state(n, 8)
    terms = W.tfim_hamiltonian(n, 0.7) + [
        W.PauliTerm(0.3, "XZ", (0, 5)), W.PauliTerm(-1.1, "YY", (1, 11)),
        W.PauliTerm(0.7, "ZXY", (2, 0, 10)), W.PauliTerm(0.25, "Y", (6,)),
        W.PauliTerm(2.0, "", ())]
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(psi0.astype(NP[dtype]))
    got = sv.expectation(terms)
    ref = oracle.expectation(psi0.astype(NP[dtype]).astype(np.complex128), terms)
    scale = sum(abs(t.coeff) for t in terms)
    assert abs(got - ref) <= TOL[dtype] * scale
    sv.close()


def test_expectation_many_terms_split_across_launches():
    n = 10
    rng = np.random.default_rng(2)
    terms = [W.PauliTerm(float(rng.normal()), "ZZ", tuple(int(v) for v in rng.choice(n, 2, replace=False)))
             for _ in range(70)]
    psi0 = W.random_state(n, 1)
    sv = pkg.StateVector(n, "c128", init_index=None)
    sv.from_numpy(psi0)
    assert abs(sv.expectation(terms) - oracle.expectation(psi0, terms)) <= 1e-12 * 70
    sv.close()


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-10), ("c64", 2e-4)])
def test_adjoint_gradient_vs_parameter_shift(dtype, tol):
    n, layers = 8, 3
    gates, npar = W.hea_ansatz(n, layers)
    theta = W.uniform_params(npar, -math.pi, math.pi, 5)
    H = W.tfim_hamiltonian(n, 0.7)
    psi = pkg.StateVector(n, dtype)
    lam = pkg.StateVector(n, dtype, init_index=None)
    e, g = pkg.cast_adjoint_grad(psi.handle, lam.handle, n, gates, theta, H)
    # psi is returned to |0...0> by the uncomputation
    back = psi.to_numpy().astype(np.complex128)
    assert abs(back[0] - 1) < 100 * TOL[dtype] and np.max(np.abs(back[1:])) < 100 * TOL[dtype]
    ps = oracle.grad_param_shift(n, gates, theta, H)
    assert abs(e - oracle.energy(n, gates, theta, H)) <= tol
    assert np.max(np.abs(g - ps)) <= tol
    psi.close()
    lam.close()


def test_adjoint_mixed_gates_and_shared_parameters():
    """Fixed gates of every class between rotations, and one parameter driving
    two gates (its gradient is the sum of both contributions)."""
    n = 6
    gates = [W.Gate("H", (0,)), W.Gate("RX", (0,), pidx=0), W.Gate("CX", (0, 3)),
             W.Gate("RZ", (3,), pidx=1), W.Gate("SWAP", (1, 4)), W.Gate("RY", (4,), pidx=0),
             W.Gate("U", (2, 5, 1), matrix=W.haar_unitary(3, np.random.default_rng(0))),
             W.Gate("RY", (5,), pidx=2), W.Gate("CP", (5, 2), (0.4,))]
    theta = np.array([0.3, -1.2, 2.1])
    H = [W.PauliTerm(0.5, "ZX", (0, 4)), W.PauliTerm(-0.8, "Y", (5,)), W.PauliTerm(1.3, "ZZ", (2, 3))]
    psi = pkg.StateVector(n, "c128")
    lam = pkg.StateVector(n, "c128", init_index=None)
    e, g = pkg.cast_adjoint_grad(psi.handle, lam.handle, n, gates, theta, H)
    fd = oracle.grad_finite_diff(n, gates, theta, H, h=1e-6)
    assert abs(e - oracle.energy(n, gates, theta, H)) < 1e-12
    assert np.max(np.abs(g - fd)) < 1e-8
    psi.close()
    lam.close()


def test_autograd_function():
    import torch
    n, layers = 5, 2
    gates, npar = W.hea_ansatz(n, layers)
    H = W.tfim_hamiltonian(n, 0.5)
    theta = torch.tensor(W.uniform_params(npar, -1, 1, 9), dtype=torch.float64, requires_grad=True)
    e = pkg.AdjointEnergy.apply(theta, n, gates, H, "c128")
    e.backward()
    ps = oracle.grad_param_shift(n, gates, theta.detach().numpy(), H)
    assert np.max(np.abs(theta.grad.numpy() - ps)) < 1e-10


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_single_qubit_state_and_k_equals_n(dtype):
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 7):
        psi0 = W.random_state(n, n)
        u = W.haar_unitary(n, rng)
        qs = tuple(rng.permutation(n))
        got = run_gate(n, dtype, psi0, qs, u)
        assert np.max(np.abs(got - oracle_gate(psi0, dtype, qs, u))) <= TOL[dtype]


def test_basis_and_copy_roundtrip():
    for dtype in ("c128", "c64"):
        n = 9
        sv = pkg.StateVector(n, dtype, init_index=(1 << n) - 1)
        v = sv.to_numpy()
        assert v[-1] == 1 and np.count_nonzero(v) == 1
        psi0 = W.random_state(n, 2).astype(NP[dtype])
        sv.from_numpy(psi0)
        assert np.array_equal(sv.to_numpy(), psi0)
        sv.apply_circuit([], fusion="none")
        assert np.array_equal(sv.to_numpy(), psi0)
        sv.close()


def test_async_copy_double_buffered_on_two_streams():
    """Two states on two streams: each one's input is queued with
    cast_sv_copy_from_host_async while the other applies a circuit; every
    step's <Z_0> and amplitudes equal the synchronous path's."""
    import torch
    n = 16
    gates = W.random_circuit(n, 4, 5)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    svs = []
    for s in streams:
        with torch.cuda.stream(s):
            svs.append(pkg.StateVector(n, "c64", init_index=None))
    inputs = [torch.from_numpy(W.random_state(n, 10 + i).astype(np.complex64)).pin_memory() for i in range(4)]
    z0 = [W.PauliTerm(1.0, "Z", (0,))]
    capi.cast_sv_copy_from_host_async(svs[0].handle, inputs[0].numpy())
    for i in range(4):
        cur, nxt = svs[i % 2], svs[(i + 1) % 2]
        if i + 1 < 4:
            capi.cast_sv_copy_from_host_async(nxt.handle, inputs[i + 1].numpy())
        cur.apply_circuit(gates, fusion="adaptive")
        z = cur.expectation(z0)
        want = oracle.apply_circuit(inputs[i].numpy().astype(np.complex128), gates)
        assert abs(z - oracle.expectation(want, z0)) < 1e-5
        assert np.max(np.abs(cur.to_numpy() - want)) < 1e-5
    with pytest.raises(ValueError):  # a temporary copy would not outlive the queued copy
        capi.cast_sv_copy_from_host_async(svs[0].handle, inputs[0].numpy().astype(np.complex128))
    for sv in svs:
        sv.close()


def test_errors_are_reported_not_raised_on_device():
    sv = pkg.StateVector(4, "c128")
    with pytest.raises(capi.CastError):
        sv.apply_gate((0, 4), np.eye(4))
    with pytest.raises(capi.CastError):
        sv.apply_gate((0, 0), np.eye(4))
    with pytest.raises(capi.CastError):
        sv.set_basis(16)
    with pytest.raises(capi.CastError):
        sv.apply_gate((0,), np.array([[np.nan, 0], [0, 1]]))
    # the state is untouched by the rejected calls
    v = sv.to_numpy()
    assert v[0] == 1 and np.count_nonzero(v) == 1
    sv.close()


def test_library_owned_state_create_destroy():
    h = capi.cast_sv_create(10, "c64")
    n, dt, ptr = capi.cast_sv_info(h)
    assert (n, dt) == (10, capi.CAST_C64) and ptr % 256 == 0
    capi.cast_apply_gate(h, (3,), oracle.gates.H())
    v = capi.cast_sv_copy_to_host(h)
    assert abs(v[0] - 2 ** -0.5) < 1e-7 and abs(v[8] - 2 ** -0.5) < 1e-7
    capi.cast_sv_destroy(h)


# ------------------------------------------------- tensor-core dense gates

@pytest.fixture
def tensor_mode():
    old = capi.cast_get_tensor_mode()
    yield capi
    capi.cast_set_tensor_mode(old)


@pytest.mark.parametrize("k", [4, 5, 6, 7])
def test_tensor_core_gate_matches_oracle(k, tensor_mode):
    """3xTF32 tcgen05 path (complex64, k = 4..7, n >= k + 7): every placement,
    a single-tile state, states with one tile per CTA, and at 22 qubits
    several tiles per CTA with ragged shares (the pipelines that carry a
    tile's accumulator or epilogue into the next tile)."""
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    rng = np.random.default_rng(500 + k)
    for n in (k + 7, k + 8, 16, 19, 22):
        psi0 = W.random_state(n, n + k)
        places = ("low", "high", "mixed", "mixed", "mixed") if n < 22 else ("low", "mixed")
        for placement in places:
            qs = W.sweep_targets(n, k, placement, rng)
            u = W.haar_unitary(k, rng)
            got = run_gate(n, "c64", psi0, qs, u)
            ref = oracle_gate(psi0, "c64", qs, u)
            err = np.max(np.abs(got - ref))
            assert err <= TOL["c64"], f"n={n} {qs}: {err:.3e}"
            # one gate: a few fp32 units relative to the state
            assert rel_err(got, ref) <= 1e-6, f"n={n} {qs}: rel {rel_err(got, ref):.3e}"


def test_tensor_core_and_fp32_paths_both_match_oracle(tensor_mode):
    """The 3xTF32 tensor-core path and the FP32 CUDA-core path, each against
    the oracle, in absolute and relative terms."""
    n = 18
    rng = np.random.default_rng(9)
    psi0 = W.random_state(n, 4)
    for k in (4, 5, 6):
        qs = W.sweep_targets(n, k, "mixed", rng)
        u = W.haar_unitary(k, rng)
        ref = oracle_gate(psi0, "c64", qs, u)
        for mode in (capi.CAST_TC_TF32X3, capi.CAST_TC_OFF):
            capi.cast_set_tensor_mode(mode)
            got = run_gate(n, "c64", psi0, qs, u)
            assert np.max(np.abs(got - ref)) <= TOL["c64"]
            assert rel_err(got, ref) <= 1e-6, (k, mode, rel_err(got, ref))


def test_tensor_core_fused_circuit(tensor_mode):
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    n = 16
    gates = W.random_circuit(n, 16, seed=12)
    ref = oracle.simulate(n, gates)
    sv = pkg.StateVector(n, "c64")
    sv.apply_circuit(gates, fusion="size", max_k=5)
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL["c64"]
    sv.close()


@pytest.mark.parametrize("k", [4, 5, 6, 7])
def test_tensor_core_norm_does_not_drift(k, tensor_mode):
    """400 Haar k-qubit gates on the tensor cores: the per-slice norm
    restoration leaves unbiased noise, so the norm stays at 1 (a bias of the
    size of the tensor cores' truncation, ~2^-23 per gate, would move it by
    ~1e-4) and the state stays within the complex64 bound of the oracle."""
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    n = 17
    rng = np.random.default_rng(900 + k)
    gates = [W.Gate("U", W.sweep_targets(n, k, ("low", "high", "mixed")[i % 3], rng),
                    matrix=W.haar_unitary(k, rng)) for i in range(400)]
    psi0 = W.random_state(n, 17)
    ref = oracle.apply_circuit(psi0.copy(), gates)
    sv = pkg.StateVector(n, "c64", init_index=None)
    sv.from_numpy(psi0.astype(np.complex64))
    sv.apply_circuit(gates, fusion="none")
    assert abs(sv.expectation([W.PauliTerm(1.0, "", ())]) - 1.0) <= 1e-5
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL["c64"]
    # relative to the state, the error is a random walk of fp32-sized steps
    assert np.linalg.norm(got - ref) <= 2e-5
    sv.close()


def test_tensor_mode_validation(tensor_mode):
    with pytest.raises(capi.CastError):
        capi.cast_set_tensor_mode(7)


@pytest.mark.parametrize("dtype,k", [("c64", 7), ("c128", 6), ("c64", 6)])
def test_many_large_gates_wrap_the_matrix_ring(dtype, k, tensor_mode):
    """Gates whose matrices go through the device ring (16 slots): 40 in a row."""
    n = 13
    rng = np.random.default_rng(77 + k)
    psi0 = W.random_state(n, 6)
    gates = [W.Gate("U", W.sweep_targets(n, k, "mixed", rng), matrix=W.haar_unitary(k, rng)) for _ in range(40)]
    ref = oracle.apply_circuit(psi0.astype(NP[dtype]).astype(np.complex128), gates)
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(psi0.astype(NP[dtype]))
    sv.apply_circuit(gates, fusion="none")
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    assert rel_err(got, ref) <= REL[dtype]
    sv.close()


# ------------------------------------------------- complex128 arithmetic modes

@pytest.fixture
def f64_mode():
    old = capi.cast_get_f64_mode()
    yield capi
    capi.cast_set_f64_mode(old)


@pytest.mark.parametrize("mode", ["emulated", "native"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_complex128_modes_match_oracle(mode, k, f64_mode):
    capi.cast_set_f64_mode(capi.CAST_F64_EMULATED if mode == "emulated" else capi.CAST_F64_NATIVE)
    rng = np.random.default_rng(900 + k)
    n = 13
    psi0 = W.random_state(n, 11)
    for placement in ("low", "high", "mixed"):
        qs = W.sweep_targets(n, k, placement, rng)
        for m in (W.haar_unitary(k, rng), random_diag(k, rng), random_monomial(k, rng)):
            got = run_gate(n, "c128", psi0, qs, m)
            assert np.max(np.abs(got - oracle_gate(psi0, "c128", qs, m))) <= 1e-12


def test_double_float_special_values(f64_mode):
    """Zeros, signed zeros, tiny and wide-ranging magnitudes survive the
    integer split / join of the double-float path within 1e-12 (absolute)."""
    capi.cast_set_f64_mode(capi.CAST_F64_EMULATED)
    n = 10
    rng = np.random.default_rng(4)
    mags = 10.0 ** rng.uniform(-40, 0, 1 << n)
    psi0 = mags * np.exp(2j * np.pi * rng.uniform(size=1 << n))
    psi0[:8] = [0, -0.0, 1e-300, -1e-300, 1.0, -1.0, 1j, -1j]
    psi0 = psi0 / np.linalg.norm(psi0)
    for k in (1, 3, 5):
        qs = W.sweep_targets(n, k, "mixed", rng)
        u = W.haar_unitary(k, rng)
        got = run_gate(n, "c128", psi0, qs, u)
        ref = oracle.apply_gate(psi0.copy(), qs, u)
        assert np.max(np.abs(got - ref)) <= 1e-12
        # relative accuracy on the larger outputs is near 2^-44
        big = np.abs(ref) > 1e-6
        assert np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big])) <= 1e-11


def test_double_float_norm_stable_over_many_gates(f64_mode):
    capi.cast_set_f64_mode(capi.CAST_F64_EMULATED)
    n = 14
    rng = np.random.default_rng(6)
    gates = [W.Gate("U", W.sweep_targets(n, 4, "mixed", rng), matrix=W.haar_unitary(4, rng)) for _ in range(200)]
    sv = pkg.StateVector(n, "c128")
    sv.apply_circuit(gates, fusion="none")
    assert abs(sv.expectation([W.PauliTerm(1.0, "", ())]) - 1.0) < 1e-12
    ref = oracle.simulate(n, gates)
    assert np.max(np.abs(sv.to_numpy() - ref)) <= 1e-12
    sv.close()
