"""The split-bf16 tensor-core mode for complex64 (CAST_TC_BF16X6: three bf16
pieces per operand, six products, per-slice norm restoration) against the
FP64 oracle: every target placement for k = 4, 5, a long gate sequence
(no norm drift), fused circuits, and the kernel choice (profiled kernel
families; k = 6, 7 stay on 3xTF32)."""
import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import REL, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture
def bf16_mode():
    old = capi.cast_get_tensor_mode()
    capi.cast_set_tensor_mode(capi.CAST_TC_BF16X6)
    yield capi
    capi.cast_set_tensor_mode(old)


def run_gate(n, psi0, qubits, m):
    sv = pkg.StateVector(n, "c64", init_index=None)
    sv.from_numpy(psi0.astype(np.complex64))
    capi.cast_profile_begin()
    sv.apply_gate(qubits, m)
    fams = [p["name"] for p in capi.cast_profile_end()]
    out = sv.to_numpy().astype(np.complex128)
    sv.close()
    return out, fams


@pytest.mark.parametrize("k", [4, 5])
def test_bf16_gate_every_placement(k, bf16_mode):
    """One Haar gate per placement: the bf16 split keeps fp32-class accuracy
    (relative error of one gate ~1e-7, the same order as 3xTF32)."""
    rng = np.random.default_rng(1200 + k)
    for n in (k + 7, k + 8, 16):
        psi0 = W.random_state(n, n + 3 * k)
        for placement in ("low", "high", "mixed", "mixed"):
            qs = W.sweep_targets(n, k, placement, rng)
            u = W.haar_unitary(k, rng)
            got, fams = run_gate(n, psi0, qs, u)
            ref = oracle.apply_gate(psi0.astype(np.complex64).astype(np.complex128), qs, u)
            assert fams == [f"tcbf_k{k}_c64"], fams
            assert np.max(np.abs(got - ref)) <= TOL, f"n={n} {qs}"
            assert rel_err(got, ref) <= 1e-6


@pytest.mark.parametrize("k", [4, 5])
def test_bf16_norm_does_not_drift(k, bf16_mode):
    """400 Haar gates: the norm stays at 1 and the state within the complex64
    bounds of the oracle (the truncated first two pieces are exact splits; the
    rounded last piece and the norm restoration leave unbiased noise)."""
    n = 17
    rng = np.random.default_rng(1300 + k)
    gates = [W.Gate("U", W.sweep_targets(n, k, ("low", "high", "mixed")[i % 3], rng),
                    matrix=W.haar_unitary(k, rng)) for i in range(400)]
    psi0 = W.random_state(n, 19)
    ref = oracle.apply_circuit(psi0.copy(), gates)
    sv = pkg.StateVector(n, "c64", init_index=None)
    sv.from_numpy(psi0.astype(np.complex64))
    sv.apply_circuit(gates, fusion="none")
    assert abs(sv.expectation([W.PauliTerm(1.0, "", ())]) - 1.0) <= 1e-5
    got = sv.to_numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL
    assert np.linalg.norm(got - ref) <= 2e-5
    sv.close()


@pytest.mark.parametrize("fam", ["RQC", "QVC", "QFT"])
def test_bf16_fused_circuits(fam, bf16_mode):
    """Fused to k <= 7: k = 4, 5 gates on the bf16 kernel, k = 6, 7 on 3xTF32."""
    n = 16
    gates = W.benchmark_family(fam, n, seed=4)[:500]
    ref = oracle.simulate(n, gates, init_index=9)
    sv = pkg.StateVector(n, "c64", init_index=9)
    capi.cast_profile_begin()
    sv.apply_circuit(gates, fusion="size", max_k=7)
    fams = {p["name"] for p in capi.cast_profile_end()}
    got = sv.to_numpy().astype(np.complex128)
    sv.close()
    assert not any(f.startswith("tc_k4") or f.startswith("tc_k5") for f in fams), fams
    assert np.max(np.abs(got - ref)) <= TOL
    assert rel_err(got, ref) <= REL["c64"]


def test_tensor_mode_accepts_bf16x6():
    old = capi.cast_get_tensor_mode()
    try:
        capi.cast_set_tensor_mode(capi.CAST_TC_BF16X6)
        assert capi.cast_get_tensor_mode() == capi.CAST_TC_BF16X6
        with pytest.raises(capi.CastError):
            capi.cast_set_tensor_mode(3)
    finally:
        capi.cast_set_tensor_mode(old)
