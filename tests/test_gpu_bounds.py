"""Parity at the stated bounds, against the oracle, for the configurations
that carry the headline numbers:

- the 12-qubit, 20-layer ansatz gradient (480 parameters, transverse-field
  Ising H with coefficient 0.7): cast_adjoint_grad against the oracle's exact
  parameter shift and central finite differences (h = 1e-6), in both
  precisions;
- the fused 26-qubit random circuit of 30 layers (the benchmark's RQC plan at
  26 qubits), forward, full state against the oracle's unfused simulation, in
  complex64 and complex128;
- the batched ansatz instances whose later qubit groups are wide, against the
  oracle's energies and parameter-shift gradients directly.

Bounds: amplitudes max |delta| <= 1e-12 (complex128) / 1e-5 (complex64) plus
the relative bound of tests.helpers.REL; expectation values and gradients
<= the amplitude bound times sum |coefficients| (|<psi|H|psi> - <phi|H|phi>|
<= 2 ||H|| ||psi - phi|| and ||H|| <= sum |c|); complex128 gradients also
<= 1e-10 of exact parameter shift.
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


# ------------------------------------------------ 12 qubits, 20 layers
@pytest.fixture(scope="module")
def ansatz12():
    n, layers = 12, 20
    gates, npar = W.hea_ansatz(n, layers)
    theta = W.uniform_params(npar, -math.pi, math.pi, 44)
    H = W.tfim_hamiltonian(n, 0.7)
    return dict(n=n, gates=gates, theta=theta, H=H,
                e=oracle.energy(n, gates, theta, H),
                ps=oracle.grad_param_shift(n, gates, theta, H),
                fd=oracle.grad_finite_diff(n, gates, theta, H, h=1e-6))


def test_oracle_gradients_agree_12q(ansatz12):
    """Parameter shift is exact; central differences carry O(h^2) plus
    rounding / h ~ 1e-10 * |E|: they agree far inside 1e-7."""
    assert np.max(np.abs(ansatz12["ps"] - ansatz12["fd"])) <= 1e-7


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_gradient_12q_20_layers(ansatz12, dtype):
    a = ansatz12
    n = a["n"]
    scale = sum(abs(t.coeff) for t in a["H"])
    psi = pkg.StateVector(n, dtype)
    lam = pkg.StateVector(n, dtype, init_index=None)
    e, g = pkg.cast_adjoint_grad(psi.handle, lam.handle, n, a["gates"], a["theta"], a["H"])
    psi.close()
    lam.close()
    assert g.shape == (480,)
    assert abs(e - a["e"]) <= TOL[dtype] * scale
    assert np.max(np.abs(g - a["ps"])) <= TOL[dtype] * scale
    if dtype == "c128":
        assert np.max(np.abs(g - a["ps"])) <= 1e-10
        assert np.max(np.abs(g - a["fd"])) <= 1e-7
    else:
        assert np.max(np.abs(g - a["fd"])) <= TOL[dtype] * scale + 1e-7


# ---------------------------------- 26 qubits, fused RQC of 30 layers, forward
N26 = 26


@pytest.fixture(scope="module")
def rqc26():
    x = W.random_basis_index(N26, 1)
    gates = W.random_circuit(N26, 30, 1)
    return x, gates, oracle.simulate(N26, gates, init_index=x)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_rqc26_fused_forward_full_state(rqc26, dtype):
    x, gates, ref = rqc26
    p = capi.cast_plan_create(N26, gates, opts=capi.options("adaptive", 5), dtype=dtype)
    sv = pkg.StateVector(N26, dtype, init_index=x)
    capi.cast_plan_apply(sv.handle, p)
    got = sv.to_numpy().astype(np.complex128)
    sv.close()
    capi.cast_plan_destroy(p)
    err = float(np.max(np.abs(got - ref)))
    rel = rel_err(got, ref)
    assert err <= TOL[dtype], err
    assert rel <= REL[dtype], rel


# -------------------------- batched ansatz, wide qubit groups, against the oracle
def _tfim(n, zz, hx):
    return [W.PauliTerm(zz, "ZZ", (i, i + 1)) for i in range(n - 1)] + \
        [W.PauliTerm(hx, "X", (i,)) for i in range(n)]


@pytest.fixture
def f64_default():
    old = capi.cast_get_f64_mode()
    capi.cast_set_f64_mode(capi.CAST_F64_EMULATED)
    yield
    capi.cast_set_f64_mode(old)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_hea_wide_groups_against_oracle(dtype, f64_default):
    """Instances of 19, 20 and 17 qubits whose later groups rotate 3..7 qubits;
    energies of every instance and 24 gradients per instance (every qubit
    group represented) against the oracle."""
    ns, layers, zz, hx = [19, 20, 17], 2, 1.0, 0.7
    b = capi.cast_hea_create(ns, layers, dtype, with_grad=True)
    npar, _ = capi.cast_hea_info(b)
    theta = W.uniform_params(npar, -math.pi, math.pi, 21)
    e, g = capi.cast_hea_grad(b, theta, zz, hx, len(ns))
    capi.cast_hea_destroy(b)
    off = 0
    rng = np.random.default_rng(5)
    for n, ei in zip(ns, e):
        th = theta[off:off + 2 * n * layers]
        gi = g[off:off + 2 * n * layers]
        off += 2 * n * layers
        gates, _ = W.hea_ansatz(n, layers)
        H = _tfim(n, zz, hx)
        scale = sum(abs(t.coeff) for t in H)
        assert abs(ei - oracle.energy(n, gates, th, H)) <= TOL[dtype] * scale
        # the last layer's RY and RZ of the top qubit and of 22 random ones
        idx = sorted({2 * n * (layers - 1) + n - 1, 2 * n * (layers - 1) + 2 * n - 1} |
                     set(int(v) for v in rng.choice(2 * n * layers, 22, replace=False)))
        ps = oracle.grad_param_shift(n, gates, th, H, indices=idx)
        assert np.max(np.abs(gi[idx] - ps)) <= TOL[dtype] * scale
        if dtype == "c128":
            assert np.max(np.abs(gi[idx] - ps)) <= 1e-10


# --------------------- complex64 reductions on a large state, against FP64
def test_c64_expectation_26q_against_oracle():
    """complex64 Pauli sums sum products in fp32 and carry compensated fp32
    partial sums (FP64 per block): on a 26-qubit state, where terms cancel
    over 2^26 amplitudes, the result stays within 1e-7 of sum |c| of the
    oracle's FP64 value on the same (rounded) amplitudes, far inside the
    1e-5 bound."""
    n = 26
    psi = W.random_state(n, 31).astype(np.complex64)
    H = W.tfim_hamiltonian(n, 0.7) + [W.PauliTerm(0.4, "XYZ", (3, 11, 25)), W.PauliTerm(-0.3, "YY", (0, 24))]
    scale = sum(abs(t.coeff) for t in H)
    sv = pkg.StateVector(n, "c64", init_index=None)
    sv.from_numpy(psi)
    got = sv.expectation(H)
    z0 = sv.expectation(W.z0_observable())
    sv.close()
    ref = oracle.expectation(psi.astype(np.complex128), H)
    assert abs(got - ref) <= 1e-7 * scale, (got, ref)
    chunk = 1 << 22
    z0_ref = sum(oracle.z_string_partial(psi[a:a + chunk], a, (0,)) for a in range(0, 1 << n, chunk))
    assert abs(z0 - z0_ref) <= 1e-7
