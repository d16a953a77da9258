"""Batched hardware-efficient ansatz (tile executor) against the oracle.

Instances of uneven qubit counts share each launch: fewer qubits than one
tile, exactly one tile, and two or three qubit groups for both precisions.
Energies are compared with the oracle's unfused simulation and Pauli-sum
expectation; gradients with the oracle's exact parameter shift.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

# complex128 runs in double-float arithmetic on the FP32 pipe (the default)
# or on the FP64 pipe; both are checked
F64_MODES = {"df": "CAST_F64_EMULATED", "fp64": "CAST_F64_NATIVE"}


@pytest.fixture
def f64(request):
    mode = getattr(request, "param", "df")
    old = capi.cast_get_f64_mode()
    capi.cast_set_f64_mode(getattr(capi, F64_MODES[mode]))
    yield mode
    capi.cast_set_f64_mode(old)


def with_modes(c128_tol, c64_tol):
    """(dtype, f64 mode, tolerance) cases: complex128 in both arithmetics."""
    return pytest.mark.parametrize("dtype,f64,tol", [("c128", "df", c128_tol), ("c128", "fp64", c128_tol),
                                                     ("c64", "df", c64_tol)], indirect=["f64"])


def tfim(n, zz, hx):
    return [W.PauliTerm(zz, "ZZ", (i, i + 1)) for i in range(n - 1)] + \
        [W.PauliTerm(hx, "X", (i,)) for i in range(n)]


def split(params, ns, layers):
    out, off = [], 0
    for n in ns:
        out.append(params[off:off + 2 * n * layers])
        off += 2 * n * layers
    return out


@with_modes(1e-10, 2e-5)
def test_hea_batch_energies(dtype, f64, tol):
    ns = [4, 7, 11, 12, 13, 16, 18, 20]
    layers, zz, hx = 3, 0.8, 0.5
    b = capi.cast_hea_create(ns, layers, dtype)
    npar, _ = capi.cast_hea_info(b)
    assert npar == sum(2 * n * layers for n in ns)
    theta = W.uniform_params(npar, -math.pi, math.pi, 3)
    e = capi.cast_hea_energy(b, theta, zz, hx, len(ns))
    for n, th, ei in zip(ns, split(theta, ns, layers), e):
        gates, _ = W.hea_ansatz(n, layers)
        ref = oracle.energy(n, gates, th, tfim(n, zz, hx))
        assert abs(ei - ref) <= tol * (n * (abs(zz) + abs(hx))), (n, ei, ref)
    # a second parameter set replays the captured graph
    theta2 = W.uniform_params(npar, -math.pi, math.pi, 4)
    e2 = capi.cast_hea_energy(b, theta2, zz, hx, len(ns))
    n0 = ns[5]
    gates, _ = W.hea_ansatz(n0, layers)
    ref = oracle.energy(n0, gates, split(theta2, ns, layers)[5], tfim(n0, zz, hx))
    assert abs(e2[5] - ref) <= tol * n0
    capi.cast_hea_destroy(b)


@with_modes(1e-10, 5e-5)
def test_hea_batch_gradients_vs_parameter_shift(dtype, f64, tol):
    ns = [5, 13, 14]
    layers, zz, hx = 2, 1.0, 0.7
    b = capi.cast_hea_create(ns, layers, dtype, with_grad=True)
    npar, _ = capi.cast_hea_info(b)
    theta = W.uniform_params(npar, -math.pi, math.pi, 8)
    e, g = capi.cast_hea_grad(b, theta, zz, hx, len(ns))
    for n, th, ei, gi in zip(ns, split(theta, ns, layers), e, split(g, ns, layers)):
        gates, _ = W.hea_ansatz(n, layers)
        H = tfim(n, zz, hx)
        assert abs(ei - oracle.energy(n, gates, th, H)) <= tol * n
        ps = oracle.grad_param_shift(n, gates, th, H)
        assert np.max(np.abs(gi - ps)) <= tol * n, (n, np.max(np.abs(gi - ps)))
    capi.cast_hea_destroy(b)


@pytest.mark.parametrize("f64", ["df", "fp64"], indirect=True)
def test_hea_matches_single_state_adjoint(f64):
    """The batched adjoint and cast_adjoint_grad on one 15-qubit instance."""
    import paper_2503_19894_gb300 as pkg
    n, layers = 15, 3
    gates, npar = W.hea_ansatz(n, layers)
    theta = W.uniform_params(npar, -math.pi, math.pi, 2)
    H = W.tfim_hamiltonian(n, 0.7)
    b = capi.cast_hea_create([n], layers, "c128", with_grad=True)
    e, g = capi.cast_hea_grad(b, theta, 1.0, 0.7, 1)
    psi = pkg.StateVector(n, "c128")
    lam = pkg.StateVector(n, "c128", init_index=None)
    e1, g1 = pkg.cast_adjoint_grad(psi.handle, lam.handle, n, gates, theta, H)
    assert abs(e[0] - e1) < 1e-11
    assert np.max(np.abs(g - g1)) < 1e-11
    psi.close()
    lam.close()
    capi.cast_hea_destroy(b)


def test_hea_arguments_rejected():
    with pytest.raises(capi.CastError):
        capi.cast_hea_create([1], 2, "c64")
    with pytest.raises(capi.CastError):
        capi.cast_hea_create([5], 0, "c64")
    b = capi.cast_hea_create([6], 1, "c64")
    with pytest.raises(capi.CastError):  # no gradient buffers
        capi.cast_hea_grad(b, np.zeros(12), 1.0, 1.0, 1)
    with pytest.raises(capi.CastError):
        capi.cast_hea_energy(b, np.full(12, np.nan), 1.0, 1.0, 1)
    capi.cast_hea_destroy(b)
