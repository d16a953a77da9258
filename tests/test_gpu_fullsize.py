"""Parity at the benchmark's full size (30 qubits), in the launch configuration
bench.py times (the same fused plans, the same kernels), checked on outputs that
closed forms give one by one, and on properties that hold at any size.

- QFT-30 of a basis state: every amplitude is exp(2 pi i (x y mod 2^30)/2^30) / 2^15
  (the phase reduced in exact integer arithmetic); sampled amplitudes plus the
  first and last ones are compared.
- A dense Haar gate on a basis state |x>: the result is the matrix column of
  x's target bits, placed at the 2^k indices that differ from x in the targets.
- The fused RQC-30 followed by its fused inverse returns |x>.
- Norms and <Z_0> = 0 after the QFT.
"""
import math

import numpy as np
import pytest
import torch

import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

N_Q = 30
TOL = {"c128": 1e-12, "c64": 1e-5}
IDENTITY = [W.PauliTerm(1.0, "", ())]


def sampled(sv, idx):
    t = torch.as_tensor(idx, dtype=torch.int64, device=sv.tensor.device)
    return sv.tensor.index_select(0, t).cpu().numpy().astype(np.complex128)


def plan(gates, dtype):
    return capi.cast_plan_create(N_Q, gates, opts=capi.options("adaptive", 5), dtype=dtype)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_qft30_closed_form_on_samples(dtype):
    x = W.random_basis_index(N_Q, 1)  # bench.py's basis state
    rng = np.random.default_rng(0)
    idx = np.concatenate([[0, 1, (1 << N_Q) - 1, x], rng.integers(0, 1 << N_Q, 4096)]).astype(np.int64)
    p = plan(W.qft_circuit(N_Q), dtype)
    sv = pkg.StateVector(N_Q, dtype, init_index=x)
    capi.cast_plan_apply(sv.handle, p)
    got = sampled(sv, idx)
    ph = ((x * idx) % (1 << N_Q)).astype(np.float64) / float(1 << N_Q)
    ref = np.exp(2j * np.pi * ph) / math.sqrt(1 << N_Q)
    err = np.abs(got - ref)
    assert err.max() <= TOL[dtype]
    # relative to the amplitude size (2^-15), the error is small too
    assert err.max() / 2.0 ** -15 <= (1e-5 if dtype == "c64" else 1e-10)
    assert abs(sv.expectation(IDENTITY) - 1.0) <= 10 * TOL[dtype]
    assert abs(sv.expectation(W.z0_observable())) <= 10 * TOL[dtype]
    sv.close()
    capi.cast_plan_destroy(p)


@pytest.mark.parametrize("k,placement", [(5, "low"), (5, "high"), (5, "mixed"), (4, "mixed"), (6, "mixed"),
                                         (3, "mixed"), (2, "high")])
def test_dense_gate_on_basis_state_full_size(k, placement):
    """complex64; k = 4..6 run on the tensor cores at this size."""
    rng = np.random.default_rng(40 + k)
    qs = W.sweep_targets(N_Q, k, placement, rng)
    u = W.haar_unitary(k, rng)
    x = int(rng.integers(0, 1 << N_Q))
    sv = pkg.StateVector(N_Q, "c64", init_index=x)
    sv.apply_gate(qs, u)
    jx = sum(((x >> q) & 1) << i for i, q in enumerate(qs))
    base = x & ~sum(1 << q for q in qs)
    idx = np.array([base | sum(((j >> i) & 1) << q for i, q in enumerate(qs)) for j in range(1 << k)])
    got = sampled(sv, idx)
    assert np.max(np.abs(got - u[:, jx])) <= TOL["c64"]
    # nothing else moved: the column has unit norm, so the rest of the state is zero
    assert abs(sv.expectation(IDENTITY) - 1.0) <= 10 * TOL["c64"]
    sv.apply_gate(qs, u.conj().T)
    back = sampled(sv, np.array([x]))
    assert abs(back[0] - 1.0) <= 10 * TOL["c64"]
    sv.close()


def inverse(gates):
    inv = {"H": "H", "X": "X", "CX": "CX"}
    out = []
    for g in reversed(gates):
        if g.name in inv:
            out.append(W.Gate(inv[g.name], g.qubits))
        else:  # RX, RY, RZ
            out.append(W.Gate(g.name, g.qubits, (-g.params[0],)))
    return out


@pytest.mark.parametrize("dtype,layers", [("c64", 30), ("c128", 4)])
def test_rqc30_fused_then_inverse_returns(dtype, layers):
    x = W.random_basis_index(N_Q, 1)
    gates = W.random_circuit(N_Q, layers, 1)
    pf, pi = plan(gates, dtype), plan(inverse(gates), dtype)
    sv = pkg.StateVector(N_Q, dtype, init_index=x)
    capi.cast_plan_apply(sv.handle, pf)
    assert abs(sv.expectation(IDENTITY) - 1.0) <= 10 * TOL[dtype]
    capi.cast_plan_apply(sv.handle, pi)
    rng = np.random.default_rng(3)
    idx = np.concatenate([[x], rng.integers(0, 1 << N_Q, 2048)]).astype(np.int64)
    got = sampled(sv, idx)
    ref = (idx == x).astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= TOL[dtype]
    sv.close()
    capi.cast_plan_destroy(pf)
    capi.cast_plan_destroy(pi)


@pytest.mark.parametrize("n,dtype,k", [(33, "c64", 5), (32, "c128", 3)])
def test_largest_states(n, dtype, k):
    """64 GiB states (2^33 complex64 / 2^32 complex128 amplitudes): slice
    counts above 2^31 and byte offsets above 2^35; a dense gate on a basis
    state reproduces the matrix column, and its inverse restores |x>."""
    rng = np.random.default_rng(n)
    qs = (0, n // 2, n - 1) + tuple(range(3, 3 + k - 3))
    u = W.haar_unitary(k, rng)
    x = (1 << (n - 1)) | (1 << (n // 2)) | 5
    sv = pkg.StateVector(n, dtype, init_index=x)
    sv.apply_gate(qs, u)
    jx = sum(((x >> q) & 1) << i for i, q in enumerate(qs))
    base = x & ~sum(1 << q for q in qs)
    idx = np.array([base | sum(((j >> i) & 1) << q for i, q in enumerate(qs)) for j in range(1 << k)])
    assert np.max(np.abs(sampled(sv, idx) - u[:, jx])) <= TOL[dtype]
    sv.apply_gate(qs, u.conj().T)
    assert abs(sampled(sv, np.array([x]))[0] - 1.0) <= 10 * TOL[dtype]
    assert abs(sv.expectation(IDENTITY) - 1.0) <= 10 * TOL[dtype]
    sv.close()
    torch.cuda.empty_cache()
