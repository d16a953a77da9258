"""Batched circuits of different shapes in one batch (cast_batch_*), against
the oracle: energies against the oracle's unfused simulation and Pauli-sum
expectation, gradients against exact parameter shift (one gate per
parameter) or central finite differences (a parameter shared by several
gates), in both precisions."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}


def qaoa_ring(n, p):
    """H on all, then p rounds of exp(-i gamma ZZ) on the ring edges (as CX, RZ,
    CX, one shared gamma per round) and RX(beta) on all (one shared beta)."""
    gates = [W.Gate("H", (q,)) for q in range(n)]
    for r in range(p):
        for i in range(n):
            a, b = i, (i + 1) % n
            gates += [W.Gate("CX", (a, b)), W.Gate("RZ", (b,), pidx=2 * r), W.Gate("CX", (a, b))]
        gates += [W.Gate("RX", (q,), pidx=2 * r + 1) for q in range(n)]
    return gates, 2 * p


def rx_cz_ansatz(n, layers):
    gates, k = [], 0
    for _ in range(layers):
        for q in range(n):
            gates.append(W.Gate("RX", (q,), pidx=k))
            k += 1
        gates += [W.Gate("CZ", (i, i + 1)) for i in range(0, n - 1, 2)]
        for q in range(n):
            gates.append(W.Gate("RY", (q,), pidx=k))
            k += 1
        gates += [W.Gate("CZ", (i, i + 1)) for i in range(1, n - 1, 2)]
    return gates, k


def mixed_fixed(n, rng):
    u = W.haar_unitary(2, rng)
    gates = [W.Gate("RY", (0,), pidx=0), W.Gate("U", (1, 3), matrix=u), W.Gate("RZ", (3,), pidx=1),
             W.Gate("SWAP", (0, 4)), W.Gate("RX", (2,), pidx=2), W.Gate("CP", (2, 4), (0.37,)),
             W.Gate("RY", (4,), pidx=3), W.Gate("T", (1,))]
    return gates, 4


def instances(rng):
    hea, nh = W.hea_ansatz(9, 2)
    qa, nq = qaoa_ring(7, 2)
    rc, nr = rx_cz_ansatz(12, 2)
    tiny, nt = W.hea_ansatz(3, 3)
    mf, nm = mixed_fixed(5, rng)
    ham_y = [W.PauliTerm(0.6, "XY", (0, 5)), W.PauliTerm(-0.4, "YZ", (3, 11)), W.PauliTerm(0.9, "Y", (7,)),
             W.PauliTerm(0.25, "ZZ", (1, 2))]
    return [
        (9, hea, nh, W.tfim_hamiltonian(9, 0.7), "ps"),
        (7, qa, nq, [W.PauliTerm(1.0, "ZZ", (i, (i + 1) % 7)) for i in range(7)] + [W.PauliTerm(0.3, "X", (2,))], "fd"),
        (12, rc, nr, ham_y, "ps"),
        (3, tiny, nt, W.tfim_hamiltonian(3, 0.5), "ps"),
        (5, mf, nm, [W.PauliTerm(1.0, "XZ", (0, 4)), W.PauliTerm(-0.5, "Y", (1,)), W.PauliTerm(0.8, "Z", (3,))], "ps"),
    ]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_of_different_shapes_against_oracle(dtype):
    rng = np.random.default_rng(7)
    inst = instances(rng)
    b = capi.Batch([(n, g, npar, H) for n, g, npar, H, _ in inst], dtype=dtype, with_grad=True)
    assert b.n_params == sum(npar for _, _, npar, _, _ in inst)
    assert b.n_steps == max(len(g) for _, g, _, _, _ in inst)
    theta = W.uniform_params(b.n_params, -math.pi, math.pi, 11)
    e = b.energy(theta)
    e2, g = b.grad(theta)
    off = 0
    for i, (n, gates, npar, H, how) in enumerate(inst):
        th = theta[off:off + npar]
        scale = sum(abs(t.coeff) for t in H)
        ref = oracle.energy(n, gates, th, H)
        assert abs(e[i] - ref) <= TOL[dtype] * scale, (i, e[i], ref)
        assert abs(e2[i] - ref) <= TOL[dtype] * scale
        gi = g[off:off + npar]
        if how == "ps":
            gref = oracle.grad_param_shift(n, gates, th, H)
            bound = 1e-10 if dtype == "c128" else TOL[dtype] * scale
        else:
            gref = oracle.grad_finite_diff(n, gates, th, H, h=1e-6)
            bound = 1e-7 if dtype == "c128" else TOL[dtype] * scale
        assert np.max(np.abs(gi - gref)) <= bound, (i, np.max(np.abs(gi - gref)))
        off += npar
    # a second parameter set replays the same graphs
    theta2 = W.uniform_params(b.n_params, -math.pi, math.pi, 12)
    e3 = b.energy(theta2)
    n, gates, npar, H, _ = inst[2]
    o2 = sum(x[2] for x in inst[:2])
    assert abs(e3[2] - oracle.energy(n, gates, theta2[o2:o2 + npar], H)) <= TOL[dtype] * sum(abs(t.coeff) for t in H)
    b.close()


def test_batch_shared_parameters_across_instances():
    """Two instances reading the same parameters (offsets 0 and 0): the
    gradient is the sum of both instances' gradients."""
    gates, npar = W.hea_ansatz(6, 2)
    H1, H2 = W.tfim_hamiltonian(6, 0.7), W.tfim_hamiltonian(6, -0.4)
    b = capi.Batch([(6, gates, npar, H1), (6, gates, npar, H2)], dtype="c128", with_grad=True, param_offsets=[0, 0])
    assert b.n_params == npar
    theta = W.uniform_params(npar, -1, 1, 3)
    e, g = b.grad(theta)
    ref = oracle.grad_param_shift(6, gates, theta, H1) + oracle.grad_param_shift(6, gates, theta, H2)
    assert np.max(np.abs(g - ref)) <= 1e-10
    assert abs(e[0] - oracle.energy(6, gates, theta, H1)) <= 1e-11
    b.close()


def test_batch_rejects_bad_instances():
    with pytest.raises(capi.CastError):
        capi.Batch([(3, [W.Gate("H", (3,))], 0, [])])
    with pytest.raises(capi.CastError) as e:
        capi.Batch([(4, [W.Gate("U", (0, 1, 2), matrix=np.eye(8))], 0, [])])
    assert e.value.status == 5
    b = capi.Batch([(4, [W.Gate("RY", (0,), pidx=0)], 1, W.tfim_hamiltonian(4, 1.0))])
    with pytest.raises(capi.CastError):  # no gradient buffers
        b.grad(np.zeros(1))
    with pytest.raises(capi.CastError):
        b.energy(np.array([np.nan]))
    b.close()
