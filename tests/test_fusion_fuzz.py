"""Randomised cross-check of the host fusion pass (cast_fuse) against the
oracle's reading of Algorithm 1 (oracle/fusion.py).

The circuits mix gates of one to four qubits, each dense (Haar), diagonal or
monomial. They are fused at every width 2..7, in size-only and adaptive
mode, with and without a measured-looking cost table. This exercises both
orders of the trial products (a small gate after a wide block and a wide
block after a small gate), refusals repeated across traversals, and the
width search. Each case must reproduce the reference's blocks, order and
operation counts, with the same matrices up to rounding. For n <= 7 the
fused circuit must also equal the unfused one by brute force."""
import numpy as np
import pytest

import oracle
import oracle.fusion as ofu
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import circuit_unitary

MS = [[0, 0, 0, 0],
      [0, 0.15, 0.16, 0.17], [0, 0.15, 0.16, 0.17], [0, 0.16, 0.17, 0.18],
      [0, 0.16, 0.18, 0.19], [0, 0.17, 0.19, 0.21], [0, 0.18, 0.22, 0.45], [0, 0.2, 0.3, 1.6]]


def random_gate(n, rng):
    k = int(rng.choice([1, 1, 2, 2, 3, 4]))
    qs = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
    d = 1 << k
    kind = rng.integers(3)
    if kind == 0:
        z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / np.sqrt(2)
        q, r = np.linalg.qr(z)
        m = q * (np.diag(r) / np.abs(np.diag(r)))
    elif kind == 1:
        m = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, d)))
    else:
        m = np.zeros((d, d), dtype=np.complex128)
        m[rng.permutation(d), np.arange(d)] = np.exp(1j * rng.uniform(0, 2 * np.pi, d))
    return W.Gate("U", qs, matrix=m)


def random_circuit(n, count, seed):
    rng = np.random.default_rng(seed)
    return [random_gate(n, rng) for _ in range(count)]


@pytest.mark.parametrize("seed", range(12))
def test_random_circuits_match_the_reference(seed):
    n = 5 + seed % 4
    gates = random_circuit(n, 24 + 2 * seed, 1000 + seed)
    for mode, max_k, cost in (("size", 2 + seed % 6, None), ("adaptive", 3 + seed % 5, None),
                              ("adaptive", 7, MS), ("adaptive", 0, MS)):
        P = (82, 16, 2)[seed % 3]
        opts = capi.options(mode, max_k, amp_ops_per_pass=P,
                            cost=capi.cost_table(MS) if cost is not None else None)
        got = capi.cast_fuse(n, gates, opts=opts)
        ref = ofu.fuse(n, gates, mode=mode, max_k=max_k, amp_ops_per_pass=P, cost=cost)
        assert [q for q, _, _ in got] == [q for q, _, _ in ref], (mode, max_k)
        assert [o for _, _, o in got] == [o for _, _, o in ref], (mode, max_k)
        for (_, a, _), (_, b, _) in zip(got, ref):
            assert np.max(np.abs(a - b)) < 1e-12
        if n <= 7:
            U = circuit_unitary(n, [(g.qubits, oracle.gate_matrix(g)) for g in gates])
            V = circuit_unitary(n, [(q, m) for q, m, _ in got])
            assert np.max(np.abs(U - V)) < 1e-12
