"""The host fusion pass (cast_fuse) against the oracle's own reading of
Algorithm 1 (oracle/fusion.py): the same fused blocks, in the same order, with
the same operation counts, and matrices equal to rounding; and the oracle's
fusion pinned to the unfused circuit by brute force."""
import numpy as np
import pytest

import oracle
import oracle.fusion as ofu
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import circuit_unitary

CASES = [
    ("rqc6", 6, lambda: W.random_circuit(6, 6, 1)),
    ("rqc9", 9, lambda: W.random_circuit(9, 5, 2)),
    ("qft8", 8, lambda: W.qft_circuit(8)),
    ("hea7", 7, lambda: W.hea_ansatz(7, 3)[0]),
]


def _compare(n, gates, theta, **kw):
    got = capi.cast_fuse(n, gates, theta, opts=capi.options(**kw))
    ref = ofu.fuse(n, gates, theta, mode=kw["fusion"], max_k=kw["max_k"],
                   agglomerative=kw["agglomerative"], amp_ops_per_pass=kw["amp_ops_per_pass"],
                   op_cap=kw.get("op_cap", 4096))
    assert [q for q, _, _ in got] == [q for q, _, _ in ref]
    assert [o for _, _, o in got] == [o for _, _, o in ref]
    for (_, a, _), (_, b, _) in zip(got, ref):
        assert np.max(np.abs(a - b)) < 1e-12
    return ref


@pytest.mark.parametrize("name,n,make", CASES)
@pytest.mark.parametrize("mode,max_k,agg,P", [("size", 2, True, 82), ("size", 4, True, 82),
                                              ("size", 5, False, 82), ("adaptive", 5, True, 82),
                                              ("adaptive", 5, True, 2), ("adaptive", 3, True, 16),
                                              ("none", 5, True, 82)])
def test_fusion_structure_matches_oracle(name, n, make, mode, max_k, agg, P):
    gates = make()
    theta = W.uniform_params(2 * n * 3, -3, 3, 0) if name.startswith("hea") else None
    _compare(n, gates, theta, fusion=mode, max_k=max_k, agglomerative=agg, amp_ops_per_pass=P)


@pytest.mark.parametrize("name,n,make", CASES)
def test_oracle_fusion_preserves_the_circuit(name, n, make):
    gates = make()
    theta = W.uniform_params(2 * n * 3, -3, 3, 0) if name.startswith("hea") else None
    fused = ofu.fuse(n, gates, theta, mode="size", max_k=4)
    ref = circuit_unitary(n, [(g.qubits, oracle.gate_matrix(g, theta)) for g in gates])
    got = circuit_unitary(n, [(q, m) for q, m, _ in fused])
    assert np.max(np.abs(got - ref)) < 1e-12
    assert all(len(q) <= 4 for q, _, _ in fused)


def test_oracle_fusion_worked_example():
    """Section IV-B's MoveBlock example: a block whose slot below is empty
    moves down and then fuses with the block two rows below it.
    Rows: 0: A(q0), B(q1); 1: C(q1); 2: D(q0, q1)."""
    gates = [W.Gate("H", (0,)), W.Gate("X", (1,)), W.Gate("Z", (1,)), W.Gate("CX", (0, 1))]
    fused = ofu.fuse(2, gates, mode="size", max_k=2)
    assert len(fused) == 1 and fused[0][0] == (0, 1)
    U = circuit_unitary(2, [(g.qubits, oracle.gate_matrix(g)) for g in gates])
    assert np.max(np.abs(fused[0][1] - U)) < 1e-14


@pytest.mark.parametrize("which", ["qft30", "rqc30"])
@pytest.mark.parametrize("P", [82, 16])
def test_benchmark_plans_match_oracle(which, P):
    """The 30-qubit fused streams bench.py times (adaptive, k <= 5; complex64
    and double-float complex128 cost constants)."""
    n = 30
    gates = W.qft_circuit(n) if which == "qft30" else W.random_circuit(n, 30, 1)
    ref = _compare(n, gates, None, fusion="adaptive", max_k=5, agglomerative=True, amp_ops_per_pass=P)
    assert len(ref) < len(gates) / 3


# a measured-looking cost table (ms per gate at 26 qubits, complex64):
# memory-bound up to k = 4, growing beyond, sparse classes cheaper
SAMPLE_MS = [[0, 0, 0, 0],
             [0, 0.15, 0.16, 0.17], [0, 0.15, 0.16, 0.17], [0, 0.16, 0.17, 0.18],
             [0, 0.16, 0.18, 0.19], [0, 0.17, 0.19, 0.21], [0, 0.18, 0.22, 0.45], [0, 0.2, 0.3, 1.6]]


@pytest.mark.parametrize("name,n,make", CASES)
@pytest.mark.parametrize("max_k", [3, 5, 0])
def test_cost_table_fusion_matches_oracle(name, n, make, max_k):
    gates = make()
    theta = W.uniform_params(2 * n * 3, -3, 3, 0) if name.startswith("hea") else None
    table = capi.cost_table(SAMPLE_MS)
    got = capi.cast_fuse(n, gates, theta, opts=capi.options("adaptive", max_k, cost=table))
    ref = ofu.fuse(n, gates, theta, mode="adaptive", max_k=max_k, cost=SAMPLE_MS)
    assert [q for q, _, _ in got] == [q for q, _, _ in ref]
    for (_, a, _), (_, b, _) in zip(got, ref):
        assert np.max(np.abs(a - b)) < 1e-12


def test_max_k_zero_needs_a_cost_table():
    with pytest.raises(capi.CastError):
        capi.cast_fuse(4, W.random_circuit(4, 2, 0), opts=capi.options("adaptive", 0))


SPARSE_FLOOR = [0, 0, 0, 0.17, 0.18, 0.2, 0.22, 0.25]
SPARSE_PER_OP = [0, 0, 0, 2e-4, 1e-4, 6e-5, 3e-5, 2e-5]


@pytest.mark.parametrize("name,n,make", CASES)
@pytest.mark.parametrize("max_k", [5, 7, 0])
def test_sparse_cost_table_fusion_matches_oracle(name, n, make, max_k):
    gates = make()
    theta = W.uniform_params(2 * n * 3, -3, 3, 0) if name.startswith("hea") else None
    table = capi.cost_table(SAMPLE_MS, sparse_floor_ms=SPARSE_FLOOR, sparse_ms_per_op=SPARSE_PER_OP)
    got = capi.cast_fuse(n, gates, theta, opts=capi.options("adaptive", max_k, cost=table))
    ref = ofu.fuse(n, gates, theta, mode="adaptive", max_k=max_k, cost=capi.cost_table_dict(table))
    assert [q for q, _, _ in got] == [q for q, _, _ in ref]
    for (_, a, _), (_, b, _) in zip(got, ref):
        assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("fam", sorted(W.FAMILIES))
def test_family_plans_match_oracle(fam):
    """The six benchmark families (20 qubits): size-only and adaptive fusion,
    the same blocks and operation counts as the reference."""
    n = 20
    gates = W.benchmark_family(fam, n, seed=4)[:500]
    for mode in ("size", "adaptive"):
        _compare(n, gates, None, fusion=mode, max_k=5, agglomerative=True, amp_ops_per_pass=16)
