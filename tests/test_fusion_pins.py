"""Pins of the fusion reference (oracle/fusion.py) that do not involve the
product's fusion pass: every decision below is worked out by hand from the
paper (Section II-B and IV-C for operation counts and the adaptive test,
Section IV-A/IV-B and Algorithm 1 for the schedule) and written into the test,
so a mistake shared by the reference and the C++ pass still fails here.

The estimate of a block of k qubits and operation count c is
    est = max(P * 128, c * 2^(7 - k)),
the adaptive test fuses iff the fused size is at most the cap, the fused
operation count is at most op_cap and est(fused) <= est(top) + est(bottom).
For a dense k-qubit block c = 2^(2k+2), so c * 2^(7-k) = 2^(k+9).
"""
import json
import os

import numpy as np
import pytest

import oracle
import oracle.fusion as ofu
import workloads as W
from oracle import gates as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _haar(k, seed):
    return W.haar_unitary(k, np.random.default_rng(seed))


def _u(qubits, seed):
    return W.Gate("U", tuple(qubits), matrix=_haar(len(qubits), seed))


def _kron(*ms):
    out = np.eye(1, dtype=np.complex128)
    for m in ms:
        out = np.kron(out, m)
    return out


# ---------------------------------------------------------------- classify
def _cp(phi):
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def _cx_control_bit0():
    # |c t> with local bit 0 = control: rows/cols 1 <-> 3
    m = np.eye(4, dtype=np.complex128)
    m[[1, 3]] = m[[3, 1]]
    return m


def _swap():
    m = np.eye(4, dtype=np.complex128)
    m[[1, 2]] = m[[2, 1]]
    return m


CLASSES = [
    ("I2", np.eye(2), ofu.IDENTITY),
    ("I8", np.eye(8), ofu.IDENTITY),
    ("I_plus_tiny", np.eye(4) + 5e-13 * np.ones((4, 4)), ofu.IDENTITY),
    ("Z", G.Z(), ofu.DIAGONAL),
    ("S", np.diag([1, 1j]), ofu.DIAGONAL),
    ("RZ", np.diag([np.exp(-0.35j), np.exp(0.35j)]), ofu.DIAGONAL),
    ("CZ", np.diag([1, 1, 1, -1]), ofu.DIAGONAL),
    ("CP", _cp(0.4), ofu.DIAGONAL),
    ("CP_zero_angle", _cp(0.0), ofu.IDENTITY),
    ("X", G.X(), ofu.MONOMIAL),
    ("Y", G.Y(), ofu.MONOMIAL),
    ("CX", _cx_control_bit0(), ofu.MONOMIAL),
    ("SWAP", _swap(), ofu.MONOMIAL),
    ("iSWAP", np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]]), ofu.MONOMIAL),
    ("X_kron_Z", _kron(G.X(), G.Z()), ofu.MONOMIAL),
    ("H", G.H(), ofu.DENSE),
    ("HxH", _kron(G.H(), G.H()), ofu.DENSE),
    ("H_kron_I", _kron(G.H(), np.eye(2)), ofu.DENSE),  # two non-zeros per row
    ("RY", np.array([[np.cos(0.2), -np.sin(0.2)], [np.sin(0.2), np.cos(0.2)]]), ofu.DENSE),
    ("offdiag_above_tol", np.eye(2) + np.array([[0, 2e-12], [0, 0]]), ofu.DENSE),
    ("offdiag_below_tol", np.eye(2) + np.array([[0, 5e-13], [0, 0]]), ofu.IDENTITY),
    ("diag_entry_off_one", np.diag([1, 1 + 1e-9]), ofu.DIAGONAL),
]


@pytest.mark.parametrize("name,m,cls", CLASSES, ids=[c[0] for c in CLASSES])
def test_classify_hand_built(name, m, cls):
    assert ofu.classify(np.asarray(m, dtype=np.complex128), 1e-12) == cls


def test_classify_haar_dense_and_kron_of_monomials():
    for k in range(1, 5):
        assert ofu.classify(_haar(k, k), 1e-12) == ofu.DENSE
    # a tensor product of monomials is monomial, of diagonals diagonal
    assert ofu.classify(_kron(G.X(), G.Y(), _swap()), 1e-12) == ofu.MONOMIAL
    assert ofu.classify(_kron(G.Z(), np.diag([1, 1j]), _cp(1.0)), 1e-12) == ofu.DIAGONAL


# ---------------------------------------------------------------- opcount
def test_opcount_against_paper_counts():
    """Section II-B: a Pauli has 2 non-zero scalars, a dense 1-qubit gate 8;
    Section IV-C: 2 operations per scalar, a dense k-qubit gate 2^(2k+2)."""
    with open(os.path.join(GOLDEN, "paper_opcounts.json")) as f:
        gold = json.load(f)
    for p, fn in (("X", G.X), ("Y", G.Y), ("Z", G.Z)):
        assert ofu.opcount(fn(), 1e-12) == 2 * gold["nonzero_scalars"][p]
    assert ofu.opcount(_haar(1, 3), 1e-12) == 2 * gold["nonzero_scalars"]["dense_1q"]
    for k in range(1, 8):
        assert ofu.opcount(_haar(k, 10 + k), 1e-12) == gold["opcount_dense"][str(k)]
    # real entries count one scalar each: H has 4 real entries -> 8 operations
    assert ofu.opcount(G.H(), 1e-12) == 8
    # S = diag(1, i): two scalars -> 4; CP(phi): 3 real ones + one complex -> 10
    assert ofu.opcount(np.diag([1, 1j]), 1e-12) == 4
    assert ofu.opcount(_cp(0.4), 1e-12) == 10


# ---------------------------------------------------------------- estimate
def _block(qubits, matrix):
    return ofu.Block(qubits, [(tuple(qubits), matrix)])


@pytest.mark.parametrize("P,k,expect", [
    # P = 82 -> floor 10496; dense k: 2^(k+9) = 1024, 2048, 4096, 8192, 16384, 32768, 65536
    (82, 1, 10496), (82, 4, 10496), (82, 5, 16384), (82, 6, 32768), (82, 7, 65536),
    # P = 2 -> floor 256: the dense term always wins
    (2, 1, 1024), (2, 2, 2048), (2, 3, 4096), (2, 4, 8192),
    # P = 40 -> floor 5120
    (40, 2, 5120), (40, 3, 5120), (40, 4, 8192),
])
def test_est_of_dense_blocks(P, k, expect):
    F = ofu.Fuser(8, "adaptive", 7, True, 1 << 20, 1e-12, P)
    assert F.est(_block(range(k), _haar(k, 7 * k + P))) == expect


def test_est_of_sparse_blocks():
    F = ofu.Fuser(8, "adaptive", 7, True, 1 << 20, 1e-12, 2)
    # CX: 4 real ones -> 8 ops, k = 2 -> 8 * 32 = 256 = the floor
    assert F.est(_block((0, 1), _cx_control_bit0())) == 256
    # CP(0.4): 10 ops, k = 2 -> 320
    assert F.est(_block((0, 1), _cp(0.4))) == 320
    # H: 8 ops, k = 1 -> 8 * 64 = 512
    assert F.est(_block((3,), G.H())) == 512


def _fused_qubits(gates, **kw):
    return [q for q, _, _ in ofu.fuse(max(max(g.qubits) for g in gates) + 1, gates, **kw)]


def test_merge_refused_by_estimate():
    """P = 2: a dense 2-qubit block (est 2^11) and a dense 3-qubit block
    (est 2^12) sharing one qubit make a dense 4-qubit block of est 2^13 >
    2^11 + 2^12: refused.  Size-only fusion (and P = 82, where both inputs
    sit at the floor 10496 and 2^13 < 2 * 10496) merges them."""
    gates = [_u((0, 1), 1), _u((1, 2, 3), 2)]
    assert _fused_qubits(gates, mode="adaptive", max_k=4, amp_ops_per_pass=2) == [(0, 1), (1, 2, 3)]
    assert _fused_qubits(gates, mode="adaptive", max_k=4, amp_ops_per_pass=82) == [(0, 1, 2, 3)]
    assert _fused_qubits(gates, mode="size", max_k=4) == [(0, 1, 2, 3)]


def test_merge_at_equal_estimate_is_taken():
    """P = 2: two dense 2-qubit blocks sharing a qubit (2^11 each) make a
    dense 3-qubit block of est 2^12 = 2^11 + 2^11: the test is <=, so it fuses."""
    gates = [_u((0, 1), 3), _u((1, 2), 4)]
    assert _fused_qubits(gates, mode="adaptive", max_k=3, amp_ops_per_pass=2) == [(0, 1, 2)]


def test_merge_refused_by_estimate_at_P40():
    """P = 40 (floor 5120): dense 4 (est 8192) + dense 2 (est 5120) sharing one
    qubit -> dense 5 of est 16384 > 13312: refused; at P = 82 the same pair
    (10496 + 10496 >= 16384) merges."""
    gates = [_u((0, 1, 2, 3), 5), _u((3, 4), 6)]
    assert _fused_qubits(gates, mode="adaptive", max_k=5, amp_ops_per_pass=40) == [(0, 1, 2, 3), (3, 4)]
    assert _fused_qubits(gates, mode="adaptive", max_k=5, amp_ops_per_pass=82) == [(0, 1, 2, 3, 4)]


def test_merge_refused_by_op_cap():
    """Two dense 3-qubit blocks sharing qubit 2 make a dense 5-qubit block,
    4096 operations: refused with op_cap 1024 although the estimate
    (16384 <= 2 * 10496 at P = 82) allows it; taken with the default cap 4096."""
    gates = [_u((0, 1, 2), 7), _u((2, 3, 4), 8)]
    assert _fused_qubits(gates, mode="adaptive", max_k=5, op_cap=1024) == [(0, 1, 2), (2, 3, 4)]
    assert _fused_qubits(gates, mode="adaptive", max_k=5, op_cap=4096) == [(0, 1, 2, 3, 4)]


def test_sparse_merge_under_the_op_cap():
    """CX(0,1) then CX(1,2) then CX(2,3): the fused 4-qubit block is a
    permutation (16 real ones, 32 operations), far below the cap, and its
    estimate sits at the floor: adaptive fusion takes it even with op_cap 64,
    where a dense 3-qubit block (256 operations) would be refused."""
    gates = [W.Gate("CX", (0, 1)), W.Gate("CX", (1, 2)), W.Gate("CX", (2, 3))]
    out = ofu.fuse(4, gates, mode="adaptive", max_k=4, op_cap=64)
    assert [q for q, _, _ in out] == [(0, 1, 2, 3)]
    assert out[0][2] == 32
    assert ofu.classify(out[0][1], 1e-12) == ofu.MONOMIAL
    dense = [_u((0, 1), 9), _u((1, 2), 10)]
    assert _fused_qubits(dense, mode="adaptive", max_k=4, op_cap=64) == [(0, 1), (1, 2)]


# ------------------------------------------------------------- cost table
def test_table_estimate_lookup_and_fallbacks():
    ms = [[0, 0, 0, 0],
          [0, 0.10, 0.11, 0.12],
          [0, 0.0, 0.13, 0.14],   # k = 2 diagonal missing -> the dense entry
          [0, 0.2, 0.3, 0.0],     # k = 3 dense missing -> the largest entry
          [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]]
    assert ofu.table_estimate(ms, 1, ofu.IDENTITY) == 0
    assert ofu.table_estimate(ms, 1, ofu.DIAGONAL) == 100000  # 0.10 ms in ns
    assert ofu.table_estimate(ms, 1, ofu.DENSE) == 120000
    assert ofu.table_estimate(ms, 2, ofu.DIAGONAL) == 140000
    assert ofu.table_estimate(ms, 3, ofu.DENSE) == 300000


def test_table_estimate_sparse_terms():
    """min(dense, max(floor, per_op * ops)) for dense-class gates of k >= 3;
    other classes and k < 3 ignore the sparse terms."""
    ms = [[0, 0, 0, 0]] + [[0, 0.1, 0.12, 0.5]] * 7
    cost = {"ms": ms, "sparse_floor_ms": [0, 0, 0, 0.2, 0.2, 0.2, 0.2, 0.2],
            "sparse_ms_per_op": [0, 0, 0, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4]}
    assert ofu.table_estimate(cost, 5, ofu.DENSE, 1000) == 200000    # floor 0.2 > 0.1
    assert ofu.table_estimate(cost, 5, ofu.DENSE, 4096) == 409600    # 0.4096 < 0.5
    assert ofu.table_estimate(cost, 5, ofu.DENSE, 8000) == 500000    # the dense kernel, 0.5
    assert ofu.table_estimate(cost, 2, ofu.DENSE, 10) == 500000      # k < 3: no sparse kernel
    assert ofu.table_estimate(cost, 5, ofu.DIAGONAL, 10) == 100000
    assert ofu.table_estimate(ms, 5, ofu.DENSE, 10) == 500000        # plain table: no sparse terms


def test_sparse_cost_lets_a_sparse_merge_through():
    """CX(0,1), CX(1,2) then H(2).  At size 2, CX(1,2) and H(2) fuse (a
    dense-class 2-qubit block, 0.3 ms <= 0.12 + 0.3).  At size 3 that block
    and CX(0,1) (0.12) would make a dense-class 3-qubit block of 32
    operations: with the sparse terms it costs max(0.2, 1e-4 * 32) = 0.2 ms
    <= 0.42 and fuses; with the plain table it costs the dense 0.5 ms > 0.42
    and is refused."""
    ms = [[0, 0, 0, 0]] + [[0, 0.1, 0.12, 0.3]] * 2 + [[0, 0.1, 0.12, 0.5]] * 5
    cost = {"ms": ms, "sparse_floor_ms": [0, 0, 0, 0.2, 0.2, 0.2, 0.2, 0.2],
            "sparse_ms_per_op": [0, 0, 0, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4]}
    gates = [W.Gate("CX", (0, 1)), W.Gate("CX", (1, 2)), W.Gate("H", (2,))]
    with_sparse = _fused_qubits(gates, mode="adaptive", max_k=3, cost=cost)
    without = _fused_qubits(gates, mode="adaptive", max_k=3, cost=ms)
    assert with_sparse == [(0, 1, 2)]
    assert without != [(0, 1, 2)]


def test_cost_table_decisions():
    """With measured costs: two diagonal 2-qubit gates fuse into a diagonal
    3-qubit gate when cost(3, diag) <= 2 cost(2, diag) and not otherwise;
    the class of the product, not its size alone, decides."""
    cheap = [[0, 0, 0, 0]] + [[0, 0.1, 0.1, 0.2]] * 7
    dear = [row[:] for row in cheap]
    dear[3] = [0, 0.25, 0.25, 0.3]
    gates = [W.Gate("CZ", (0, 1)), W.Gate("CP", (1, 2), (0.7,))]
    assert _fused_qubits(gates, mode="adaptive", max_k=3, cost=cheap) == [(0, 1, 2)]
    assert _fused_qubits(gates, mode="adaptive", max_k=3, cost=dear) == [(0, 1), (1, 2)]


# ---------------------------------------------------------------- schedule
def test_commuting_fusion_row_by_row():
    """H(0), H(1) land in row 0 side by side (Section IV-A: each gate goes to
    the first row below every row holding one of its qubits).  Traverse(k=2):
    no row 1, so no consecutive fusion; the commuting step looks at
    T[0][0], T[0][1], fuses them, and the product over sorted qubits (0, 1)
    is H (x) H with bit 0 <-> qubit 0, i.e. kron(H_q1, H_q0)."""
    out = ofu.fuse(2, [W.Gate("H", (0,)), W.Gate("H", (1,))], mode="size", max_k=2)
    assert len(out) == 1 and out[0][0] == (0, 1)
    assert np.max(np.abs(out[0][1] - np.kron(G.H(), G.H()))) < 1e-15


def test_commuting_fusion_needs_adjacent_slots():
    """H(0), H(2) in row 0 with slot 1 empty: the commuting step only compares
    T[r][q-1] with T[r][q], so nothing fuses (the reading of Algorithm 1)."""
    out = ofu.fuse(3, [W.Gate("H", (0,)), W.Gate("H", (2,))], mode="size", max_k=2)
    assert [q for q, _, _ in out] == [(0,), (2,)]


def test_rows_of_the_circuit_tile():
    """Section IV-A: CX(0,1), H(2), CX(1,2), H(0) give rows
    0: [CX01, CX01, H2], 1: [H0, CX12, CX12]."""
    T = ofu.Tile(3)
    blocks = [ofu.Block(g.qubits, []) for g in
              (W.Gate("CX", (0, 1)), W.Gate("H", (2,)), W.Gate("CX", (1, 2)), W.Gate("H", (0,)))]
    for b in blocks:
        T.append(b)
    assert len(T.rows) == 2
    assert T.rows[0] == [blocks[0], blocks[0], blocks[1]]
    assert T.rows[1] == [blocks[3], blocks[2], blocks[2]]


def test_size_cap_blocks_consecutive_fusion():
    gates = [W.Gate("CX", (0, 1)), W.Gate("CX", (1, 2))]
    assert _fused_qubits(gates, mode="size", max_k=2) == [(0, 1), (1, 2)]
    assert _fused_qubits(gates, mode="size", max_k=3) == [(0, 1, 2)]


def test_fused_product_order_top_acts_first():
    """Consecutive fusion multiplies U_bot * U_top: X(0) then Z(0) fuse to
    Z X = [[0, 1], [-1, 0]], not X Z."""
    out = ofu.fuse(1, [W.Gate("X", (0,)), W.Gate("Z", (0,))], mode="size", max_k=2)
    assert len(out) == 1
    assert np.max(np.abs(out[0][1] - G.Z() @ G.X())) < 1e-15


def test_agglomerative_schedule_grows_sizes():
    """A chain of 2-qubit gates on (0,1), (1,2), (2,3), (3,4): with the
    agglomerative schedule (sizes 2, 3, 4 in turn) and max_k = 4 the result
    covers every gate and has at most 4 qubits per block; the product equals
    the circuit's unitary."""
    gates = [_u((i, i + 1), 20 + i) for i in range(4)]
    out = ofu.fuse(5, gates, mode="size", max_k=4)
    assert all(len(q) <= 4 for q, _, _ in out)
    from tests.helpers import circuit_unitary
    ref = circuit_unitary(5, [(g.qubits, g.matrix) for g in gates])
    got = circuit_unitary(5, [(q, m) for q, m, _ in out])
    assert np.max(np.abs(got - ref)) < 1e-13


# --------------------------------------------------------- planted mistakes
def test_planted_shift_in_estimate_is_caught(monkeypatch):
    """est off by one shift (2^(6-k) instead of 2^(7-k)) flips the P = 40
    decision of test_merge_refused_by_estimate_at_P40."""
    def bad(self, block):
        k = len(block.qubits)
        return max(self.P * 128, self.info(block)[1] << (6 - k))
    monkeypatch.setattr(ofu.Fuser, "est", bad)
    gates = [_u((0, 1, 2, 3), 5), _u((3, 4), 6)]
    assert _fused_qubits(gates, mode="adaptive", max_k=5, amp_ops_per_pass=40) != [(0, 1, 2, 3), (3, 4)]


def test_planted_monomial_as_dense_is_caught(monkeypatch):
    """With a cost table where monomial gates cost 0.1 ms and dense ones 0.5 ms
    (k <= 2) or 1.5 ms (k = 3), CX(0,1) then CX(1,2) fuse into one 3-qubit
    permutation (0.1 <= 0.2); a classify that calls every off-diagonal matrix
    dense refuses that merge (1.5 > 1.0)."""
    table = [[0, 0, 0, 0]] + [[0, 0.1, 0.1, 0.5]] * 2 + [[0, 0.1, 0.1, 1.5]] * 5
    gates = [W.Gate("CX", (0, 1)), W.Gate("CX", (1, 2))]
    assert _fused_qubits(gates, mode="adaptive", max_k=3, cost=table) == [(0, 1, 2)]

    def bad(m, tol):
        nz = (np.abs(m.real) > tol) | (np.abs(m.imag) > tol)
        off = nz & ~np.eye(m.shape[0], dtype=bool)
        return ofu.DENSE if off.any() else ofu.DIAGONAL
    monkeypatch.setattr(ofu, "classify", bad)
    assert _fused_qubits(gates, mode="adaptive", max_k=3, cost=table) != [(0, 1, 2)]


def test_planted_wrong_product_order_is_caught(monkeypatch):
    """Fusing with the bottom block acting first breaks the unitary."""
    orig = ofu.Fuser.fusible

    def swapped(self, top, bot, k):
        f = orig(self, top, bot, k)
        if f is not None:
            f = ofu.Block(f.qubits, bot.gates + top.gates)
        return f
    monkeypatch.setattr(ofu.Fuser, "fusible", swapped)
    out = ofu.fuse(1, [W.Gate("X", (0,)), W.Gate("Z", (0,))], mode="size", max_k=2)
    assert np.max(np.abs(out[0][1] - G.Z() @ G.X())) > 0.5
