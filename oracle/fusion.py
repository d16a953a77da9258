"""Reference agglomerative gate fusion (Section IV, Algorithm 1), in plain Python.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written from the paper's
description, step by step, with these readings where the text is silent or
inconsistent (MoveBlock moves a block only when all of its slots below are
empty; a fused gate may reach, not only stay below, the size cap k):

CircuitTile (Section IV-A): a list of rows; each row has one slot per qubit,
holding a GateBlock or None.  A gate is appended as a new block in the first
row below every row that already holds one of its qubits.

Traverse(T, k) (Algorithm 1): for each row r, top to bottom:
  1. for each qubit q with a block b_top in T[r][q]: if every slot of b_top's
     qubits in row r+1 is empty, move b_top down to row r+1 (MoveBlock);
     otherwise let b_bot = T[r+1][q] and fuse the two when Fusible
     (consecutive fusion);
  2. for q = 1 .. n-1, fuse T[r][q-1] and T[r][q] when Fusible (commuting
     fusion).
Fuse removes both blocks and puts the product into row r+1 when all its slots
there are free, else into row r, else into a new row inserted after row r.
Fusible: two different non-empty blocks whose joint qubit set has at most k
qubits; in adaptive mode also: the product's operation count is at most the
cap, and est(product) <= est(top) + est(bottom), where, for a block of k
qubits and operation count c, est = max(P * 128, c * 2^(7-k)).
Operation count (Section IV-C): 2 x the non-zero real scalars of the matrix.
After every traversal empty rows are removed.  The agglomerative schedule
(Section IV-B) raises the allowed size from 2 to max_k and repeats Traverse
at each size until nothing is fused.

Block matrices are formed by the oracle itself: column c of a block's matrix
is the block's gate sequence applied (oracle.apply_gate) to basis vector |c>.
"""
import numpy as np

from . import apply_gate, gate_matrix


class Block:
    __slots__ = ("qubits", "gates", "info")

    def __init__(self, qubits, gates):
        self.qubits = tuple(sorted(qubits))
        self.gates = gates  # list of (qubits, matrix) in time order
        self.info = None    # (matrix, operation count), formed on first use


def block_matrix(block):
    """2^k x 2^k matrix over block.qubits (bit i <-> i-th smallest qubit)."""
    k = len(block.qubits)
    pos = {q: i for i, q in enumerate(block.qubits)}
    m = np.zeros((1 << k, 1 << k), dtype=np.complex128)
    for c in range(1 << k):
        v = np.zeros(1 << k, dtype=np.complex128)
        v[c] = 1.0
        for qs, g in block.gates:
            apply_gate(v, tuple(pos[q] for q in qs), g)
        m[:, c] = v
    return m


def opcount(m, zero_tol):
    return 2 * int(np.sum(np.abs(m.real) > zero_tol) + np.sum(np.abs(m.imag) > zero_tol))


IDENTITY, DIAGONAL, MONOMIAL, DENSE = 0, 1, 2, 3


def classify(m, zero_tol):
    """identity / diagonal / monomial (one non-zero per row and column) / dense."""
    nz = (np.abs(m.real) > zero_tol) | (np.abs(m.imag) > zero_tol)
    off = nz & ~np.eye(m.shape[0], dtype=bool)
    if not off.any():
        return IDENTITY if np.all(np.abs(np.diag(m) - 1) <= zero_tol) else DIAGONAL
    if np.all(nz.sum(axis=0) == 1) and np.all(nz.sum(axis=1) == 1):
        return MONOMIAL
    return DENSE


def table_estimate(cost, k, cls, ops=0):
    """A measured gate time in integer nanoseconds (identity costs nothing;
    a missing entry falls back to the dense entry, then to the largest).

    cost is either the table ms[k][class] or a dict holding it under "ms"
    with the sparse kernel's per-k "sparse_floor_ms" and "sparse_ms_per_op":
    a dense-class gate of k >= 3 qubits and operation count ops then costs
    min(ms[k][dense], max(floor[k], per_op[k] * ops)) (the sparse kernel's
    time grows with the operation count, Section IV-C)."""
    ms = cost["ms"] if isinstance(cost, dict) else cost
    if cls == IDENTITY:
        return 0
    v = ms[k][cls]
    if not v > 0:
        v = ms[k][DENSE]
    if not v > 0:
        v = max(ms[kk][c] for kk in range(1, len(ms)) for c in (1, 2, 3))
    if isinstance(cost, dict) and cls == DENSE and k >= 3:
        floor, per_op = cost["sparse_floor_ms"][k], cost["sparse_ms_per_op"][k]
        if floor > 0 and per_op > 0:
            v = min(v, max(floor, per_op * ops))
    return int(round(v * 1e6))


class Tile:
    def __init__(self, n):
        self.n = n
        self.rows = []

    def append(self, block):
        last = -1
        for r in range(len(self.rows) - 1, -1, -1):
            if any(self.rows[r][q] is not None for q in block.qubits):
                last = r
                break
        if last + 1 == len(self.rows):
            self.rows.append([None] * self.n)
        for q in block.qubits:
            self.rows[last + 1][q] = block

    def free(self, r, qubits):
        return 0 <= r < len(self.rows) and all(self.rows[r][q] is None for q in qubits)

    def place(self, r, block):
        for q in block.qubits:
            self.rows[r][q] = block

    def remove(self, r, block):
        for q in block.qubits:
            if self.rows[r][q] is block:
                self.rows[r][q] = None

    def compress(self):
        self.rows = [row for row in self.rows if any(b is not None for b in row)]


class Fuser:
    def __init__(self, n, mode, max_k, agglomerative, op_cap, zero_tol, amp_ops_per_pass, cost=None):
        self.T = Tile(n)
        self.mode = mode
        self.max_k = max_k
        self.agg = agglomerative
        self.op_cap = op_cap
        self.tol = zero_tol
        self.P = amp_ops_per_pass
        self.cost = cost  # ms[k][class] table (or dict, see table_estimate), or None for the operation-count model

    def info(self, block):
        if block.info is None:
            m = block_matrix(block)
            block.info = (m, opcount(m, self.tol))
        return block.info

    def est(self, block):
        k = len(block.qubits)
        if self.cost is not None:
            m, ops = self.info(block)
            return table_estimate(self.cost, k, classify(m, self.tol), ops)
        return max(self.P * 128, self.info(block)[1] << (7 - k))

    def fusible(self, top, bot, k):
        if top is None or bot is None or top is bot:
            return None
        qs = set(top.qubits) | set(bot.qubits)
        if len(qs) > k:
            return None
        fused = Block(qs, top.gates + bot.gates)  # top acts first
        if self.mode == "adaptive":
            if self.info(fused)[1] > self.op_cap:
                return None
            if self.est(fused) > self.est(top) + self.est(bot):
                return None
        return fused

    def fuse(self, r, top, r_bot, bot, fused):
        self.T.remove(r, top)
        self.T.remove(r_bot, bot)
        if self.T.free(r + 1, fused.qubits):
            self.T.place(r + 1, fused)
        elif self.T.free(r, fused.qubits):
            self.T.place(r, fused)
        else:
            self.T.rows.insert(r + 1, [None] * self.T.n)
            self.T.place(r + 1, fused)

    def traverse(self, k):
        delta = False
        r = 0
        while r < len(self.T.rows):
            for q in range(self.T.n):
                top = self.T.rows[r][q]
                if top is None:
                    continue
                if r + 1 < len(self.T.rows) and self.T.free(r + 1, top.qubits):
                    self.T.remove(r, top)  # MoveBlock
                    self.T.place(r + 1, top)
                    continue
                if r + 1 >= len(self.T.rows):
                    continue
                bot = self.T.rows[r + 1][q]
                fused = self.fusible(top, bot, k)
                if fused is not None:
                    self.fuse(r, top, r + 1, bot, fused)
                    delta = True
            for q in range(1, self.T.n):
                a, b = self.T.rows[r][q - 1], self.T.rows[r][q]
                fused = self.fusible(a, b, k)
                if fused is not None:
                    self.fuse(r, a, r, b, fused)
                    delta = True
            r += 1
        return delta

    def run(self):
        if self.mode == "none":
            return
        k0 = min(2, self.max_k) if self.agg else self.max_k
        for k in range(k0, self.max_k + 1):
            while self.traverse(k):
                self.T.compress()
            self.T.compress()

    def output(self):
        out, seen = [], set()
        for row in self.T.rows:
            for b in row:
                if b is not None and id(b) not in seen:
                    seen.add(id(b))
                    m, ops = self.info(b)
                    out.append((b.qubits, m, ops))
        return out


def fuse(n, gates, theta=None, mode="adaptive", max_k=5, agglomerative=True, op_cap=4096,
         zero_tol=1e-12, amp_ops_per_pass=82, cost=None):
    """Fused gate list [(sorted qubits, matrix, operation count)] of a
    workloads gate list.  With a cost table (ms[k][class]) the adaptive test
    compares measured times; with max_k = 0 every width 2..7 is tried and the
    plan of least estimated total time kept (ties: the smaller width)."""
    if cost is not None and max_k == 0:
        best, best_plan = None, None
        for k in range(2, 8):
            plan = fuse(n, gates, theta, mode, k, agglomerative, op_cap, zero_tol, amp_ops_per_pass, cost)
            total = sum(table_estimate(cost, len(q), classify(m, zero_tol), ops) for q, m, ops in plan)
            if best is None or total < best:
                best, best_plan = total, plan
        return best_plan
    blocks = [Block(g.qubits, [(tuple(g.qubits), gate_matrix(g, theta))]) for g in gates]
    if mode == "none":  # every gate as given, re-expressed over its sorted qubits
        out = []
        for b in blocks:
            m = block_matrix(b)
            out.append((b.qubits, m, opcount(m, zero_tol)))
        return out
    F = Fuser(n, mode, max_k, agglomerative, op_cap, zero_tol, amp_ops_per_pass, cost)
    for b in blocks:
        F.T.append(b)
    F.run()
    return F.output()
