"""The sparsity-specialised kernels (per-row lists of tagged non-zero
entries, k = 3..7) against the oracle: every entry kind, every target
placement, both state types, small states with one tile and states of many
tiles, dense matrices through the same kernel, fused sparse-class circuits in
the default (automatic) mode, and a full-size 30-qubit gate on a basis state."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import REL, rel_err

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}
NP = {"c128": np.complex128, "c64": np.complex64}
KIND_VALUES = [1, -1, 1j, -1j]


@pytest.fixture
def sparse_mode():
    old = capi.cast_get_sparse_mode()
    yield capi
    capi.cast_set_sparse_mode(old)


def tagged_matrix(k, rng, density=0.3):
    """A 2^k x 2^k matrix whose non-zeros mix every kind: general complex,
    real, imaginary, +-1 and +-i; at least two per row (so it is not
    diagonal or monomial); scaled to spectral norm 1."""
    d = 1 << k
    m = np.zeros((d, d), dtype=np.complex128)
    for r in range(d):
        cols = rng.choice(d, size=max(2, int(density * d)), replace=False)
        for c in cols:
            kind = rng.integers(0, 4)
            if kind == 0:
                m[r, c] = rng.normal() + 1j * rng.normal()
            elif kind == 1:
                m[r, c] = rng.normal()
            elif kind == 2:
                m[r, c] = 1j * rng.normal()
            else:
                m[r, c] = KIND_VALUES[rng.integers(0, 4)]
    return m / np.linalg.norm(m, 2)


def run_gate(n, dtype, psi0, qubits, m):
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(psi0.astype(NP[dtype]))
    sv.apply_gate(qubits, m)
    out = sv.to_numpy().astype(np.complex128)
    sv.close()
    return out


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [3, 4, 5, 6, 7])
def test_sparse_kernel_every_kind_and_placement(dtype, k, sparse_mode):
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_ALWAYS)
    rng = np.random.default_rng(700 + k)
    for n in (12, 13, 16):  # one super-tile of 4096 amplitudes, two, sixteen
        psi0 = W.random_state(n, n + k)
        for placement in ("low", "high", "mixed", "mixed"):
            qs = W.sweep_targets(n, k, placement, rng)
            m = tagged_matrix(k, rng)
            got = run_gate(n, dtype, psi0, qs, m)
            ref = oracle.apply_gate(psi0.astype(NP[dtype]).astype(np.complex128), qs, m)
            err = float(np.max(np.abs(got - ref)))
            assert err <= TOL[dtype], f"n={n} {qs}: {err:.3e}"
            assert rel_err(got, ref) <= (1e-13 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [3, 5, 7])
def test_sparse_kernel_runs_dense_matrices(dtype, k, sparse_mode):
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_ALWAYS)
    rng = np.random.default_rng(810 + k)
    n = 16
    psi0 = W.random_state(n, 3)
    for placement in ("low", "mixed"):
        qs = W.sweep_targets(n, k, placement, rng)
        u = W.haar_unitary(k, rng)
        got = run_gate(n, dtype, psi0, qs, u)
        ref = oracle.apply_gate(psi0.astype(NP[dtype]).astype(np.complex128), qs, u)
        assert np.max(np.abs(got - ref)) <= TOL[dtype]
        assert rel_err(got, ref) <= (1e-13 if dtype == "c128" else 1e-6)


def test_sparse_kernel_zero_row_and_exact_units(sparse_mode):
    """A row with no entry gives exactly 0; rows of +-1 and +-i entries only
    (additions, no multiplies) match the oracle."""
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_ALWAYS)
    k, n = 3, 10
    d = 1 << k
    m = np.zeros((d, d), dtype=np.complex128)
    for r in range(1, d):  # row 0 stays empty
        m[r, (r + 1) % d] = KIND_VALUES[r % 4]
        m[r, (r + 3) % d] = -KIND_VALUES[(r + 1) % 4]
    qs = (2, 7, 4)
    for dtype in ("c128", "c64"):
        psi0 = W.random_state(n, 9).astype(NP[dtype])
        got = run_gate(n, dtype, psi0, qs, m)
        ref = oracle.apply_gate(psi0.astype(np.complex128), qs, m)
        assert np.max(np.abs(got - ref)) <= TOL[dtype]
        idx0 = [x for x in range(1 << n) if all(((x >> q) & 1) == 0 for q in qs)]
        assert np.all(got[idx0] == 0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("fam", ["IQP", "HES", "QFT", "RQC", "ALA", "QVC"])
def test_fused_families_default_mode(dtype, fam, sparse_mode):
    """The six benchmark families at 16 qubits, fused adaptively (k <= 5) and
    with size-only fusion up to 7 qubits, in the default kernel choice."""
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_AUTO)
    n = 16
    gates = W.benchmark_family(fam, n, seed=2)
    if len(gates) > 600:
        gates = gates[:600]
    ref = oracle.simulate(n, gates, init_index=5)
    for opts in (dict(fusion="adaptive", max_k=5), dict(fusion="size", max_k=7)):
        sv = pkg.StateVector(n, dtype, init_index=5)
        sv.apply_circuit(gates, **opts)
        got = sv.to_numpy().astype(np.complex128)
        sv.close()
        assert np.max(np.abs(got - ref)) <= TOL[dtype], (opts, np.max(np.abs(got - ref)))
        assert rel_err(got, ref) <= REL[dtype]


@pytest.mark.parametrize("dtype,k", [("c64", 7), ("c128", 6)])
def test_sparse_full_size_basis_column(dtype, k, sparse_mode):
    """30 qubits: a sparse gate on a basis state |x> reproduces the matrix
    column of x's target bits at the 2^k indices that differ from x in the
    targets, and the rest of the state stays zero."""
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_ALWAYS)
    n = 30
    rng = np.random.default_rng(31 + k)
    qs = W.sweep_targets(n, k, "mixed", rng)
    m = tagged_matrix(k, rng, density=0.1)
    x = int(rng.integers(0, 1 << n))
    sv = pkg.StateVector(n, dtype, init_index=x)
    sv.apply_gate(qs, m)
    jx = sum(((x >> q) & 1) << i for i, q in enumerate(qs))
    base = x & ~sum(1 << q for q in qs)
    idx = np.array([base | sum(((j >> i) & 1) << q for i, q in enumerate(qs)) for j in range(1 << k)])
    t = torch.as_tensor(idx, dtype=torch.int64, device=sv.tensor.device)
    got = sv.tensor.index_select(0, t).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - m[:, jx])) <= TOL[dtype]
    # nothing else moved: total weight equals the column's
    w = sv.expectation([W.PauliTerm(1.0, "", ())])
    assert abs(w - float(np.sum(np.abs(m[:, jx]) ** 2))) <= 10 * TOL[dtype]
    sv.close()
    torch.cuda.empty_cache()


def test_sparse_mode_validation(sparse_mode):
    with pytest.raises(capi.CastError):
        capi.cast_set_sparse_mode(9)
