"""cast_expectation_noalloc against the FP64 oracle and against cast_expectation (GPU).

The allocation-free call serves callers that cannot allocate device or pinned
memory (a state that already fills the GPU, an outside memory manager, loops
that must not stall on cudaMalloc/cudaFree); it keeps its partial sums in a
fixed device array inside the library.  This file is collected last, so a
failure here comes after every other test has run; it also passes on its own
in a fresh process, where the first call performs the per-device set-up.
"""
import re

import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}
SCRATCH = 65536  # CAST_NOALLOC_SCRATCH_DOUBLES


def _terms(n):
    return W.tfim_hamiltonian(n, 0.7) + [W.PauliTerm(0.3, "XZ", (0, 5)), W.PauliTerm(-1.1, "YY", (1, n - 1)),
                                         W.PauliTerm(0.7, "ZXY", (2, 0, n - 2)), W.PauliTerm(0.25, "Y", (6,))]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_matches_oracle_twice(dtype):
    n = 14
    terms = _terms(n)
    scale = sum(abs(t.coeff) for t in terms)
    psi = W.random_state(n, 21).astype(np.complex64 if dtype == "c64" else np.complex128)
    exact = oracle.expectation(psi.astype(np.complex128), terms)
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(psi)
    ref = capi.cast_expectation(sv.handle, terms)
    first = capi.cast_expectation_noalloc(sv.handle, terms)
    second = capi.cast_expectation_noalloc(sv.handle, terms)
    for v in (first, second):
        assert abs(v - exact) <= TOL[dtype] * scale
        assert abs(v - ref) <= TOL[dtype] * scale
    sv.close()


def _x_masks(n, count):
    """`count` Pauli terms with pairwise distinct X masks (one launch each)."""
    out = []
    for m in range(1, 1 << n):
        qs = tuple(q for q in range(n) if (m >> q) & 1)
        out.append(W.PauliTerm(1.0 / (1 + len(out)), "X" * len(qs), qs))
        if len(out) == count:
            return out
    raise ValueError("n too small")


def test_noalloc_scratch_boundary():
    """Sizes come from the library's own message, so the boundary holds on
    any SM count: floor((scratch - 1) / blocks) launches fit, one more is
    refused with CAST_ERR_ARG."""
    n = 12
    sv = pkg.StateVector(n, "c128", init_index=None)
    sv.from_numpy(W.random_state(n, 5))
    with pytest.raises(capi.CastError) as e:
        capi.cast_expectation_noalloc(sv.handle, _x_masks(n, (1 << n) - 1))
    assert e.value.status == 1 and "scratch" in str(e.value)
    blocks = int(re.search(r"launches x (\d+) blocks", str(e.value)).group(1))
    fit = (SCRATCH - 1) // blocks
    terms = _x_masks(n, fit)
    psi = sv.to_numpy()
    exact = oracle.expectation(psi, terms)
    got = capi.cast_expectation_noalloc(sv.handle, terms)
    assert abs(got - exact) <= 1e-12 * sum(abs(t.coeff) for t in terms)
    with pytest.raises(capi.CastError) as e:
        capi.cast_expectation_noalloc(sv.handle, _x_masks(n, fit + 1))
    assert e.value.status == 1
    sv.close()


def test_noalloc_reports_a_timed_out_wait_like_the_allocating_call():
    """A tensor-core launch whose bounded wait gave up (test hook, no fault)
    makes both expectation calls return CAST_ERR_TIMEOUT; the flag is taken
    once, and the next call succeeds."""
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    n, rng = 16, np.random.default_rng(0)
    qs, u = W.sweep_targets(n, 5, "mixed", rng), W.haar_unitary(5, rng)
    terms = _terms(n)
    for call in (capi.cast_expectation_noalloc, capi.cast_expectation):
        sv = pkg.StateVector(n, "c64")
        capi.cast_debug_inject_timeout(1 << 12)
        sv.apply_gate(qs, u)
        with pytest.raises(capi.CastError) as e:
            call(sv.handle, terms)
        assert e.value.status == 4
        sv.set_basis(0)
        assert abs(call(sv.handle, terms) - oracle.expectation(sv.to_numpy().astype(np.complex128), terms)) <= 1e-5 * 4 * n
        sv.close()
