"""cast_expectation_noalloc against cast_expectation (GPU).

The allocation-free call serves callers that cannot allocate device or pinned
memory (a state that already fills the GPU, an outside memory manager, loops
that must not stall on cudaMalloc/cudaFree); it keeps its partial sums in a
fixed device array inside the library.  This file is collected last, so a
failure here comes after every other test has run; it also passes on its own
in a fresh process, where the first call performs the per-device set-up.
"""
import numpy as np
import pytest

import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}


def _terms(n):
    return W.tfim_hamiltonian(n, 0.7) + [W.PauliTerm(0.3, "XZ", (0, 5)), W.PauliTerm(-1.1, "YY", (1, n - 1)),
                                         W.PauliTerm(0.7, "ZXY", (2, 0, n - 2)), W.PauliTerm(0.25, "Y", (6,))]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_matches_allocating_call_twice(dtype):
    n = 14
    terms = _terms(n)
    scale = sum(abs(t.coeff) for t in terms)
    sv = pkg.StateVector(n, dtype, init_index=None)
    sv.from_numpy(W.random_state(n, 21).astype(np.complex64 if dtype == "c64" else np.complex128))
    ref = capi.cast_expectation(sv.handle, terms)
    first = capi.cast_expectation_noalloc(sv.handle, terms)
    second = capi.cast_expectation_noalloc(sv.handle, terms)
    assert abs(first - ref) <= TOL[dtype] * scale
    assert abs(second - ref) <= TOL[dtype] * scale
    sv.close()


def test_noalloc_rejects_sums_beyond_the_fixed_scratch():
    n = 12
    # 66 distinct X-pair masks -> 66 launches; beyond 107 launches the call must refuse
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    terms = [W.PauliTerm(1.0, "XX", p) for p in pairs]  # 66 launches: fits
    sv = pkg.StateVector(n, "c128")
    assert abs(capi.cast_expectation_noalloc(sv.handle, terms) - capi.cast_expectation(sv.handle, terms)) < 1e-12
    many = terms + [W.PauliTerm(1.0, "XXX", (i, j, k)) for i in range(n) for j in range(i + 1, n)
                    for k in range(j + 1, n)][:80]
    with pytest.raises(capi.CastError) as e:
        capi.cast_expectation_noalloc(sv.handle, many)
    assert e.value.status == 1 and "scratch" in str(e.value)
    sv.close()
