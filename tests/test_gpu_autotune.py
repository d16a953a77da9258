"""Autotuner (measured cost table) on the GPU: it measures every size and
class, installing its launch widths keeps results exact, and a plan whose
width and fusion decisions come from the table matches the oracle."""
import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture
def table_reset():
    yield
    capi.cast_set_cost_table(None)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotune_measures_and_keeps_results_exact(dtype, table_reset):
    t = capi.cast_autotune(dtype, 20)
    assert t.n_qubits == 20 and t.dtype == capi._dt(dtype)
    for k in range(1, 8):
        for c in (1, 2, 3):
            assert t.ms[k][c] > 0
            assert t.blocks_per_sm[k][c] in (1, 2, 4, 8)
    capi.cast_set_cost_table(t)
    n = 14
    gates = W.random_circuit(n, 10, 4)
    ref = oracle.simulate(n, gates)
    tol = 1e-12 if dtype == "c128" else 1e-5
    for fusion, max_k in (("none", 5), ("size", 3), ("adaptive", 0)):
        sv = pkg.StateVector(n, dtype)
        capi.cast_apply_circuit(sv.handle, n, gates, None, capi.options(fusion, max_k, cost=t))
        assert np.max(np.abs(sv.to_numpy().astype(np.complex128) - ref)) <= tol
        sv.close()
