"""Failure detection without a GPU fault: a tensor-core launch whose MMA
completion never arrives (test hook) gives up after its bounded wait, the host
reports CAST_ERR_TIMEOUT, and the context keeps working."""
import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [4, 5, 6, 7])
def test_bounded_wait_reports_timeout_and_context_survives(k):
    """k = 4: the warps' hand-off barrier and the MMA completion barrier;
    k = 5: MMA completion barrier; k = 6, 7: also the W-chunk bulk-copy
    pipeline."""
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    n, rng = 16, np.random.default_rng(0)
    qs, u = W.sweep_targets(n, k, "mixed", rng), W.haar_unitary(k, rng)
    sv = pkg.StateVector(n, "c64")
    capi.cast_debug_inject_timeout(1 << 12)
    sv.apply_gate(qs, u)  # queued; the failure surfaces at the next synchronisation
    with pytest.raises(capi.CastError) as e:
        sv.to_numpy()
    assert e.value.status == 4 and "bounded wait" in str(e.value)
    # the error was taken; the same state and the context keep working
    sv.set_basis(0)
    psi0 = W.random_state(n, 3).astype(np.complex64)
    sv.from_numpy(psi0)
    sv.apply_gate(qs, u)
    ref = oracle.apply_gate(psi0.astype(np.complex128), qs, u)
    assert np.max(np.abs(sv.to_numpy().astype(np.complex128) - ref)) <= 1e-5
    sv.close()


def test_inject_rejects_zero_limit():
    with pytest.raises(capi.CastError):
        capi.cast_debug_inject_timeout(0)


def test_bounded_wait_in_the_complex128_digit_kernel():
    """The complex128 digit kernel (k = 4, MMA completion barrier): the same
    hook, the same report, and the next gate on the same state is exact."""
    old = capi.cast_get_c128_tensor_mode()
    capi.cast_set_c128_tensor_mode(capi.CAST_C128_TC_OZAKI)
    try:
        n, rng = 16, np.random.default_rng(1)
        qs, u = W.sweep_targets(n, 4, "mixed", rng), W.haar_unitary(4, rng)
        sv = pkg.StateVector(n, "c128")
        capi.cast_debug_inject_timeout(1 << 12)
        capi.cast_profile_begin()
        sv.apply_gate(qs, u)
        with pytest.raises(capi.CastError) as e:
            sv.to_numpy()
        assert e.value.status == 4 and "bounded wait" in str(e.value)
        assert [p["name"] for p in capi.cast_profile_end()] == ["ozdense_k4_c128"]
        sv.set_basis(0)
        psi0 = W.random_state(n, 3)
        sv.from_numpy(psi0)
        sv.apply_gate(qs, u)
        ref = oracle.apply_gate(psi0.copy(), qs, u)
        assert np.max(np.abs(sv.to_numpy() - ref)) <= 1e-12
        sv.close()
    finally:
        capi.cast_set_c128_tensor_mode(old)
