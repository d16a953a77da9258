"""The tensor-pipe measurements (cast_measure_tensor_peak,
cast_measure_mma_issue): plausible values and the relations the kernels'
designs rely on, and argument validation."""
import pytest

from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu


def test_tensor_peaks_are_plausible():
    """Dense kind::tf32 and bf16 peaks of a GB300 (nominal 1.1 / 2.25 PFLOP/s
    dense): bf16 close to twice tf32."""
    tf32 = capi.cast_measure_tensor_peak(capi.CAST_PEAK_TF32)
    bf16 = capi.cast_measure_tensor_peak(capi.CAST_PEAK_BF16)
    assert 300.0 < tf32 < 1500.0
    assert 600.0 < bf16 < 3000.0
    assert 1.6 < bf16 / tf32 < 2.4


def test_small_mmas_cost_their_issue():
    """An M = 128, K = 16 MMA takes about the same time for every N up to 64
    and about twice as long at N = 256 as at N = 128 (the arithmetic then
    sets the pace), whether A comes from tensor memory or shared memory."""
    for a_tmem in (True, False):
        c = {n: capi.cast_measure_mma_issue(n, a_tmem) for n in (16, 32, 64, 128, 256)}
        assert all(v > 0 for v in c.values()), c
        assert max(c[16], c[32], c[64]) < 1.3 * min(c[16], c[32], c[64]), c
        assert 1.6 < c[256] / c[128] < 2.4, c
        assert c[64] > 0.6 * c[128], c  # N = 64 is far from a quarter of N = 256


def test_mma_issue_validation():
    for bad in (0, 8, 24, 272):
        with pytest.raises(capi.CastError):
            capi.cast_measure_mma_issue(bad, True)
