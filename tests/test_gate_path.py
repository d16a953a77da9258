"""Kernel choice on the host (cast_gate_path, the same decision chain
cast_apply_gate launches through): the documented dispatch of every gate
class, size and state type, the crossover densities between the complex128
digit kernel and the list kernel (Section IV-C's operation count), and the
effect of each mode setting.  No GPU is needed."""
import numpy as np
import pytest

import workloads as W
from paper_2503_19894_gb300 import capi

DIGIT, LIST, CHUNKED, TENSOR, DF, CORE = (capi.CAST_PATH_DIGIT, capi.CAST_PATH_LIST,
                                          capi.CAST_PATH_TENSOR_CHUNKED, capi.CAST_PATH_TENSOR,
                                          capi.CAST_PATH_DOUBLE_FLOAT, capi.CAST_PATH_CUDA_CORE)


@pytest.fixture(autouse=True)
def default_modes():
    saved = (capi.cast_get_tensor_mode(), capi.cast_get_f64_mode(), capi.cast_get_c128_tensor_mode(),
             capi.cast_get_sparse_mode())
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    capi.cast_set_f64_mode(capi.CAST_F64_EMULATED)
    capi.cast_set_c128_tensor_mode(capi.CAST_C128_TC_OZAKI)
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_AUTO)
    yield
    capi.cast_set_tensor_mode(saved[0])
    capi.cast_set_f64_mode(saved[1])
    capi.cast_set_c128_tensor_mode(saved[2])
    capi.cast_set_sparse_mode(saved[3])


def path(n, dt, k, m):
    return capi.cast_gate_path(n, dt, tuple(range(k)), m)


def haar(k, seed=0):
    return W.haar_unitary(k, np.random.default_rng(seed))


def with_ops(k, ops):
    """A real dense-class matrix whose operation count (2 per non-zero real
    scalar) is exactly `ops`: the diagonal first, then off-diagonal entries
    row by row (every row with two or more entries keeps the class dense)."""
    d = 1 << k
    assert ops % 2 == 0 and d < ops // 2 <= d * d
    m = np.zeros((d, d))
    cells = [(r, r) for r in range(d)] + [(r, c) for r in range(d) for c in range(d) if c != r]
    for r, c in cells[:ops // 2]:
        m[r, c] = 0.25 + 0.01 * ((r * 7 + c * 3) % 11)
    assert capi.cast_opcount(m) == ops
    return m


def test_default_dispatch_of_dense_unitaries():
    assert [path(20, "c64", k, haar(k)) for k in range(1, 8)] == [CORE, CORE, CORE, TENSOR, TENSOR, CHUNKED, CHUNKED]
    assert [path(20, "c128", k, haar(k)) for k in range(1, 8)] == [DF, DF, DIGIT, DIGIT, DIGIT, DIGIT, DIGIT]


def test_diagonal_monomial_identity():
    d4 = np.diag(np.exp(1j * np.arange(16)))
    assert path(20, "c64", 4, d4) == CORE
    assert path(20, "c128", 4, d4) == DF
    assert path(20, "c128", 6, np.diag(np.exp(1j * np.arange(64)))) == CORE  # double-float covers k <= 5
    perm = np.eye(8)[[3, 1, 2, 0, 5, 4, 7, 6]] * 1j
    assert path(20, "c128", 3, perm) == DF
    assert path(20, "c128", 3, np.eye(8)[[3, 1, 2, 0, 5, 4, 7, 6]]) == CORE  # unit phases: moves only
    assert path(20, "c64", 5, np.eye(32)) == CORE


@pytest.mark.parametrize("k,num,den", [(3, 1, 3), (4, 1, 6), (5, 1, 9), (6, 1, 10), (7, 1, 20)])
def test_complex128_crossover_densities(k, num, den):
    """Dense-class complex128 gates go to the digit kernel when their
    operation count exceeds num/den of the dense count (measured crossover
    with the list kernel), else to the list kernel."""
    dense = 1 << (2 * k + 2)
    edge = dense * num / den
    below = int(edge) - (int(edge) % 2)          # largest even count <= the edge
    above = below + 2
    assert path(20, "c128", k, with_ops(k, below)) == LIST
    assert path(20, "c128", k, with_ops(k, above)) == DIGIT


def test_size_limits():
    """Tensor-core and digit kernels need n >= k + 7, the list kernel n >= 12."""
    assert path(11, "c64", 5, haar(5)) == CORE
    assert path(12, "c64", 5, haar(5)) == TENSOR
    assert path(11, "c128", 5, haar(5)) == DF
    assert path(12, "c128", 5, haar(5)) == DIGIT
    assert path(13, "c128", 6, haar(6)) == DIGIT
    assert path(12, "c128", 6, haar(6)) == LIST   # below k + 7: the list kernel
    assert path(11, "c128", 6, haar(6)) == CORE   # below 12 as well; no double-float kernel for k = 6


def test_modes():
    capi.cast_set_tensor_mode(capi.CAST_TC_BF16X6)
    assert [path(20, "c64", k, haar(k)) for k in (4, 5, 6, 7)] == [TENSOR, TENSOR, CHUNKED, CHUNKED]
    capi.cast_set_tensor_mode(capi.CAST_TC_OFF)
    assert [path(20, "c64", k, haar(k)) for k in (4, 5, 6, 7)] == [CORE] * 4
    assert path(20, "c64", 5, with_ops(5, 400)) == LIST  # sparse enough for the list kernel
    capi.cast_set_tensor_mode(capi.CAST_TC_TF32X3)
    # non-unitary dense complex64: not on the tensor cores
    assert path(20, "c64", 5, 2.0 * haar(5)) == CORE
    capi.cast_set_c128_tensor_mode(capi.CAST_C128_TC_OFF)
    assert [path(20, "c128", k, haar(k)) for k in (3, 5, 7)] == [LIST] * 3
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_OFF)
    assert [path(20, "c128", k, haar(k)) for k in (3, 5, 7)] == [DF, DF, CORE]
    capi.cast_set_c128_tensor_mode(capi.CAST_C128_TC_OZAKI)
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_ALWAYS)
    assert path(20, "c128", 5, haar(5)) == LIST and path(20, "c64", 5, haar(5)) == LIST
    capi.cast_set_sparse_mode(capi.CAST_SPARSE_AUTO)
    capi.cast_set_f64_mode(capi.CAST_F64_NATIVE)
    assert [path(20, "c128", k, haar(k)) for k in (1, 3, 5, 7)] == [CORE] * 4


def test_arguments_are_validated():
    for args in ((0, "c64", (0,), np.eye(2)), (35, "c64", (0,), np.eye(2)),
                 (4, "c64", (0, 0), np.eye(4)), (4, "c64", (4,), np.eye(2))):
        with pytest.raises(capi.CastError):
            capi.cast_gate_path(*args)
    bad = np.eye(2, dtype=complex)
    bad[0, 0] = np.nan
    with pytest.raises(capi.CastError):
        capi.cast_gate_path(4, "c64", (0,), bad)
