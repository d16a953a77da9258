"""Dense-gate sweep: Haar-random k-qubit unitaries, k = 1..7, on low, high and
mixed targets, in every arithmetic mode, each scored against the FP64 oracle.

- complex64 on FP32 CUDA cores and on 3xTF32 tensor cores (k = 4..6);
- complex128 in double-float arithmetic (k <= 5) and on the FP64 pipe.
Scored at 20 qubits against the oracle, gate by gate (8 gates per case);
at 28 qubits (the full state the sweep runs on, 2 GiB complex64) the same
gates followed by their inverses must return the initial basis state.
"""
import numpy as np
import pytest

import oracle
import paper_2503_19894_gb300 as pkg
import workloads as W
from paper_2503_19894_gb300 import capi

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-12}
MODES = [("c64", "fp32"), ("c64", "tf32x3"), ("c64", "bf16x6"), ("c128", "double-float"), ("c128", "fp64")]


@pytest.fixture
def modes():
    tc, f64 = capi.cast_get_tensor_mode(), capi.cast_get_f64_mode()
    yield
    capi.cast_set_tensor_mode(tc)
    capi.cast_set_f64_mode(f64)


def set_mode(mode):
    capi.cast_set_tensor_mode({"tf32x3": capi.CAST_TC_TF32X3, "bf16x6": capi.CAST_TC_BF16X6}.get(mode, capi.CAST_TC_OFF))
    capi.cast_set_f64_mode(capi.CAST_F64_NATIVE if mode == "fp64" else capi.CAST_F64_EMULATED)


@pytest.mark.parametrize("dtype,mode", MODES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_sweep_against_fp64(dtype, mode, k, modes):
    set_mode(mode)
    n = 20
    worst = 0.0
    for placement in ("low", "high", "mixed"):
        gates = W.gate_sweep(n, k, placement, 8, 1000 * k + len(placement))
        psi0 = W.random_state(n, k).astype(np.complex64 if dtype == "c64" else np.complex128)
        ref = oracle.apply_circuit(psi0.astype(np.complex128), gates)
        sv = pkg.StateVector(n, dtype, init_index=None)
        sv.from_numpy(psi0)
        sv.apply_circuit(gates, fusion="none")
        worst = max(worst, float(np.max(np.abs(sv.to_numpy().astype(np.complex128) - ref))))
        sv.close()
    assert worst <= TOL[dtype], f"{dtype}/{mode} k={k}: {worst:.3e}"


def inverse(gates):
    return [W.Gate("U", g.qubits, matrix=g.matrix.conj().T) for g in reversed(gates)]


@pytest.mark.parametrize("mode", ["fp32", "tf32x3"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_sweep_round_trip_full_state(mode, k, modes):
    set_mode(mode)
    n = 28
    import torch
    for placement in ("low", "high", "mixed"):
        gates = W.gate_sweep(n, k, placement, 8, 7000 + 10 * k + len(placement))
        x = 12345
        sv = pkg.StateVector(n, "c64", init_index=x)
        sv.apply_circuit(gates + inverse(gates), fusion="none")
        v = sv.tensor[x].item()
        assert abs(v - 1.0) <= 10 * TOL["c64"], (placement, v)
        assert abs(sv.expectation([W.PauliTerm(1.0, "", ())]) - 1.0) <= 10 * TOL["c64"]
        sv.close()
        torch.cuda.empty_cache()


# ---------------------------------------------------------------- 30 qubits
# One gate per (k, placement, arithmetic mode) at the full size, applied in
# turn to one random state; each output is checked on 64 sampled slices,
# computed by the oracle from the same slices' inputs read back before the
# gate (slice s, member j <-> amplitude base_s + sum_i bit_i(j) 2^qubits[i]).
N_FULL = 30
N_SLICES = 64


def slice_indices(n, qs, rng):
    mask = sum(1 << q for q in qs)
    bases = rng.integers(0, 1 << n, N_SLICES, dtype=np.int64) & ~mask
    bases[0], bases[-1] = 0, ((1 << n) - 1) & ~mask
    off = np.array([sum(((j >> i) & 1) << q for i, q in enumerate(qs)) for j in range(1 << len(qs))],
                   dtype=np.int64)
    return (bases[:, None] + off[None, :]).ravel()


def sampled(sv, idx):
    import torch
    t = torch.as_tensor(idx, dtype=torch.int64, device=sv.tensor.device)
    return sv.tensor.index_select(0, t).cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_sweep_full_size_sampled(dtype, modes):
    import torch
    psi = W.random_state_device(N_FULL, dtype, 2)
    sv = pkg.StateVector(N_FULL, dtype, init_index=None, tensor=psi)
    scale = 2.0 ** (-N_FULL / 2)  # typical amplitude size
    rng = np.random.default_rng(30)
    worst = {}
    for mode in [m for d, m in MODES if d == dtype]:
        set_mode(mode)
        for k in range(1, 8):
            for placement in ("low", "high", "mixed"):
                (g,) = W.gate_sweep(N_FULL, k, placement, 1, 3000 + 10 * k + len(placement))
                idx = slice_indices(N_FULL, g.qubits, rng)
                x = sampled(sv, idx)
                sv.apply_gate(g.qubits, g.matrix)
                y = sampled(sv, idx)
                # the sampled slices as one small state: slice s in the high bits,
                # member j in the low k bits; the oracle applies U on qubits 0..k-1
                ref = oracle.apply_gate(x.copy(), tuple(range(k)), g.matrix)
                err = float(np.max(np.abs(y - ref)))
                worst[(mode, k, placement)] = err
                assert err <= TOL[dtype], (mode, k, placement, err)
                # relative to the amplitude size, too
                assert err / scale <= (1e-5 if dtype == "c64" else 1e-11), (mode, k, placement, err / scale)
    sv.close()
    del psi
    torch.cuda.empty_cache()
