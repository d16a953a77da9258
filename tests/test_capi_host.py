"""C ABI checks that need no GPU: the library loads and exports every entry
point of include/cast.h; host-only calls (operation count, gate table, fusion
pass) against the oracle's gate table, the paper's stated numbers and brute
force; argument validation happens before any CUDA call."""
import ctypes
import json
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2503_19894_gb300 import capi
from tests.helpers import circuit_unitary, sorted_gate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cast.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cast_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("cast_sv_create", "cast_apply_gate", "cast_apply_circuit", "cast_expectation",
                 "cast_adjoint_grad"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    out = subprocess.run(["nm", "-D", "--defined-only", capi.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (cast_[a-z0-9_]+)", out))
    for name in header_functions():
        assert name in exported, f"{name} declared in cast.h but not exported"
        assert getattr(lib, name) is not None
    assert set(capi.EXPORTS) <= exported


def test_version_string():
    assert "sm_103a" in capi.cast_version()


def test_opcount_matches_paper():
    with open(os.path.join(ROOT, "tests", "golden", "paper_opcounts.json")) as f:
        gold = json.load(f)
    for p in ("X", "Y", "Z"):
        assert capi.cast_opcount(oracle.gates.matrix(p)) == 2 * gold["nonzero_scalars"][p]
    rng = np.random.default_rng(1)
    for k in range(1, 8):
        assert capi.cast_opcount(W.haar_unitary(k, rng)) == gold["opcount_dense"][str(k)]
    # zero tolerance applies per real scalar
    m = np.array([[1, 1e-13], [1e-13j, 1]], dtype=np.complex128)
    assert capi.cast_opcount(m, 1e-12) == 4
    assert capi.cast_opcount(m, 0.0) == 8


ALL_TABLE_GATES = [W.Gate("H", (3,)), W.Gate("X", (0,)), W.Gate("Y", (2,)), W.Gate("Z", (1,)),
                   W.Gate("S", (0,)), W.Gate("T", (3,)), W.Gate("RX", (1,), (0.37,)),
                   W.Gate("RY", (2,), (-1.21,)), W.Gate("RZ", (0,), (2.5,)),
                   W.Gate("U3", (3,), (0.3, -0.9, 1.7)), W.Gate("CX", (2, 0)), W.Gate("CZ", (1, 3)),
                   W.Gate("CP", (3, 1), (0.77,)), W.Gate("SWAP", (0, 2))]


def test_product_gate_table_matches_oracle_gate_table():
    """Unfused export returns each gate's matrix in sorted-qubit order; it must
    equal the oracle's independently written textbook matrix."""
    out = capi.cast_fuse(4, ALL_TABLE_GATES, opts=capi.options("none"))
    assert len(out) == len(ALL_TABLE_GATES)
    for g, (qs, m, ops) in zip(ALL_TABLE_GATES, out):
        rq, rm = sorted_gate(g.qubits, oracle.gate_matrix(g))
        assert qs == rq
        assert np.max(np.abs(m - rm)) < 1e-15, g.name


def test_parametrised_gate_reads_parameter_array():
    gates = [W.Gate("RY", (0,), pidx=1), W.Gate("CP", (0, 1), pidx=0)]
    theta = np.array([0.4, -1.3])
    out = capi.cast_fuse(2, gates, theta, opts=capi.options("none"))
    assert np.max(np.abs(out[0][1] - oracle.gates.RY(-1.3))) < 1e-15
    assert np.max(np.abs(out[1][1] - oracle.gates.CP(0.4))) < 1e-15


@pytest.mark.parametrize("mode", ["size", "adaptive"])
@pytest.mark.parametrize("agglomerative", [True, False])
@pytest.mark.parametrize("max_k", [2, 3, 5])
def test_fusion_preserves_the_circuit(mode, agglomerative, max_k):
    n = 6
    gates = W.random_circuit(n, 6, seed=max_k)
    fused = capi.cast_fuse(n, gates, opts=capi.options(mode, max_k, agglomerative))
    assert 0 < len(fused) < len(gates)
    for qs, m, ops in fused:
        assert 1 <= len(qs) <= max_k and list(qs) == sorted(qs)
        assert ops == capi.cast_opcount(m, 1e-12)
    ref = circuit_unitary(n, [(g.qubits, oracle.gate_matrix(g)) for g in gates])
    got = circuit_unitary(n, [(qs, m) for qs, m, _ in fused])
    assert np.max(np.abs(got - ref)) < 1e-12


def test_fusion_of_qft_preserves_the_circuit():
    n = 7
    gates = W.qft_circuit(n)
    fused = capi.cast_fuse(n, gates, opts=capi.options("adaptive", 4))
    ref = circuit_unitary(n, [(g.qubits, oracle.gate_matrix(g)) for g in gates])
    got = circuit_unitary(n, [(qs, m) for qs, m, _ in fused])
    assert np.max(np.abs(got - ref)) < 1e-12
    assert len(fused) < len(gates)


def test_adaptive_respects_op_cap():
    n = 8
    gates = W.random_circuit(n, 8, seed=3)
    for cap in (64, 256, 1024):
        fused = capi.cast_fuse(n, gates, opts=capi.options("adaptive", 5, op_cap=cap))
        assert all(ops <= cap or len(qs) == 1 or _is_input_gate(qs, gates) for qs, _, ops in fused)


def _is_input_gate(qs, gates):
    return any(tuple(sorted(g.qubits)) == qs for g in gates)


def test_adaptive_fuses_no_more_than_size_only():
    """Section IV-C, fusion-configuration table: adaptive fusion trades a few
    more blocks for a lower total operation count than size-only fusion."""
    n = 10
    gates = W.random_circuit(n, 10, seed=5)
    size = capi.cast_fuse(n, gates, opts=capi.options("size", 5))
    adap = capi.cast_fuse(n, gates, opts=capi.options("adaptive", 5, amp_ops_per_pass=8))
    assert len(adap) >= len(size)
    assert sum(o for *_, o in adap) <= sum(o for *_, o in size)


def _err(fn):
    with pytest.raises(capi.CastError) as e:
        fn()
    return e.value.status


def test_validation_before_any_cuda_call():
    assert _err(lambda: capi.cast_sv_create(0, "c64")) == 1
    assert _err(lambda: capi.cast_sv_create(35, "c64")) == 1
    assert _err(lambda: capi.cast_sv_create(4, 7)) == 1
    assert _err(lambda: capi.cast_sv_wrap(0, 4, "c64")) == 1
    assert _err(lambda: capi.cast_sv_wrap(0x1010, 4, "c64")) == 1  # misaligned
    bad = [
        [W.Gate("CX", (0, 0))],                 # duplicate qubit
        [W.Gate("H", (5,))],                    # qubit >= n
        [W.Gate("RY", (0,), pidx=3)],           # parameter outside the array
        [W.Gate("H", (0, 1))],                  # arity mismatch
        [W.Gate("U", tuple(range(5)), matrix=np.eye(32))],  # k > n
    ]
    for gates in bad:
        assert _err(lambda: capi.cast_fuse(4, gates, np.zeros(2))) == 1
    assert "qubit" in capi.cast_last_error() or "size" in capi.cast_last_error()
    # state calls reject a null handle before touching the device
    lib = capi.load()
    host = np.zeros(16, dtype=np.complex64)
    assert lib.cast_sv_copy_from_host_async(None, host.ctypes.data) == 1
    assert lib.cast_sv_copy_from_host(None, host.ctypes.data) == 1
    assert lib.cast_sv_set_basis(None, 0) == 1


def test_fuse_reports_required_capacity():
    lib = capi.load()
    gates = W.random_circuit(4, 2, seed=0)
    circ = capi._Circuit(4, gates, 0)
    o = capi.options("none")
    n = ctypes.c_int(1)
    st = lib.cast_fuse(ctypes.byref(circ.c), None, ctypes.byref(o), ctypes.byref(n), None, None, None, None)
    assert st == 1 and n.value == len(gates)


def test_plan_default_cost_constant_follows_the_state_type():
    """cast_plan_create (host only) with amp_ops_per_pass = 0 takes the state
    type's constant: 82 for complex64, 64 for complex128 in the emulated mode,
    2 with native FP64; the plans equal those made with the constant given."""
    import workloads as W
    n = 14
    gates = W.benchmark_family("HES", n, seed=1)[:300]
    old = capi.cast_get_f64_mode()

    def info(dtype, P):
        p = capi.cast_plan_create(n, gates, opts=capi.options("adaptive", 5, amp_ops_per_pass=P), dtype=dtype)
        out = capi.cast_plan_info(p)
        capi.cast_plan_destroy(p)
        return out

    try:
        capi.cast_set_f64_mode(capi.CAST_F64_EMULATED)
        assert info("c64", 0) == info("c64", 82)
        assert info("c128", 0) == info("c128", 64)
        capi.cast_set_f64_mode(capi.CAST_F64_NATIVE)
        assert info("c128", 0) == info("c128", 2)
        # the constants differ in effect on this circuit: 2 fuses less than 64
        assert info("c128", 2)[0] > info("c128", 64)[0]
    finally:
        capi.cast_set_f64_mode(old)


def test_options_are_validated():
    """Negative caps and constants and a non-boolean schedule flag are refused
    before any work; zero keeps its documented meaning (the default
    constant)."""
    gates = [W.Gate("H", (0,)), W.Gate("CX", (0, 1))]
    for kw in (dict(op_cap=-1), dict(amp_ops_per_pass=-5), dict(zero_tol=-1.0)):
        assert _err(lambda: capi.cast_fuse(3, gates, opts=capi.options("adaptive", 3, **kw))) == 1
    o = capi.options("adaptive", 3)
    o.agglomerative = 2
    assert _err(lambda: capi.cast_fuse(3, gates, opts=o)) == 1
    assert len(capi.cast_fuse(3, gates, opts=capi.options("adaptive", 3, amp_ops_per_pass=0))) == 1
    assert len(capi.cast_fuse(3, gates, opts=capi.options("adaptive", 3, op_cap=0))) == 2
