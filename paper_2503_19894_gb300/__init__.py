"""GB300-native state-vector gate engine (the hot path of the CAST simulator).

The compute lives in libcast.so (hand-written CUDA for sm_103a behind the C ABI
of include/cast.h).  This package only marshals arguments:

  capi          ctypes binding, one Python function per C entry point
  StateVector   a 2^n state whose memory is a torch CUDA tensor (torch's
                caching allocator) wrapped with cast_sv_wrap; all work runs on
                torch's current CUDA stream
  AdjointEnergy torch.autograd.Function: forward returns E(theta) and keeps
                dE/dtheta from cast_adjoint_grad for the backward pass

There is no CPU fallback: without a CUDA device every call raises CastError,
and without the built library the import of capi's functions raises.
"""
from . import capi
from .capi import (CastError, cast_adjoint_grad, cast_apply_circuit, cast_apply_gate,
                   cast_expectation, cast_fuse, cast_last_error, cast_opcount, cast_sv_copy_from_host,
                   cast_sv_copy_to_host, cast_sv_create, cast_sv_destroy, cast_sv_info,
                   cast_sv_set_basis, cast_sv_wrap, cast_version, options, cast_plan_create,
                   cast_plan_apply, cast_plan_info, cast_plan_destroy, cast_profile_begin,
                   cast_profile_end)

__all__ = ["capi", "CastError", "StateVector", "AdjointEnergy", "cast_adjoint_grad",
           "cast_apply_circuit", "cast_apply_gate", "cast_expectation", "cast_fuse",
           "cast_last_error", "cast_opcount", "cast_sv_copy_from_host", "cast_sv_copy_to_host",
           "cast_sv_create", "cast_sv_destroy", "cast_sv_info", "cast_sv_set_basis",
           "cast_sv_wrap", "cast_version", "options", "cast_plan_create", "cast_plan_apply",
           "cast_plan_info", "cast_plan_destroy", "cast_profile_begin", "cast_profile_end"]


def _torch_dtype(dtype):
    import torch
    return torch.complex64 if capi._dt(dtype) == capi.CAST_C64 else torch.complex128


class StateVector:
    """2^n amplitudes in a torch CUDA tensor, initialised to |init_index>."""

    def __init__(self, n, dtype="c128", init_index=0, tensor=None):
        import torch
        self.n = int(n)
        self.dt = capi._dt(dtype)
        if tensor is None:
            tensor = torch.empty(1 << self.n, dtype=_torch_dtype(self.dt), device="cuda")
        if tensor.numel() != (1 << self.n) or tensor.dtype != _torch_dtype(self.dt) or not tensor.is_cuda \
                or not tensor.is_contiguous():
            raise ValueError("tensor must be a contiguous CUDA tensor of 2^n amplitudes of the state's type")
        self.tensor = tensor
        self.handle = cast_sv_wrap(tensor.data_ptr(), self.n, self.dt,
                                   torch.cuda.current_stream(tensor.device).cuda_stream)
        if init_index is not None:
            cast_sv_set_basis(self.handle, init_index)

    def set_basis(self, index):
        cast_sv_set_basis(self.handle, index)

    def apply_gate(self, qubits, matrix):
        cast_apply_gate(self.handle, qubits, matrix)

    def apply_circuit(self, gates, params=None, fusion="adaptive", max_k=5, **kw):
        cast_apply_circuit(self.handle, self.n, gates, params, options(fusion, max_k, **kw))

    def expectation(self, terms):
        return cast_expectation(self.handle, terms)

    def to_numpy(self, out=None):
        return cast_sv_copy_to_host(self.handle, out)

    def from_numpy(self, host):
        cast_sv_copy_from_host(self.handle, host)

    def close(self):
        if getattr(self, "handle", None):
            cast_sv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _adjoint_function():
    import torch

    class AdjointEnergy(torch.autograd.Function):
        """E(theta) = <0|U(theta)^dag H U(theta)|0>; backward uses the gradient
        that cast_adjoint_grad computed together with E (two state vectors)."""

        @staticmethod
        def forward(ctx, theta, n, gates, terms, dtype="c128"):
            import numpy as np
            psi = StateVector(n, dtype)
            lam = StateVector(n, dtype, init_index=None)
            try:
                e, g = cast_adjoint_grad(psi.handle, lam.handle, n, gates,
                                         theta.detach().cpu().numpy().astype(np.float64), terms)
            finally:
                psi.close()
                lam.close()
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return torch.tensor(e, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_e):
            (g,) = ctx.saved_tensors
            return grad_e * g, None, None, None, None

    return AdjointEnergy


def __getattr__(name):
    if name == "AdjointEnergy":
        fn = _adjoint_function()
        globals()["AdjointEnergy"] = fn
        return fn
    raise AttributeError(name)
