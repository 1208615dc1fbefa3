"""Batched QNN ansatz states, expectations and adjoint gradients (binding
of the mera_batch_* and mera_adjoint_grad calls in include/mera.h).

The ansatz stands in for the paper's QNN neuron (Sec. IV-D): L layers of
RY(theta[l, 0, q]) and RZ(theta[l, 1, q]) on every qubit q, then the CNOT
ring q -> q+1 mod n.  Angles have shape [..., L, 2, n].
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .core import _stream_ptr


class Batch:
    """``capacity`` slot states of n qubits on the current device."""

    def __init__(self, n: int, capacity: int, dtype: str = "c64", stream=None):
        self.n, self.capacity, self.dtype = int(n), int(capacity), dtype
        code = L.MERA_C128 if dtype == "c128" else L.MERA_C64
        h = C.c_void_p()
        L.check(L.lib().mera_batch_create(self.n, self.capacity, code, _stream_ptr(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().mera_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        L.check(L.lib().mera_batch_set_stream(self._h, _stream_ptr(stream)))

    @staticmethod
    def _ints(slots):
        a = np.ascontiguousarray(np.asarray(slots, dtype=np.int32))
        return a, a.ctypes.data_as(L.IP)

    def reset(self, slots):
        a, p = self._ints(slots)
        L.check(L.lib().mera_batch_reset(self._h, p, a.size))

    def layer(self, slots, theta_layer):
        """One ansatz layer; theta_layer[len(slots), 2, n]."""
        a, p = self._ints(slots)
        th = np.ascontiguousarray(np.asarray(theta_layer, dtype=np.float64).reshape(a.size, 2, self.n))
        L.check(L.lib().mera_batch_layer(self._h, p, a.size, th.ctypes.data_as(L.DP)))

    def forward(self, theta):
        """Slots 0..B-1 from |0>: theta[B, L, 2, n]."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        B, Ly = th.shape[0], th.shape[1]
        L.check(L.lib().mera_batch_forward(self._h, B, Ly, th.ctypes.data_as(L.DP)))

    def observables(self, slots, q: int = 0) -> np.ndarray:
        """[len(slots), 3]: norm^2, <Z_q>, sum_q <Z_q> (float64)."""
        a, p = self._ints(slots)
        out = np.empty((a.size, 3), dtype=np.float64)
        L.check(L.lib().mera_batch_observables(self._h, p, a.size, int(q), out.ctypes.data_as(L.DP)))
        return out

    def states(self, slots) -> np.ndarray:
        """Copy of the listed slot states (host, complex)."""
        dt = np.complex128 if self.dtype == "c128" else np.complex64
        out = np.empty((len(slots), 1 << self.n), dtype=dt)
        for j, s in enumerate(slots):
            L.check(L.lib().mera_batch_copy_to_host(self._h, int(s), C.c_void_p(out[j].ctypes.data)))
        return out

    def adjoint_grad(self, theta):
        """loss[B] = sum_q <Z_q> and grad[B, L, 2, n] by adjoint differentiation."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        B, Ly = th.shape[0], th.shape[1]
        loss = np.empty(B, dtype=np.float64)
        grad = np.empty(th.shape, dtype=np.float64)
        L.check(L.lib().mera_adjoint_grad(self._h, B, Ly, th.ctypes.data_as(L.DP), loss.ctypes.data_as(L.DP),
                                          grad.ctypes.data_as(L.DP)))
        return loss, grad


class AdjointExpectation(torch.autograd.Function):
    """loss = mean over the batch of sum_q <Z_q>, gradients by the adjoint
    kernels.  theta: float64 tensor [B, L, 2, n] (any device)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, batch: "Batch"):
        th = theta.detach().to("cpu", torch.float64).contiguous().numpy()
        loss, grad = batch.adjoint_grad(th)
        B = th.shape[0]
        ctx.save_for_backward(torch.from_numpy(grad / B).to(theta.device, theta.dtype))
        return torch.tensor(float(loss.mean()), dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None
