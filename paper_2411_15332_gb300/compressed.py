"""DAX and DAS operation matrices on the device (Sec. III-A of the paper):
construction, MTP (Kronecker product) and the materialised MVM, all run by
the CUDA library."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .core import State, _stream_ptr


class _Compressed:
    _kind = None   # "dax" / "das"

    def __init__(self, handle):
        self._h = handle

    def _fn(self, name):
        return getattr(L.lib(), f"mera_{self._kind}_{name}")

    @classmethod
    def from_dense(cls, M, stream=None):
        M = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
        nq = int(round(np.log2(M.shape[0])))
        if M.shape != (1 << nq, 1 << nq):
            raise ValueError("square power-of-two matrix expected")
        h = C.c_void_p()
        L.check(getattr(L.lib(), f"mera_{cls._kind}_from_dense")(
            M.ctypes.data_as(L.DP), nq, _stream_ptr(stream), C.byref(h)))
        return cls(h)

    @classmethod
    def from_host(cls, nq, words, values, stream=None):
        w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
        v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128))
        h = C.c_void_p()
        L.check(getattr(L.lib(), f"mera_{cls._kind}_from_host")(
            int(nq), w.size, w.ctypes.data_as(L.U64P), v.ctypes.data_as(L.DP), _stream_ptr(stream), C.byref(h)))
        return cls(h)

    def kron(self, other, stream=None):
        """MTP: self (x) other, computed on the device."""
        h = C.c_void_p()
        L.check(self._fn("kron")(self._h, other._h, _stream_ptr(stream), C.byref(h)))
        return type(self)(h)

    def mvm(self, src: State, dst: State):
        """dst = M src (out of place)."""
        L.check(self._fn("mvm")(self._h, src.handle, dst.handle))

    def info(self):
        nq = C.c_int()
        nnz = C.c_uint64()
        L.check(self._fn("info")(self._h, C.byref(nq), C.byref(nnz)))
        return nq.value, nnz.value

    @property
    def nq(self):
        return self.info()[0]

    @property
    def nnz(self):
        return self.info()[1]

    @property
    def nbytes(self):
        """Bytes of the entries: 24 per non-zero (Sec. III-A.1)."""
        return 24 * self.nnz

    def export(self):
        """(index or distance words uint64, values complex128) on the host."""
        nnz = self.nnz
        w = np.empty(nnz, dtype=np.uint64)
        v = np.empty(nnz, dtype=np.complex128)
        L.check(self._fn("export")(self._h, w.ctypes.data_as(L.U64P), v.ctypes.data_as(L.DP)))
        return w, v

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._fn("destroy")(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DAX(_Compressed):
    _kind = "dax"


class DAS(_Compressed):
    _kind = "das"
