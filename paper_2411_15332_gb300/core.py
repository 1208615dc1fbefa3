"""Python face of the state-vector library: argument marshalling only.

Every step runs in the CUDA library behind include/mera.h; torch provides
the device memory (the state is a torch tensor wrapped with
``mera_state_wrap``) and the stream (torch's current stream).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _stream_ptr(stream=None):
    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


class State:
    """A 2^n-amplitude state vector on the current CUDA device.

    dtype: "c128" (float64 re/im, the paper's precision) or "c64".
    The amplitudes live in ``self.tensor`` (torch, shape [2^n, 2] real) and
    start as |0...0>.
    """

    def __init__(self, n: int, dtype: str = "c128", device=None, stream=None, tensor=None):
        if dtype not in ("c128", "c64"):
            raise ValueError("dtype must be 'c128' or 'c64'")
        self.n = int(n)
        self.dtype = dtype
        self._code = L.MERA_C128 if dtype == "c128" else L.MERA_C64
        real = torch.float64 if dtype == "c128" else torch.float32
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if tensor is None:
            tensor = torch.empty((1 << self.n, 2), dtype=real, device=dev)
        elif tensor.dtype != real or tensor.numel() != 2 << self.n or not tensor.is_contiguous():
            raise ValueError("tensor must be contiguous, 2^(n+1) real elements of the state dtype")
        self.tensor = tensor
        self._stream = stream
        h = C.c_void_p()
        L.check(L.lib().mera_state_wrap(C.c_void_p(tensor.data_ptr()), self.n, self._code,
                                        _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.set_basis(0)

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().mera_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self._stream = stream
        L.check(L.lib().mera_state_set_stream(self._h, _stream_ptr(stream)))

    def synchronize(self):
        L.check(L.lib().mera_state_synchronize(self._h))

    # -- contents --------------------------------------------------------
    def set_basis(self, index: int = 0):
        L.check(L.lib().mera_state_set_basis(self._h, int(index)))

    def from_numpy(self, psi: np.ndarray):
        dt = np.complex128 if self.dtype == "c128" else np.complex64
        a = np.ascontiguousarray(np.asarray(psi, dtype=dt))
        if a.size != 1 << self.n:
            raise ValueError("wrong length")
        L.check(L.lib().mera_state_copy_from_host(self._h, C.c_void_p(a.ctypes.data)))

    def from_host_async(self, psi):
        """Enqueue the upload of ``psi`` (a contiguous array of the state's
        complex dtype, ideally page-locked, e.g. a pinned torch tensor's
        numpy view) on the state's stream and return at once; ``psi`` must
        stay alive and unchanged until the stream has passed the copy."""
        dt = np.complex128 if self.dtype == "c128" else np.complex64
        if not isinstance(psi, np.ndarray) or psi.dtype != dt or psi.size != 1 << self.n or \
                not psi.flags["C_CONTIGUOUS"]:
            raise ValueError("psi must be a contiguous array of 2^n amplitudes of the state's dtype")
        L.check(L.lib().mera_state_copy_from_host_async(self._h, C.c_void_p(psi.ctypes.data)))

    def to_numpy(self) -> np.ndarray:
        dt = np.complex128 if self.dtype == "c128" else np.complex64
        out = np.empty(1 << self.n, dtype=dt)
        L.check(L.lib().mera_state_copy_to_host(self._h, C.c_void_p(out.ctypes.data)))
        return out

    def amplitudes(self, idx) -> np.ndarray:
        """Amplitudes at the given basis indices, as complex128."""
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64).reshape(-1))
        out = np.empty(2 * ix.size, dtype=np.float64)
        L.check(L.lib().mera_state_get_amplitudes(
            self._h, ix.ctypes.data_as(L.U64P), ix.size, out.ctypes.data_as(L.DP)))
        return out[0::2] + 1j * out[1::2]

    # -- gates -----------------------------------------------------------
    def apply_gate(self, name: str, targets=(), controls=(), params=()):
        t = (C.c_int * max(1, len(targets)))(*targets)
        c = (C.c_int * max(1, len(controls)))(*controls)
        ps = list(params)
        if name in ("U", "U3") and len(ps) == 3:
            ps.append(0.0)
        p = (C.c_double * max(1, len(ps)))(*ps)
        L.check(L.lib().mera_apply_gate(self._h, L.GATE_ID[name], t, len(targets), c, len(controls),
                                        p if ps else None))

    def apply_matrix(self, matrix, targets, controls=()):
        m = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
        t = (C.c_int * len(targets))(*targets)
        c = (C.c_int * max(1, len(controls)))(*controls)
        L.check(L.lib().mera_apply_matrix(self._h, m.ctypes.data_as(L.DP), t, len(targets), c, len(controls)))

    def apply_circuit(self, ops, mode: str = "fused"):
        arr, keep = L.ops_to_array(ops)
        md = L.MODE_FUSED if mode == "fused" else L.MODE_PER_GATE
        L.check(L.lib().mera_apply_circuit(self._h, C.c_void_p(arr.ctypes.data), len(arr), md))
        del keep

    def apply_circuit_observe(self, ops, q: int = 0, mode: str = "fused"):
        """apply_circuit then observables(q) in one call: (norm^2, <Z_q>,
        sum_q <Z_q>).  In fused mode the circuit's last pass sums the readout
        while it writes the state when it can (see mera_apply_circuit_observe)."""
        arr, keep = L.ops_to_array(ops)
        md = L.MODE_FUSED if mode == "fused" else L.MODE_PER_GATE
        out = (C.c_double * 3)()
        L.check(L.lib().mera_apply_circuit_observe(self._h, C.c_void_p(arr.ctypes.data), len(arr), md, int(q), out))
        del keep
        return tuple(out)

    def hadamard_layer(self, mask: int):
        """H on every qubit in ``mask`` (the RH structure, Sec. III-B)."""
        L.check(L.lib().mera_hadamard_layer(self._h, int(mask)))

    # -- readouts --------------------------------------------------------
    def norm2(self) -> float:
        v = C.c_double()
        L.check(L.lib().mera_norm2(self._h, C.byref(v)))
        return v.value

    def expect_z(self, q: int) -> float:
        v = C.c_double()
        L.check(L.lib().mera_expect_z(self._h, int(q), C.byref(v)))
        return v.value

    def expect_z_sum(self) -> float:
        v = C.c_double()
        L.check(L.lib().mera_expect_z_sum(self._h, C.byref(v)))
        return v.value

    def observables(self, q: int = 0):
        out = (C.c_double * 3)()
        L.check(L.lib().mera_observables(self._h, int(q), out))
        return tuple(out)

    def argmax(self):
        i = C.c_uint64()
        p = C.c_double()
        L.check(L.lib().mera_argmax(self._h, C.byref(i), C.byref(p)))
        return int(i.value), p.value

    def measure(self, us) -> np.ndarray:
        u = np.ascontiguousarray(np.asarray(us, dtype=np.float64))
        out = np.empty(u.size, dtype=np.uint64)
        L.check(L.lib().mera_measure(self._h, u.ctypes.data_as(L.DP), u.size, out.ctypes.data_as(L.U64P)))
        return out.astype(np.int64)


def gate_matrix(name: str, params=()) -> np.ndarray:
    """The library's matrix of a catalogue gate."""
    ps = list(params)
    if name in ("U", "U3") and len(ps) == 3:
        ps.append(0.0)
    p = (C.c_double * 4)(*(ps + [0.0] * (4 - len(ps))))
    nt = C.c_int()
    out = (C.c_double * 128)()
    L.check(L.lib().mera_gate_matrix(L.GATE_ID[name], p, C.byref(nt), out))
    d = 1 << nt.value
    a = np.array(out[: 2 * d * d])
    return (a[0::2] + 1j * a[1::2]).reshape(d, d)


def plan_summary(n: int, ops, dtype: str = "c128") -> str:
    """How the fused mode would run ``ops`` (host only, no GPU needed): a
    header line (tile bits, passes, whether the state stays fixed point), then one line
    per pass (engine, Hadamard levels, phases, op kinds, the kernel that
    runs it, gathers / scatters, resident scaling); see mera_plan_summary."""
    arr, keep = L.ops_to_array(ops)
    buf = C.create_string_buffer(1 << 20)
    npass = C.c_int()
    L.check(L.lib().mera_plan_summary(int(n), L.MERA_C128 if dtype == "c128" else L.MERA_C64,
                                      C.c_void_p(arr.ctypes.data), len(arr), buf, len(buf), C.byref(npass)))
    del keep
    return buf.value.decode()


RH_METHODS = ("nonopt", "quarter", "block", "log")


def rh_mvm(src: State, dst: State, method: str = "log", block: int = 0) -> int:
    """The paper's RH-MVM dst = H^(x)n src (Sec. III-B.2, Algorithm 1) with
    one of its four sign methods (RH_METHODS); returns the number of sign
    computations (Table II).  Out of place, complex128, 2 <= n <= 18."""
    cnt = C.c_uint64()
    L.check(L.lib().mera_rh_mvm(src.handle, dst.handle, RH_METHODS.index(method), int(block), C.byref(cnt)))
    return int(cnt.value)


def launch_count() -> int:
    return int(L.lib().mera_launch_count())


def profile_enable(on: bool = True):
    L.check(L.lib().mera_profile_enable(1 if on else 0))


def profile_read():
    """{class: (launches, ms, algorithmic bytes)} since profile_enable."""
    n = (C.c_uint64 * L.KCLASS_COUNT)()
    ms = (C.c_double * L.KCLASS_COUNT)()
    by = (C.c_double * L.KCLASS_COUNT)()
    L.check(L.lib().mera_profile_read(n, ms, by))
    return {L.KCLASS_NAMES[k]: (int(n[k]), float(ms[k]), float(by[k])) for k in range(L.KCLASS_COUNT)}
