"""ctypes declarations of the C ABI in include/mera.h.

The library is the in-tree build ``_build/libmera.so``.  Loading fails
loudly when it is missing: there is no other implementation behind these
names.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libmera.so")

MERA_OK, MERA_EINVAL, MERA_ENOMEM, MERA_EUNSUPPORTED, MERA_ECUDA, MERA_ETIMEOUT = range(6)
MERA_C64, MERA_C128 = 0, 1
MODE_PER_GATE, MODE_FUSED = 0, 1
(KCLASS_GATE, KCLASS_TILE, KCLASS_REDUCE, KCLASS_DAX, KCLASS_QNN, KCLASS_HPASS, KCLASS_DPASS,
 KCLASS_GATE_DIAG, KCLASS_GATE_1Q, KCLASS_RH, KCLASS_AMP) = range(11)
KCLASS_COUNT = 11
KCLASS_NAMES = ("gate", "tile", "reduce", "dax", "qnn", "hpass", "dpass", "gate_diag", "gate_1q", "rh", "amp")

GATES = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SX", "SXDG", "P", "RX", "RY", "RZ",
         "R", "U2", "U", "SWAP", "ISWAP", "DCX", "ECR", "RXX", "RYY", "RZZ", "RZX", "FLIP", "MATRIX"]
GATE_ID = {g: i for i, g in enumerate(GATES)}
GATE_ID["U1"] = GATE_ID["P"]
GATE_ID["U3"] = GATE_ID["U"]

# struct mera_op (include/mera.h), 80 bytes
OP_DTYPE = np.dtype({
    "names": ["gate", "nt", "targets", "reserved", "cmask", "cvals", "params", "matrix"],
    "formats": [np.int32, np.int32, (np.int32, 3), np.int32, np.uint64, np.uint64, (np.float64, 4), np.uint64],
    "offsets": [0, 4, 8, 20, 24, 32, 40, 72],
    "itemsize": 80,
})


class MeraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mera error {code}: {msg}")
        self.code = code


_lib = None

P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I = C.c_int
U64 = C.c_uint64
D = C.c_double
DP = C.POINTER(C.c_double)
U64P = C.POINTER(C.c_uint64)
IP = C.POINTER(C.c_int)
SZ = C.c_size_t

PROTOS = {
    "mera_last_error": (C.c_char_p, []),
    "mera_version": (C.c_char_p, []),
    "mera_launch_count": (U64, []),
    "mera_state_create": (I, [I, I, PP]),
    "mera_state_wrap": (I, [P, I, I, P, PP]),
    "mera_state_destroy": (I, [P]),
    "mera_state_set_stream": (I, [P, P]),
    "mera_state_info": (I, [P, PP, IP, IP]),
    "mera_state_set_basis": (I, [P, U64]),
    "mera_state_copy_from_host": (I, [P, P]),
    "mera_state_copy_to_host": (I, [P, P]),
    "mera_state_get_amplitudes": (I, [P, U64P, SZ, DP]),
    "mera_state_synchronize": (I, [P]),
    "mera_state_copy_from_host_async": (I, [P, P]),
    "mera_gate_matrix": (I, [I, DP, IP, DP]),
    "mera_apply_gate": (I, [P, I, IP, I, IP, I, DP]),
    "mera_apply_matrix": (I, [P, DP, IP, I, IP, I]),
    "mera_apply_circuit": (I, [P, P, SZ, I]),
    "mera_apply_circuit_observe": (I, [P, P, SZ, I, I, DP]),
    "mera_hadamard_layer": (I, [P, U64]),
    "mera_plan_summary": (I, [I, I, P, SZ, C.c_char_p, SZ, IP]),
    "mera_norm2": (I, [P, DP]),
    "mera_expect_z": (I, [P, I, DP]),
    "mera_expect_z_sum": (I, [P, DP]),
    "mera_observables": (I, [P, I, DP]),
    "mera_observables_noalloc": (I, [P, I, I, I, P, DP]),
    "mera_argmax": (I, [P, U64P, DP]),
    "mera_measure": (I, [P, DP, SZ, U64P]),
    "mera_dax_from_dense": (I, [DP, I, P, PP]),
    "mera_das_from_dense": (I, [DP, I, P, PP]),
    "mera_dax_from_host": (I, [I, U64, U64P, DP, P, PP]),
    "mera_das_from_host": (I, [I, U64, U64P, DP, P, PP]),
    "mera_dax_kron": (I, [P, P, P, PP]),
    "mera_das_kron": (I, [P, P, P, PP]),
    "mera_dax_mvm": (I, [P, P, P]),
    "mera_das_mvm": (I, [P, P, P]),
    "mera_dax_info": (I, [P, IP, U64P]),
    "mera_das_info": (I, [P, IP, U64P]),
    "mera_dax_export": (I, [P, U64P, DP]),
    "mera_das_export": (I, [P, U64P, DP]),
    "mera_dax_destroy": (I, [P]),
    "mera_das_destroy": (I, [P]),
    "mera_batch_create": (I, [I, I, I, P, PP]),
    "mera_batch_destroy": (I, [P]),
    "mera_batch_info": (I, [P, PP, IP, IP, IP]),
    "mera_batch_set_stream": (I, [P, P]),
    "mera_batch_copy_to_host": (I, [P, I, P]),
    "mera_batch_reset": (I, [P, IP, I]),
    "mera_batch_layer": (I, [P, IP, I, DP]),
    "mera_batch_forward": (I, [P, I, I, DP]),
    "mera_batch_observables": (I, [P, IP, I, I, DP]),
    "mera_adjoint_grad": (I, [P, I, I, DP, DP, DP]),
    "mera_rh_mvm": (I, [P, P, I, I, U64P]),
    "mera_test_bulk_shortfall": (I, [C.c_uint]),
    "mera_profile_enable": (I, [I]),
    "mera_profile_read": (I, [U64P, DP, DP]),
}


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2411_15332_gb300.build.build() "
                               "(the CUDA library is the only implementation)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != MERA_OK:
        raise MeraError(code, lib().mera_last_error().decode())


def ops_to_array(ops):
    """Gate list (inputs.Op tuples) -> numpy array of struct mera_op, plus
    the matrices kept alive for MATRIX ops."""
    arr = np.zeros(len(ops), dtype=OP_DTYPE)
    keep = []
    for j, (name, targets, controls, params, cvals) in enumerate(ops):
        arr[j]["gate"] = GATE_ID[name] if isinstance(name, str) else GATE_ID["MATRIX"]
        arr[j]["nt"] = len(targets)
        for t, q in enumerate(targets):
            arr[j]["targets"][t] = q
        cm = 0
        cv = 0
        for c_idx, q in enumerate(controls):
            cm |= 1 << q
            if (cvals >> c_idx) & 1:
                cv |= 1 << q
        arr[j]["cmask"] = cm
        arr[j]["cvals"] = cv
        ps = list(params)
        if isinstance(name, str) and name in ("U", "U3") and len(ps) == 3:
            ps.append(0.0)
        for t, v in enumerate(ps):
            arr[j]["params"][t] = v
        if not isinstance(name, str):          # an explicit matrix
            m = np.ascontiguousarray(np.asarray(name, dtype=np.complex128))
            keep.append(m)
            arr[j]["matrix"] = m.ctypes.data
    return arr, keep
