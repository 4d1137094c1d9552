"""ctypes loader for the oracle's C loops (oracle.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

HID, CTX, NSYM, NCHAN = 64, 4, 256, 56


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no CUDA).  -ffp-contract=off keeps any float op unfused."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", _LIB, _SRC])
    return _LIB


class Model(ctypes.Structure):
    """Frozen integer context model, field for field as the C struct or_model."""
    _fields_ = [
        ("w1", ctypes.c_int8 * (HID * CTX)),
        ("b1", ctypes.c_int32 * (NCHAN * HID)),
        ("m1", ctypes.c_int32), ("sh1", ctypes.c_int32),
        ("w2", ctypes.c_int8 * (HID * HID)),
        ("b2", ctypes.c_int32 * HID),
        ("m2", ctypes.c_int32), ("sh2", ctypes.c_int32),
        ("w3", ctypes.c_int8 * (NSYM * HID)),
        ("b3", ctypes.c_int32 * NSYM),
        ("ms", ctypes.c_uint32), ("ss", ctypes.c_uint32),
    ]


def model_struct(m: dict) -> Model:
    s = Model()
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        arr = np.ascontiguousarray(m[k]).ravel()
        ctypes.memmove(ctypes.addressof(getattr(s, k)), arr.ctypes.data, arr.nbytes)
    for k in ("m1", "sh1", "m2", "sh2", "ms", "ss"):
        setattr(s, k, int(m[k]))
    return s


class PeModel(ctypes.Structure):
    """Frozen position-aware model, field for field as the C struct or_pe_model."""
    _fields_ = [
        ("s1", ctypes.c_float), ("s2", ctypes.c_float), ("smu", ctypes.c_float), ("slr", ctypes.c_float),
        ("b1", ctypes.c_int32 * (NCHAN * HID)),
        ("b2", ctypes.c_int32 * HID),
        ("b3", ctypes.c_int32 * 2),
        ("w1", ctypes.c_int8 * (HID * 80)),
        ("w2", ctypes.c_int8 * (HID * HID)),
        ("w3", ctypes.c_int8 * (2 * HID)),
    ]


def pe_model_struct(m: dict) -> PeModel:
    s = PeModel()
    for k, dt in (("b1", np.int32), ("b2", np.int32), ("b3", np.int32), ("w1", np.int8), ("w2", np.int8),
                  ("w3", np.int8)):
        arr = np.ascontiguousarray(np.asarray(m[k]).astype(dt)).ravel()
        ctypes.memmove(ctypes.addressof(getattr(s, k)), arr.ctypes.data, arr.nbytes)
    for k in ("s1", "s2", "smu", "slr"):
        setattr(s, k, float(m[k]))
    return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        L.or_rans_encode.restype = i64
        L.or_rans_encode.argtypes = [i64, i64, P, P, P, P, i64, P, P]
        L.or_rans_decode_static.restype = ctypes.c_int
        L.or_rans_decode_static.argtypes = [i64, P, P, P, ctypes.c_int, P, i64, P, P, P]
        L.or_rans_decode_static16.restype = ctypes.c_int
        L.or_rans_decode_static16.argtypes = [i64, P, P, P, ctypes.c_int, P, i64, P, P, P]
        L.or_model_logits.restype = None
        L.or_model_logits.argtypes = [P, P, ctypes.c_int, P]
        L.or_logits_to_freq.restype = None
        L.or_logits_to_freq.argtypes = [P, u32, u32, P, P]
        L.or_learned_freq.restype = None
        L.or_learned_freq.argtypes = [P, P, P, i64, i64, ctypes.c_int, P]
        L.or_learned_fc.restype = None
        L.or_learned_fc.argtypes = [P, P, P, P, i64, i64, P, P]
        L.or_rans_decode_learned.restype = ctypes.c_int
        L.or_rans_decode_learned.argtypes = [P, P, P, i64, i64, P, i64, P, P, P]
        L.or_calib_max.restype = None
        L.or_calib_max.argtypes = [P, P, i32, i32, P, P, P, P, P, P, i64, P, P]
        L.or_model_size.restype = ctypes.c_int
        L.or_pe_model_size.restype = ctypes.c_int
        assert L.or_pe_model_size() == ctypes.sizeof(PeModel)
        L.or_pe_phi.restype = None
        L.or_pe_phi.argtypes = [P, ctypes.c_int, P, P]
        L.or_pe_head.restype = None
        L.or_pe_head.argtypes = [P, P, ctypes.c_int, P, P, P]
        L.or_pe_cdf.restype = u32
        L.or_pe_cdf.argtypes = [i32, i32, ctypes.c_int, P]
        L.or_rans_decode_pe.restype = ctypes.c_int
        L.or_rans_decode_pe.argtypes = [P, P, P, P, i64, ctypes.c_int, P, i64, i64, P, i64, P, P, P]
        assert L.or_model_size() == ctypes.sizeof(Model)
        _lib = L
    return _lib


def ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)
