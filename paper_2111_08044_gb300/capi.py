"""ctypes binding of the C ABI declared in include/floquet_sv.h.

Argument marshalling only: every step of the evolution runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfloquetsv.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "floquet_sv.h")

SV_OK = 0
SV_EINVAL = -1
SV_ENOMEM = -2
SV_ECUDA = -3
SV_ETIMEOUT = -4
SV_ESTATE = -5
SV_EUNSUPPORTED = -6
SV_C64 = 0
SV_C128 = 1
SV_DF64 = 2
SV_MODE_PLAIN = 0
SV_MODE_BLOCK = 1
SV_MODE_MULTIGATE = 2
SV_SPLIT_BF16X3 = 0
SV_SPLIT_FP32 = 1
SV_BATCH_AUTO = -1
SV_BATCH_PLAIN = 0
SV_BATCH_BLOCK_SIMT = 1
SV_BATCH_BLOCK_TC = 2
SV_BATCH_RESIDENT = 3
SV_BATCH_MULTIGATE = 4

_ERRNAMES = {SV_EINVAL: "SV_EINVAL", SV_ENOMEM: "SV_ENOMEM", SV_ECUDA: "SV_ECUDA",
             SV_ETIMEOUT: "SV_ETIMEOUT", SV_ESTATE: "SV_ESTATE",
             SV_EUNSUPPORTED: "SV_EUNSUPPORTED"}


class SvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sv_floquet_params(ctypes.Structure):
    _fields_ = [
        ("J", ctypes.c_double),
        ("hx", ctypes.c_double),
        ("hz", ctypes.c_double),
        ("T", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("edge_field_weight", ctypes.c_double),
        ("K", ctypes.c_int32),
        ("first_layer", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("block_n", ctypes.c_int32),
        ("split", ctypes.c_int32),
        ("renorm_every", ctypes.c_int32),
        ("n_period_params", ctypes.c_int64),
        ("theta_p", ctypes.POINTER(ctypes.c_double)),
        ("hx_p", ctypes.POINTER(ctypes.c_double)),
        ("inverse", ctypes.c_int32),
        ("h_bonds", ctypes.POINTER(ctypes.c_double)),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t
_pp = ctypes.POINTER(sv_floquet_params)

SIGNATURES = {
    "sv_version": ([], _i32),
    "sv_create": ([ctypes.POINTER(_vp), _i32, _i32, _vp], _i32),
    "sv_attach_state": ([_vp, _vp, _sz], _i32),
    "sv_init": ([_vp, _i32, _dp], _i32),
    "sv_build_floquet": ([_vp, _pp], _i32),
    "sv_evolve": ([_vp, _i64, _dp, _dp], _i32),
    "sv_evolve_profiled": ([_vp, _i64, _dp, _dp, _dp], _i32),
    "sv_expect_energy": ([_vp, _dp, _dp], _i32),
    "sv_renormalize": ([_vp, _dp], _i32),
    "sv_adjoint": ([_vp, _i64, _dp, _dp, _dp], _i32),
    "sv_get_state": ([_vp, _vp, _sz], _i32),
    "sv_set_state": ([_vp, _vp, _sz, _i64], _i32),
    "sv_save": ([_vp, ctypes.c_char_p], _i32),
    "sv_set_layout_policy": ([_vp, _i32], _i32),
    "sv_load": ([_vp, ctypes.c_char_p], _i32),
    "sv_checkpoint_info": ([ctypes.c_char_p, _ip, _ip, ctypes.POINTER(_i64)], _i32),
    "sv_period_counter": ([_vp], _i64),
    "sv_pass_info": ([_vp, _ip, _ip, _ip], _i32),
    "sv_build_bytes": ([_vp, ctypes.POINTER(_sz)], _i32),
    "sv_form_info": ([_vp, _ip, _ip], _i32),
    "sv_energy_noalloc": ([_vp, _i32, _i32, _pp, _dp, _vp], _i32),
    "sv_last_error": ([_vp], ctypes.c_char_p),
    "sv_destroy": ([_vp], None),
    "sv_host_bond_gates": ([_i32, _pp, _dp, _dp], _i32),
    "sv_host_period_gates": ([_i32, _pp, _ip, _ip, _dp], _i32),
    "sv_host_fusion_plan": ([_i32, _pp, _i32, _ip, _ip, _ip, _dp], _i32),
    "sv_energy_moments": ([_vp, _dp, _dp, _dp], _i32),
    "sv_overlap_product": ([_vp, _dp, _dp, _dp], _i32),
    "sv_init_pairs": ([_vp, _i32, _dp], _i32),
    "sv_overlap_pairs": ([_vp, _dp, _dp, _dp], _i32),
    "sv_host_pass_operand": ([_i32, _pp, _i32, _i32, _i32, _dp], _i32),
    "sv_host_block_layout": ([_i32, _pp, _i32, _ip, _ip, _ip, _vp, _ip, _ip, _vp], _i32),
    "sv_host_store_view": ([_i32, _pp, _i32, _i32, _ip, _vp, _vp, _vp, _ip], _i32),
    "sv_batch_state_bytes": ([_i32, _ip], _sz),
    "sv_batch_create": ([ctypes.POINTER(_vp), _i32, _i32, _ip, _pp, _dp, _vp, _sz, _i32, _vp],
                        _i32),
    "sv_batch_evolve": ([_vp, _i64, _dp, _dp], _i32),
    "sv_batch_forms": ([_vp, _ip], _i32),
    "sv_batch_widths": ([_vp, _ip], _i32),
    "sv_batch_last_error": ([_vp], ctypes.c_char_p),
    "sv_batch_destroy": ([_vp], None),
}

_lib = None


def load(path: Optional[str] = None):
    """Load libfloquetsv.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
            " (the simulator has no CPU fallback)")
    lib = ctypes.CDLL(p)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def header_symbols():
    """Names of the functions include/floquet_sv.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sv_\w+)\s*\(", text, re.M)))


def check(rc: int, ctx=None, what: str = ""):
    if rc != SV_OK:
        msg = ""
        if ctx is not None:
            m = load().sv_last_error(ctx)
            msg = m.decode() if m else ""
        raise SvError(rc, f"{what}: {msg}".strip(": "))
    return rc


def make_params(J=1.0, hx=0.9, hz=0.4, T=0.5, theta=0.3, edge_field_weight=0.5, K=4,
                first_layer=0, mode=SV_MODE_PLAIN, block_n=0, split=SV_SPLIT_BF16X3,
                renorm_every=0, theta_p=None, hx_p=None, inverse=0, h_bonds=None):
    """sv_floquet_params plus the arrays it points to (keep both alive)."""
    import numpy as np
    p = sv_floquet_params()
    p.J, p.hx, p.hz, p.T, p.theta = J, hx, hz, T, theta
    p.edge_field_weight = edge_field_weight
    p.K, p.first_layer, p.mode, p.block_n, p.split = K, first_layer, mode, block_n, split
    p.renorm_every = renorm_every
    p.inverse = int(inverse)
    keep = []
    n = 0
    for name, arr in (("theta_p", theta_p), ("hx_p", hx_p)):
        if arr is not None:
            a = np.ascontiguousarray(arr, dtype=np.float64)
            keep.append(a)
            n = a.size
            setattr(p, name, a.ctypes.data_as(_dp))
    p.n_period_params = n
    if h_bonds is not None:
        hb = np.ascontiguousarray(h_bonds, dtype=np.complex128)
        keep.append(hb)
        p.h_bonds = hb.ctypes.data_as(_dp)
    return p, keep
