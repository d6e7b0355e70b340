"""Thin ctypes binding of the C ABI in ``include/ccm.h``.

Every function of the header is available under the same name through
``lib()``; this module only marshals arguments (pointers, sizes, the current
CUDA stream of a torch tensor) and turns status codes into exceptions.  All
computation happens in the CUDA library ``libccm.so``; there is no fallback:
if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libccm.so")

CCM_OK, CCM_ERR_INVALID, CCM_ERR_OOM, CCM_ERR_CUDA, CCM_ERR_TIMEOUT, CCM_ERR_BUSY, \
    CCM_ERR_NOT_READY, CCM_ERR_UNKNOWN_TICKET = range(8)
STATUS_NAMES = ["CCM_OK", "CCM_ERR_INVALID", "CCM_ERR_OOM", "CCM_ERR_CUDA", "CCM_ERR_TIMEOUT",
                "CCM_ERR_BUSY", "CCM_ERR_NOT_READY", "CCM_ERR_UNKNOWN_TICKET"]
CCM_FLAG_NO_CULL = 1
CCM_N_COUNTERS = 8
CCM_SAVED_FLOATS = 28
COUNTER_NAMES = ["dirs", "dirs_live", "maxpass", "gatepass", "eval_grad", "eval_val",
                 "contacts", "features"]
BWD_COUNTER_NAMES = ["dirs", "dirs_live", "maxpass", "gatepass", "p1_grad", "p1_val", "p2_hv",
                     "p2_grad"]


class CcmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class ccm_params(C.Structure):
    _fields_ = [("tau_sdf", C.c_float), ("tau_trace", C.c_float), ("tau_clip", C.c_float),
                ("tau_blend", C.c_float), ("d_max", C.c_float), ("gate_width", C.c_float),
                ("trace_iters", C.c_int32), ("flags", C.c_uint32)]


class ccm_body_desc(C.Structure):
    _fields_ = [("n_pieces", C.c_int32), ("nv", C.c_void_p), ("nf", C.c_void_p),
                ("ne", C.c_void_p), ("verts", C.c_void_p), ("planes", C.c_void_p),
                ("edges", C.c_void_p)]


class ccm_tuning(C.Structure):
    _fields_ = [("item_v", C.c_int32), ("item_e", C.c_int32), ("item_vb", C.c_int32),
                ("item_eb", C.c_int32), ("fwd_warps", C.c_int32), ("groups", C.c_int32),
                ("stage_planes", C.c_int32), ("stage_verts", C.c_int32),
                ("groups_b", C.c_int32), ("flat_records", C.c_int32),
                ("stage_tma", C.c_int32), ("stage_wait", C.c_int32),
                ("flat_forward", C.c_int32), ("pdl", C.c_int32)]


class ccm_spline_desc(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("dims", C.c_void_p), ("coef", C.c_void_p)]


class ccm_serve_config(C.Structure):
    _fields_ = [("max_wave_pairs", C.c_int64), ("max_wave_requests", C.c_int64),
                ("max_queued", C.c_int64), ("params", ccm_params), ("tuning", ccm_tuning)]


class ccm_serve_counters(C.Structure):
    _fields_ = [("waves", C.c_int64), ("served", C.c_int64), ("wave_pairs", C.c_int64),
                ("wave_items", C.c_int64), ("gpu_s", C.c_double), ("form_s", C.c_double)]


class ccm_request(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("A", C.c_void_p), ("B", C.c_void_p),
                ("pose_a", C.c_void_p), ("pose_b", C.c_void_p), ("y", C.c_void_p),
                ("ybar", C.c_void_p), ("grad", C.c_void_p)]


_SIGS = {
    "ccm_default_params": (None, [C.c_void_p]),
    "ccm_create": (C.c_int, [C.c_int, C.c_size_t, C.c_void_p]),
    "ccm_destroy": (None, [C.c_void_p]),
    "ccm_last_error": (C.c_char_p, []),
    "ccm_load_geometry": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ccm_free_geometry": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "ccm_output_size": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_batch_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_batch_destroy": (None, [C.c_void_p]),
    "ccm_batch_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_batch_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ccm_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ccm_contacts": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "ccm_contacts_counted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_contacts_backward": (C.c_int, [C.c_void_p] * 10),
    "ccm_contacts_backward_noalloc": (C.c_int, [C.c_void_p] * 10),
    "ccm_contacts_save": (C.c_int, [C.c_void_p] * 7),
    "ccm_contacts_backward_saved": (C.c_int, [C.c_void_p] * 11),
    "ccm_contacts_step_host": (C.c_int, [C.c_void_p] * 11),
    "ccm_serve_replay": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
    "ccm_contacts_backward_counted": (C.c_int, [C.c_void_p] * 12),
    "ccm_peak_probe": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_default_serve_config": (None, [C.c_void_p]),
    "ccm_serve_start": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ccm_serve_stop": (C.c_int, [C.c_void_p]),
    "ccm_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ccm_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "ccm_serve_hold": (C.c_int, [C.c_void_p, C.c_int]),
    "ccm_poll_completed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "ccm_serve_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ccm_attach_splines": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    "ccm_batch_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ccm_build_voxel_grids": (C.c_int, [C.c_void_p, C.c_int]),
    "ccm_kernel_launches": (C.c_int, [C.c_void_p]),
}


def kernel_launches() -> int:
    """Kernels the library has launched in this process (host-side count)."""
    n = C.c_int64()
    check(lib().ccm_kernel_launches(C.byref(n)))
    return n.value

_lib = None


def exported_symbols():
    """Names of the C ABI functions the binding expects (from ccm.h)."""
    return list(_SIGS)


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with "
                               "`python -m paper_2604_17538_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != CCM_OK:
        msg = lib().ccm_last_error()
        raise CcmError(status, msg.decode() if msg else "")


def default_params(**kw) -> ccm_params:
    p = ccm_params()
    lib().ccm_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_serve_config(**kw) -> ccm_serve_config:
    c = ccm_serve_config()
    lib().ccm_default_serve_config(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def ptr(t):
    """Device or host address of a torch tensor or numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def stream_of(t):
    import torch
    return torch.cuda.current_stream(t.device).cuda_stream
