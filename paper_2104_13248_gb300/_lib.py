"""ctypes binding of libbp.so (declarations of include/bp.h, unet.h and iter.h).

Argument marshalling only: every computation runs in the CUDA library. The
library is loaded from paper_2104_13248_gb300/_build/libbp.so; a missing or
unloadable library raises immediately (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

BP_OK, BP_ERR_INVALID_ARG, BP_ERR_UNSUPPORTED, BP_ERR_OOM, BP_ERR_CUDA, BP_ERR_TIMEOUT, BP_ERR_DEVICE = range(7)
BP_F32, BP_F16 = 0, 1
STATUS_NAMES = {0: "BP_OK", 1: "BP_ERR_INVALID_ARG", 2: "BP_ERR_UNSUPPORTED", 3: "BP_ERR_OOM",
                4: "BP_ERR_CUDA", 5: "BP_ERR_TIMEOUT", 6: "BP_ERR_DEVICE"}


class bp_geometry(ctypes.Structure):
    _fields_ = [("sid", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("u_off_px", ctypes.c_double), ("v_off_px", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("sx", ctypes.c_double), ("sy", ctypes.c_double), ("sz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_d = ctypes.c_double
_ll = ctypes.c_longlong
_dptr = ctypes.POINTER(ctypes.c_double)
_iptr = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); the symbols every header declaration maps to
PROTOTYPES = {
    "bp_create": (_i, [ctypes.POINTER(bp_geometry), ctypes.POINTER(_vp)]),
    "bp_create_from_matrices": (_i, [_dptr, _i, _i, _i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "bp_filter": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "bp_filter_views": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "bp_backproject": (_i, [_vp, _vp, _i, _vp, _i, _f, _i, _vp]),
    "bp_backproject_views": (_i, [_vp, _vp, _i, _i, _i, _ll, _vp, _i, _f, _i, _vp]),
    "bp_backproject_slab": (_i, [_vp, _vp, _i, _i, _i, _ll, _i, _i, _i, _vp, _i, _f, _i, _vp]),
    "fp_project": (_i, [_vp, _vp, _vp, _i, _f, _vp]),
    "bp_phantom_project": (_i, [_vp, _dptr, _i, _vp, _vp]),
    "bp_get_matrices": (_i, [_vp, _dptr]),
    "bp_get_dims": (_i, [_vp, _iptr, _iptr, _iptr, _iptr, _iptr, _iptr]),
    "bp_device_status": (_i, [_vp, _vp]),
    "bp_set_tuning": (_i, [_vp, _i, _i]),
    "bp_set_pipeline_depth": (_i, [_vp, _i]),
    "bp_set_symmetry": (_i, [_vp, _i]),
    "bp_set_timeout": (_i, [_vp, _d]),
    "bp_test_drop_view": (_i, [_vp, _i]),
    "bp_test_live_allocations": (_i, []),
    "bp_get_plan": (_i, [_vp, _iptr, _iptr, _iptr, _iptr, _iptr, _iptr]),
    "bp_last_error": (ctypes.c_char_p, [_vp]),
    "bp_destroy": (None, [_vp]),
    # unet.h
    "cnn_conv3d_forward": (_i, [_vp, _i, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_conv3d_dgrad": (_i, [_vp, _i, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_conv3d_dgrad_noalloc": (_i, [_vp, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_conv3d_wgrad": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_head_forward": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_head_backward": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_maxpool2_forward": (_i, [_vp, _i, _i, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_maxpool2_backward": (_i, [_vp, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_upsample2_forward": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_upsample2_backward": (_i, [_vp, _i, _i, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_relu_backward": (_i, [_vp, _i, _i, _vp, _i, _i, _ll, _i, _vp]),
    "cnn_pack_input": (_i, [_vp, _vp, _i, _ll, _vp]),
    "cnn_stem_forward": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_stem_pool_forward": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_stem_wgrad": (_i, [_vp, _vp, _i, _i, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_conv3d_forward_head": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_head1_forward": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _ll, _i, _vp]),
    "cnn_head1_backward": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _ll, _i, _vp]),
    "cnn_upsample2_add_forward": (_i, [_vp, _vp, _i, _i, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "cnn_upsample2_add_head1_forward": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "cnn_mse": (_i, [_vp, _vp, _vp, _vp, _ll, _vp]),
    "cnn_adam": (_i, [_vp, _vp, _vp, _vp, _vp, _ll, _f, _f, _f, _f, _i, _vp]),
    "cnn_set_tensor_path": (_i, [_i]),
    "cnn_device_status": (_i, [_vp]),
    # include/iter.h
    "it_fill": (_i, [_vp, _ll, _f, _vp]),
    "it_ratio": (_i, [_vp, _vp, _vp, _ll, _f, _vp]),
    "it_residual": (_i, [_vp, _vp, _vp, _vp, _ll, _f, _vp]),
    "it_mlem_update": (_i, [_vp, _vp, _vp, _ll, _f, _vp]),
    "it_sart_update": (_i, [_vp, _vp, _vp, _ll, _f, _i, _f, _vp]),
    "it_ls_residual": (_i, [_vp, _vp, _vp, _ll, _vp, _vp]),
    "it_scale": (_i, [_vp, _vp, _vp, _ll, _vp]),
    "it_gd_step": (_i, [_vp, _vp, _ll, _f, _vp]),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libbp.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libbp.so is not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class BPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, ctx=None):
    if status != BP_OK:
        msg = load().bp_last_error(ctx).decode(errors="replace")
        raise BPError(status, msg)
