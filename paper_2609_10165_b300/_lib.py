"""ctypes declarations of the C ABI in include/ebr.h (argument marshalling only).

Loading fails loudly when the CUDA library has not been built: there is no
fallback implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libebr.so")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

STATUS = {
    0: "EBR_OK", -1: "EBR_EINVAL", -2: "EBR_ENOMEM", -3: "EBR_ECUDA", -4: "EBR_ECYCLE",
    -5: "EBR_ESTENCIL_OOB", -6: "EBR_ESTENCIL_SOLID", -7: "EBR_ETIMEOUT", -8: "EBR_ENONFINITE",
    -9: "EBR_ESHAPE",
}


class Grid(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("reserved", c_int32), ("n", c_int64 * 3),
                ("lo", c_double * 3), ("hi", c_double * 3)]


class Body(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("centre", c_double * 3),
                ("radii", c_double * 3), ("rot", c_double * 9), ("thickness", c_double),
                ("chord", c_double)]


class GeomCounts(ctypes.Structure):
    _fields_ = [("n_cells", c_int64), ("n_interface", c_int64), ("n_ghosts", c_int64),
                ("n_levels", c_int32), ("reserved", c_int32)]


_SIGS = {
    "ebr_create": (c_int32, [ctypes.POINTER(c_void_p)]),
    "ebr_destroy": (None, [c_void_p]),
    "ebr_last_error": (ctypes.c_char_p, [c_void_p]),
    "ebr_plan": (c_int32, [c_void_p, c_int32, ctypes.POINTER(Grid), ctypes.POINTER(Body), c_int32,
                           c_void_p, c_void_p]),
    "ebr_plan_faces": (c_int32, [c_void_p, c_int32, ctypes.POINTER(Grid), ctypes.POINTER(c_void_p),
                                 ctypes.POINTER(Body), c_int32, c_void_p, c_void_p]),
    "ebr_classify": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ebr_classify_levels": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ebr_move": (c_int32, [c_void_p, ctypes.POINTER(Body), c_void_p, c_void_p]),
    "ebr_layout": (c_int32, [c_void_p, ctypes.POINTER(c_int64)]),
    "ebr_counts": (c_int32, [c_void_p, ctypes.POINTER(GeomCounts)]),
    "ebr_build_levels": (c_int32, [c_void_p, c_void_p]),
    "ebr_ghost_info": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_void_p, c_void_p]),
    "ebr_reconstruct": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_void_p),
                                  ctypes.POINTER(c_int32), ctypes.POINTER(c_void_p), c_int32,
                                  c_int32, c_void_p]),
    "ebr_boundary_forces": (c_int32, [c_void_p, ctypes.POINTER(c_void_p), c_void_p, c_int32,
                                      c_double, ctypes.POINTER(c_double), c_void_p, c_void_p]),
    "ebr_reconstruct_adjoint": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32),
                                          ctypes.POINTER(c_int32), c_int32, c_double,
                                          ctypes.POINTER(c_double), c_void_p,
                                          ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                          c_int32, c_int32, c_int32, c_void_p]),
    "ebr_reconstruct_packed": (c_int32, [c_void_p, c_int32, c_void_p, ctypes.POINTER(c_int32),
                                         c_void_p, c_int32, c_void_p]),
    "ebr_reconstruct_packed_adjoint": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_int32), c_void_p,
                                                 c_void_p, c_int32, c_void_p]),
    "ebr_tiled_plan": (c_int32, [c_void_p, ctypes.POINTER(c_int32), c_void_p]),
    "ebr_reconstruct_tiled": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_int32),
                                        ctypes.POINTER(c_void_p), c_int32, c_void_p]),
    "ebr_tiled_info": (c_int32, [c_void_p, ctypes.POINTER(c_int64), c_int32]),
    "ebr_tiled_lists": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "ebr_tiled_wait_test": (c_int32, [c_void_p, c_int32]),
    "ebr_stats": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p]),
    "ebr_sync_status": (c_int32, [c_void_p, c_void_p]),
    "ebr_diagnostics": (c_int32, [c_void_p, ctypes.POINTER(c_int64), c_int32, c_void_p]),
    "ebr_launch_count": (c_int64, [c_void_p]),
    "ebr_set_pdl": (None, [c_int32]),
    "ebr_get_pdl": (c_int32, []),
    "ebr_profile": (c_int32, [c_void_p, c_int32]),
    "ebr_profile_read": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32]),
    "ebr_profile_timeline": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "ebr_tunable_kernels": (c_int32, [c_void_p, c_int32]),
    "ebr_set_block_size": (c_int32, [c_void_p, ctypes.c_char_p, c_int32]),
    "ebr_get_block_size": (c_int32, [c_void_p, ctypes.c_char_p]),
    "ebr_classify_cells_static": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Body), c_void_p,
                                            c_void_p, c_void_p]),
}

EXPORTED = tuple(_SIGS)

_lib = None


def load(path=LIB_PATH):
    """Load libebr.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build() or "
                           "python -m paper_2609_10165_b300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EBRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code
        self.name = STATUS.get(code, "?")
