"""ctypes binding of libsps.so (include/sps.h): argument marshalling only.

Every numerical step runs inside the CUDA library.  Torch tensors supply
device memory and the CUDA stream; the wrappers pass raw pointers.  There is
no fallback: if the library cannot be loaded, or a call fails, an exception is
raised.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsps.so")

SPS_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED",
          5: "BREAKDOWN", 6: "CAPACITY", 7: "NO_GEOMETRY", 8: "NONFINITE"}
SPS_FP64, SPS_MIXED, SPS_FP64_DW = 0, 1, 2
SPS_OP_S, SPS_OP_K, SPS_OP_A = 0, 1, 2
SPS_MOB_BIE, SPS_MOB_IDENTITY = 0, 1
SPS_SEARCH_AUTO, SPS_SEARCH_ALL_PAIRS, SPS_SEARCH_CELLS = 0, 1, 2


class sps_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("beta", ctypes.c_double), ("delta", ctypes.c_double),
                ("a_c_scale", ctypes.c_double), ("gmres_tol", ctypes.c_double),
                ("gmres_max", ctypes.c_int), ("bbpgd_tol", ctypes.c_double),
                ("bbpgd_max", ctypes.c_int), ("precision", ctypes.c_int),
                ("bb_variant", ctypes.c_int), ("ir_tol", ctypes.c_double), ("ir_max", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("bb_safeguard", ctypes.c_int),
                ("mobility", ctypes.c_int), ("contact_search", ctypes.c_int),
                ("delta_rel", ctypes.c_double), ("bb_warm", ctypes.c_int), ("ir_dw", ctypes.c_int),
                ("lcp_solver", ctypes.c_int)]


class sps_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("mobility_solves", ctypes.c_int),
                ("gmres_iters", ctypes.c_int), ("gmres_iters_max", ctypes.c_int),
                ("bbpgd_iters", ctypes.c_int), ("mvops", ctypes.c_int),
                ("n_contacts", ctypes.c_int), ("n_active", ctypes.c_int),
                ("n_near_pairs", ctypes.c_int), ("ir_sweeps", ctypes.c_int),
                ("bb_safeguards", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong), ("final_phi", ctypes.c_double),
                ("gmres_res_max", ctypes.c_double), ("layer_applies", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "sps_default_params": (_I, [ctypes.POINTER(sps_params)]),
    "sps_create": (_I, [ctypes.POINTER(sps_params), _P, ctypes.POINTER(_P)]),
    "sps_destroy": (_I, [_P]),
    "sps_last_error": (ctypes.c_char_p, [_P]),
    "sps_set_geometry": (_I, [_P, _I, _P, _P]),
    "sps_nodes": (_I, [_P, _P, _P, _P, ctypes.POINTER(_I)]),
    "sps_geometry_counts": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "sps_near_lists": (_I, [_P, _P, _P]),
    "sps_set_orientation": (_I, [_P, _I, _P]),
    "sps_set_walls": (_I, [_P, _I, _P]),
    "sps_layer_apply": (_I, [_P, _I, _P, _P]),
    "sps_build_contacts": (_I, [_P, _I, _P, _P, ctypes.POINTER(_I)]),
    "sps_get_contacts": (_I, [_P, _P, _P, _P]),
    "sps_contact_force": (_I, [_P, _P, _P]),
    "sps_contact_rate": (_I, [_P, _P, _P]),
    "sps_mobility_apply": (_I, [_P, _I, _P, _P, _P, _P, ctypes.POINTER(sps_stats)]),
    "sps_resolve_collisions": (_I, [_P, _I, _P, _P, _P, _D, _P, _I, _P, _P,
                                    ctypes.POINTER(sps_stats)]),
    "sps_resolve_collisions_host": (_I, [_P, _I, _P, _P, _P, _D, _P, _I, _P, _P,
                                         ctypes.POINTER(_I), ctypes.POINTER(sps_stats)]),
    "sps_unit_tables": (_I, [_I, _P, _P, _P, _P]),
    "sps_profile": (_I, [_P, _I]),
    "sps_layer_apply_transpose": (_I, [_P, _I, _P, _P]),
    "sps_mobility_adjoint": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(sps_stats)]),
    "sps_collision_adjoint": (_I, [_P, _I, _P, _P, _P, ctypes.c_double, _P, _P, _P, _P,
                                   ctypes.POINTER(sps_stats)]),
    "sps_build_contacts_noalloc": (_I, [_I, _P, _P, _D, _D, _I, _P, _P, _P, ctypes.POINTER(_I), _P]),
    "sps_profile_read": (_I, [_P, _P, _P]),
    "sps_simulate": (_I, [_P, _I, _P, _P, _P, _D, _I, _P, ctypes.POINTER(sps_stats),
                          ctypes.POINTER(_I)]),
}

_lib = None


def load(path=LIB_PATH):
    """Loads libsps.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libsps.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class SPSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
