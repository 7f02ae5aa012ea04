"""ctypes declarations mirroring include/pb.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpbgpu.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOCONV, ERR_TIMEOUT, ERR_STATE, ERR_UNIMPL = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "PB_OK", -1: "PB_ERR_ARG", -2: "PB_ERR_OOM", -3: "PB_ERR_CUDA",
                -4: "PB_ERR_NOCONV", -5: "PB_ERR_TIMEOUT", -6: "PB_ERR_STATE", -7: "PB_ERR_UNIMPL"}
BC_ZERO, BC_COULOMB, BC_DH = 0, 1, 2
FP64, MIXED = 0, 1
HOST, DEVICE = 0, 1
CT_BOUNDARY, CT_SURFACE, CT_PAIRS, CT_ALL = 1, 2, 4, 7
(ARR_INSIDE, ARR_CROSS_ID, ARR_CROSS_ALPHA, ARR_CROSS_RP, ARR_CROSS_SIGN, ARR_WX, ARR_WY, ARR_WZ,
 ARR_KAPPA, ARR_DIAG, ARR_RHS, ARR_BC, ARR_PHI, ARR_PHI_SURF, ARR_PSI_SURF, ARR_OCT_BRICKS,
 ARR_OCT_KIND, ARR_MC_WEIGHT, ARR_MC_NORMAL, ARR_PSI_N) = range(20)
GRID_UNIFORM, GRID_OCTREE = 0, 1


class PBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class GridSpecC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("h", C.c_double), ("fill", C.c_double), ("h_fine", C.c_double),
                ("h_bulk", C.c_double), ("refine_dist", C.c_double),
                ("h_tight", C.c_double), ("tight_fill", C.c_double)]


class ParamsC(C.Structure):
    _fields_ = [("eps_in", C.c_double), ("eps_out", C.c_double), ("ionic_strength_M", C.c_double),
                ("temperature_K", C.c_double), ("bc", C.c_int32)]


class SolveOptsC(C.Structure):
    _fields_ = [("precision", C.c_int32), ("rtol", C.c_double), ("max_iter", C.c_int32),
                ("max_outer", C.c_int32), ("inner_rtol", C.c_double), ("time_budget_s", C.c_double)]


class SolveStatsC(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters_inner", C.c_int32), ("iters_outer", C.c_int32),
                ("kc", C.c_int32), ("true_rel_res", C.c_double), ("seconds", C.c_double), ("dof", C.c_int64),
                ("model_bytes", C.c_int64)]


class EnergyC(C.Structure):
    _fields_ = [("e_coul", C.c_double), ("e_pol", C.c_double), ("e_ion_surf", C.c_double),
                ("e_ion_flux", C.c_double), ("e_total", C.c_double), ("flux_charge", C.c_double),
                ("e_ion_mc", C.c_double)]


class GridInfoC(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("origin", C.c_double * 3), ("h", C.c_double),
                ("n_nodes", C.c_int64), ("n_atoms", C.c_int64), ("n_cross", C.c_int64),
                ("n_flux", C.c_int64), ("n_inside", C.c_int64), ("kind", C.c_int32),
                ("n_levels", C.c_int32), ("n_bricks", C.c_int64)]


class EngineResultC(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("system", C.c_void_p), ("stats", SolveStatsC),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# every function of include/pb.h with its ctypes signature
P = C.c_void_p
SIGNATURES = {
    "pb_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, P]),
    "pb_build_grid": (C.c_int, [P, P, C.c_int64, C.c_int32, P, P]),
    "pb_grid_info_get": (C.c_int, [P, P]),
    "pb_grid_free": (None, [P]),
    "pb_assemble_coeffs": (C.c_int, [P, P, P, P]),
    "pb_system_free": (None, [P]),
    "pb_coulomb_terms": (C.c_int, [P, C.c_int32, P]),
    "pb_solve": (C.c_int, [P, P, P, P, P]),
    "pb_energy": (C.c_int, [P, P, P]),
    "pb_get_phi": (C.c_int, [P, P, C.c_int32, P]),
    "pb_get_array": (C.c_int, [P, P, C.c_int32, P, C.c_size_t, C.c_int32, P]),
    "pb_apply": (C.c_int, [P, C.c_int32, P, P, P]),
    "pb_solve_batch": (C.c_int, [P, C.c_int32, P, P, P]),
    "pb_profile_kernels": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, P]),
    "pb_kernel_launches": (C.c_int64, []),
    "pb_set_tuning": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32]),
    "pb_set_wait_limit": (C.c_int, [C.c_int64]),
    "pb_solve_split": (C.c_int, [P, C.c_int32, P, P, P]),
    "pb_apply_dot_noalloc": (C.c_int, [P, P, P, P, P]),
    "pb_engine_create": (C.c_int, [C.c_int32, C.c_int32, P, P]),
    "pb_engine_submit": (C.c_int, [P, P, P, P]),
    "pb_engine_wait": (C.c_int, [P, C.c_double, P, C.c_int32, P]),
    "pb_engine_query": (C.c_int, [P, P, P, P]),
    "pb_engine_destroy": (C.c_int, [P]),
    "pb_last_error": (C.c_char_p, []),
    "pb_version": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None
_keep: list = []


def lib():
    """Load libpbgpu.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"libpbgpu.so not found at {LIB_PATH}; build it with "
                    "`python -m paper_2502_09323_gb300.build` (needs nvcc)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def keep_alive(*objs):
    _keep[:] = list(objs)


def kept():
    return tuple(_keep)


def check(rc: int) -> None:
    if rc != OK:
        raise PBError(rc, lib().pb_last_error().decode())


def grid_info(handle) -> GridInfoC:
    info = GridInfoC()
    check(lib().pb_grid_info_get(handle, C.byref(info)))
    return info


def struct_dict(s) -> dict:
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        out[name] = list(v) if isinstance(v, C.Array) else v
    return out
