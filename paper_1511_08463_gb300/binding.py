"""ctypes binding of libpf (include/pf.h).  Argument marshalling only: every step of the
solver runs in the CUDA library.  PyTorch supplies device memory (the workspace and operand
buffers) and streams.  Importing this module loads the library and fails loudly if it is
missing; there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

from . import _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ENOTCONV, PF_ENUMERIC, PF_ETIMEOUT, PF_ECUDA, PF_EBUSY = range(8)
PF_MESH_RIGHT, PF_MESH_CROSSED = 0, 1
PF_AT1, PF_AT2 = 1, 2
PF_PLANE_STRAIN, PF_PLANE_STRESS = 0, 1
PF_FP64, PF_MIXED = 0, 1
PF_ALGO_AM, PF_ALGO_ORAM, PF_ALGO_ORAM_N = 0, 1, 2
PF_MAX_PINS, PF_MAX_BOXES = 8, 8
STATUS_NAMES = ["PF_OK", "PF_EINVAL", "PF_ENOMEM", "PF_ENOTCONV", "PF_ENUMERIC", "PF_ETIMEOUT",
                "PF_ECUDA", "PF_EBUSY"]


class pf_mesh_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("x0", C.c_double), ("y0", C.c_double), ("lx", C.c_double), ("ly", C.c_double),
                ("fixed", (C.c_uint8 * 3) * 4), ("load", (C.c_double * 3) * 4),
                ("n_pins", C.c_int32), ("pin_x2", C.c_int32 * PF_MAX_PINS),
                ("pin_y2", C.c_int32 * PF_MAX_PINS), ("pin_comp", C.c_int32 * PF_MAX_PINS),
                ("pin_load", C.c_double * PF_MAX_PINS), ("n_boxes", C.c_int32),
                ("box", (C.c_int32 * 4) * PF_MAX_BOXES), ("box_value", C.c_double * PF_MAX_BOXES),
                ("mode_I", C.c_int32), ("mode_I_param", C.c_double * 4)]


class pf_material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("Gc", C.c_double), ("ell", C.c_double),
                ("k_ell", C.c_double), ("model", C.c_int32), ("plane", C.c_int32),
                ("beta", C.c_double), ("pen", C.c_double)]


class pf_load(C.Structure):
    _fields_ = [("t", C.c_double), ("dT", C.c_double)]


class pf_solver_opts(C.Structure):
    _fields_ = [("algo", C.c_int32), ("precision", C.c_int32), ("omega", C.c_double),
                ("am_tol", C.c_double), ("am_maxit", C.c_int32), ("u_rtol", C.c_double),
                ("inner_rtol", C.c_double), ("cg_maxit", C.c_int32), ("rs_rtol", C.c_double),
                ("rs_maxit", C.c_int32), ("alpha_cg_rtol", C.c_double), ("zeta", C.c_double),
                ("mg_levels_max", C.c_int32), ("mg_degree", C.c_int32),
                ("switch_tol", C.c_double), ("newton_rtol", C.c_double),
                ("newton_maxit", C.c_int32), ("minres_maxit", C.c_int32),
                ("minres_rtol", C.c_double), ("use_graphs", C.c_int32),
                ("batch_workers", C.c_int32), ("am_forcing", C.c_double),
                ("am_forcing_max", C.c_double), ("mg_tail", C.c_int32),
                ("mg_coarse_degree", C.c_int32), ("omega_rule", C.c_int32),
                ("omega_auto", C.c_int32), ("omega_max", C.c_double),
                ("autotune", C.c_int32), ("tile_rows_fine", C.c_int32),
                ("tile_rows_coarse", C.c_int32)]


class pf_step_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("am_iters", C.c_int32), ("rs_iters", C.c_int32),
                ("newton_iters", C.c_int32), ("cg_iters_u", C.c_int64),
                ("cg_iters_alpha", C.c_int64), ("krylov_iters_newton", C.c_int64),
                ("outer_refinements", C.c_int64), ("dalpha_inf", C.c_double),
                ("du_rel", C.c_double), ("phi_norm", C.c_double), ("phi_start", C.c_double),
                ("omega_bar_min", C.c_double), ("energy", C.c_double * 3),
                ("seconds", C.c_double), ("u_solves_reused", C.c_int64),
                ("u_notconv", C.c_int64), ("newton_steepest", C.c_int64),
                ("alpha_notconv", C.c_int64), ("omega_final", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["energy"] = list(self.energy)
        return d


class pf_tune_report(C.Structure):
    _fields_ = [("mg_degree", C.c_int32), ("mg_coarse_degree", C.c_int32),
                ("tile_rows_fine", C.c_int32), ("tile_rows_coarse", C.c_int32),
                ("trials", C.c_int32), ("iters_best", C.c_int32), ("iters_default", C.c_int32),
                ("ms_best", C.c_double), ("ms_default", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_job(C.Structure):
    _fields_ = [("mesh", pf_mesh_desc), ("material", pf_material),
                ("loads", C.POINTER(pf_load)), ("n_loads", C.c_int32),
                ("opts", pf_solver_opts), ("arrival", C.c_double),
                ("u_out", C.POINTER(C.c_double)), ("alpha_out", C.POINTER(C.c_double)),
                ("reports", C.POINTER(pf_step_report)), ("step_latency", C.POINTER(C.c_double))]


class pf_job_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps_done", C.c_int32), ("arrival", C.c_double),
                ("admitted", C.c_double), ("finished", C.c_double), ("footprint", C.c_size_t)]


class pf_server_stats(C.Structure):
    _fields_ = [("jobs_done", C.c_int64), ("steps_done", C.c_int64),
                ("arena_bytes", C.c_size_t), ("arena_peak", C.c_size_t),
                ("max_active", C.c_int32), ("workers", C.c_int32)]


_VP = C.c_void_p
_SIGS = {
    "pf_last_error": (C.c_char_p, []),
    "pf_version": (C.c_char_p, []),
    "pf_default_opts": (C.c_int, [C.POINTER(pf_solver_opts)]),
    "pf_ctx_create": (C.c_int, [C.c_int, C.POINTER(_VP)]),
    "pf_ctx_destroy": (None, [_VP]),
    "pf_workspace_bytes": (C.c_size_t, [C.POINTER(pf_mesh_desc), C.c_int]),
    "pf_create_mesh": (C.c_int, [_VP, C.POINTER(pf_mesh_desc), _VP, C.c_size_t, C.POINTER(_VP)]),
    "pf_set_material": (C.c_int, [_VP, C.POINTER(pf_material)]),
    "pf_load_step": (C.c_int, [_VP, C.POINTER(pf_load), C.POINTER(pf_solver_opts), _VP,
                               C.POINTER(pf_step_report)]),
    "pf_energy": (C.c_int, [_VP, _VP, C.POINTER(C.c_double)]),
    "pf_solve_batch": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(pf_load), C.c_int,
                                 C.POINTER(pf_solver_opts), _VP, C.POINTER(pf_step_report)]),
    "pf_get_fields": (C.c_int, [_VP, _VP, _VP, _VP]),
    "pf_set_fields": (C.c_int, [_VP, _VP, _VP, _VP]),
    "pf_sim_info": (C.c_int, [_VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int32)]),
    "pf_destroy": (None, [_VP]),
    "pf_set_load": (C.c_int, [_VP, C.POINTER(pf_load)]),
    "pf_op_elastic_apply": (C.c_int, [_VP, C.c_int, C.c_int, _VP, _VP, _VP]),
    "pf_op_elastic_residual": (C.c_int, [_VP, C.c_int, _VP, C.POINTER(C.c_double), _VP]),
    "pf_op_damage_gradient": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, C.POINTER(C.c_double), _VP]),
    "pf_op_damage_apply": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP]),
    "pf_op_coupling_apply": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP]),
    "pf_op_u_solve": (C.c_int, [_VP, C.POINTER(pf_solver_opts), _VP, C.POINTER(pf_step_report)]),
    "pf_op_alpha_solve": (C.c_int, [_VP, C.POINTER(pf_solver_opts), _VP,
                                    C.POINTER(pf_step_report)]),
    "pf_op_full_residual": (C.c_int, [_VP, C.POINTER(C.c_double), _VP]),
    "pf_autotune": (C.c_int, [_VP, C.POINTER(pf_solver_opts), _VP, C.POINTER(pf_tune_report)]),
    "pf_energy_noalloc": (C.c_int, [C.POINTER(pf_mesh_desc), C.POINTER(pf_material),
                                    C.POINTER(pf_load), _VP, _VP, C.POINTER(C.c_double), _VP]),
    "pf_server_create": (C.c_int, [_VP, _VP, C.c_size_t, C.c_int, C.POINTER(_VP)]),
    "pf_server_now": (C.c_double, [_VP]),
    "pf_server_submit": (C.c_int, [_VP, C.POINTER(pf_job), C.POINTER(C.c_int64)]),
    "pf_server_wait": (C.c_int, [_VP, C.c_int64, C.POINTER(pf_job_info)]),
    "pf_server_drain": (C.c_int, [_VP]),
    "pf_server_get_stats": (C.c_int, [_VP, C.POINTER(pf_server_stats)]),
    "pf_server_destroy": (None, [_VP]),
    "pf_prof_enable": (C.c_int, [C.c_int, C.c_int]),
    "pf_prof_reset": (C.c_int, []),
    "pf_launch_count": (C.c_int64, []),
    "pf_prof_class_count": (C.c_int, []),
    "pf_prof_get": (C.c_int, [C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64), C.POINTER(C.c_double),
                              C.POINTER(C.c_double)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libpf.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise OSError(f"libpf.so not found at {p}; run __graft_entry__.build()")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class PFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def check(status: int, allow=(PF_OK,)):
    if status not in allow:
        raise PFError(status, load().pf_last_error().decode())
    return status


def prof_table():
    """Per kernel class: name -> dict(launches, timed, ms, bytes)."""
    lib = load()
    out = {}
    for k in range(lib.pf_prof_class_count()):
        nm, la, ti, ms, by = C.c_char_p(), C.c_int64(), C.c_int64(), C.c_double(), C.c_double()
        check(lib.pf_prof_get(k, C.byref(nm), C.byref(la), C.byref(ti), C.byref(ms), C.byref(by)))
        if la.value or ti.value:
            out[nm.value.decode()] = dict(id=k, launches=la.value, timed=ti.value, ms=ms.value,
                                          bytes=by.value)
    return out
