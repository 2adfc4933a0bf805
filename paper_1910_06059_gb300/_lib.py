"""ctypes binding of libbo.so (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python and
NumPy arguments to the C ABI of ``include/bo.h`` and raises on error.  There
is no CPU fallback: when the library is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbo.so")

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
P = c_void_p


class BoFluid(ctypes.Structure):
    _fields_ = [("g", c_double), ("rho_s", c_double * 3), ("p_ref", c_double),
                ("bw_ref", c_double), ("c_w", c_double), ("mu_w", c_double), ("R_sb", c_double),
                ("p_b", c_double), ("Bo_slope", c_double), ("c_o", c_double),
                ("mu_o0", c_double), ("mu_o_r", c_double), ("c_mu", c_double),
                ("p_sc", c_double), ("Z", c_double), ("mu_g0", c_double), ("mu_g_p", c_double),
                ("c_r", c_double), ("s_wco", c_double), ("s_orw", c_double), ("s_org", c_double),
                ("n_corey", c_double)]


class BoWell(ctypes.Structure):
    _fields_ = [("kind", c_int), ("phase", c_int), ("control", c_int), ("ncon", c_int),
                ("cells", ctypes.POINTER(c_int)), ("target", c_double),
                ("bhp_limit", c_double), ("rw", c_double), ("skin", c_double)]


class BoNewtonOpts(ctypes.Structure):
    _fields_ = [("tol_mb", c_double), ("tol_cnv", c_double), ("tol_well", c_double),
                ("max_newton", c_int), ("tol_lin", c_double), ("max_lin", c_int),
                ("max_cuts", c_int), ("ds_max", c_double), ("dp_rel_max", c_double),
                ("drs_rel_max", c_double), ("eps_switch", c_double),
                ("bp_overshoot", c_double), ("dt_init", c_double), ("cut_factor", c_double)]


class BoSolveOpts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("max_it", c_int)]


class BoSolveReport(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("status", c_int), ("restarts", c_int),
                ("rel_res", c_double), ("fallback", c_int)]


PRECISION = {"fp64": 0, "mixed": 1}

LEARN_NPARAM = 25865


class BoLearnOpts(ctypes.Structure):
    _fields_ = [("samples", c_int), ("epochs", c_int), ("lr", c_double)]


class BoLearnReport(ctypes.Structure):
    _fields_ = [("systems", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("fallbacks", ctypes.c_longlong), ("first_loss", c_double),
                ("last_loss", c_double), ("train_ms", c_double),
                ("guard_stage_its", ctypes.c_longlong), ("guard_plain_its", ctypes.c_longlong),
                ("guard_state", c_int)]


class BoStepReport(ctypes.Structure):
    _fields_ = [("newton_its", c_int), ("lin_its", c_int), ("cuts", c_int),
                ("substeps", c_int), ("status", c_int), ("mb", c_double * 3),
                ("cnv", c_double * 3), ("well_res", c_double), ("ms_assemble", c_double),
                ("ms_factor", c_double), ("ms_solve", c_double), ("ms_update", c_double)]


# name -> argtypes (restype is always bo_status = int)
_SIGS = {
    "bo_create_grid": [c_int, c_int, c_int, P, P, P, c_double, P],
    "bo_set_properties": [P, P, P, P, P, c_int],
    "bo_get_static": [P, P, P, P, P, P, P],
    "bo_init_hydrostatic": [P, c_double, c_double, c_double],
    "bo_set_state": [P, P, P, P, P, P],
    "bo_get_state": [P, P, P, P, P, P],
    "bo_set_state_dev": [P, P, P, P, P, P],
    "bo_get_state_dev": [P, P, P, P, P, P],
    "bo_set_stream": [P, P],
    "bo_begin_step": [P],
    "bo_assemble": [P, c_double],
    "bo_norms": [P, c_double, P],
    "bo_get_system": [P, P, P, P, P, P],
    "bo_get_wells": [P, P, P, P, P, P],
    "bo_get_well_rates": [P, P, P, P],
    "bo_factor": [P, P],
    "bo_precond_apply": [P, P, P],
    "bo_apply_op": [P, P, P],
    "bo_solve": [P, P, P, P],
    "bo_newton_update": [P, P],
    "bo_step": [P, c_double, P, P],
    "bo_get_step_control": [P, P],
    "bo_set_step_control": [P, c_double],
    "bo_set_timing": [P, c_int],
    "bo_set_precision": [P, c_int],
    "bo_set_subdomains": [P, c_int, c_int],
    "bo_init_equilibrium": [P, P],
    "bo_get_subdomains": [P, P, P],
    "bo_ensemble_create": [P, c_int, c_int, P],
    "bo_ensemble_set_schedule": [P, c_int, c_int],
    "bo_ensemble_get_schedule": [P, P, P],
    "bo_ensemble_step": [P, c_double, P, P, P],
    "bo_ensemble_autotune": [P, c_double, P, P, c_int, P],
    "bo_ensemble_last_step_ms": [P, P],
    "bo_ensemble_autotune_precond": [P, c_double, P, P, P, P],
    "bo_ensemble_autotune_schedule": [P, c_double, P, P, P, P],
    "bo_ensemble_destroy": [P],
    "bo_learn_set_params": [P, P, c_int],
    "bo_learn_get_params": [P, P, c_int],
    "bo_learn_enable": [P, c_int],
    "bo_learn_online": [P, P],
    "bo_learn_get_report": [P, P],
    "bo_learn_delta": [P, P, P],
    "bo_learn_loss_grad": [P, P, P, P],
    "bo_get_precision": [P, P],
    "bo_get_timing": [P, c_int, P, P, P, P],
    "bo_get_launch_count": [P, P],
    "bo_set_well_model": [P, c_int, c_int],
    "bo_dd_solve": [P, P, P, P],
    "bo_set_sweep_ctas_per_sm": [P, c_int],
    "bo_learn_set_engine": [P, c_int],
    "bo_learn_collect": [P, c_int, c_int],
    "bo_learn_set_info": [P, P, P],
    "bo_learn_train_offline": [P, c_int, c_double, P, P],
    "bo_learn_get_engine": [P, P],
    "bo_get_well_model": [P, P],
    "bo_get_std_wells": [P, P, P, P, P, P],
    "bo_set_preconditioner": [P, c_int],
    "bo_learn_guard": [P, c_int],
    "bo_get_preconditioner": [P, P],
    "bo_set_solve_schedule": [P, c_int],
    "bo_get_solve_schedule": [P, P],
    "bo_cpr_hierarchy": [P, c_int, P, P, P],
    "bo_cpr_pressure_system": [P, P, P],
    "bo_cpr_vcycle": [P, P, P],
    "bo_selftest_bounded_wait": [P, P],
    "bo_residual_norms_noalloc": [P, P, P, c_int, c_double, P, P],
    "bo_sizes": [P, P, P, P, P],
    "bo_destroy": [P],
}
EXPORTED = sorted(list(_SIGS) + ["bo_last_error"])

PRECONDITIONER = {"ilu0": 0, "cpr": 1}
SCHEDULE = {"tiled": 0, "block": 1}
WELL_MODEL = {"reduced": 0, "standard": 1}

STATUS = {0: "BO_OK", 1: "BO_ERR_INVALID_ARG", 2: "BO_ERR_CUDA", 3: "BO_ERR_OOM",
          4: "BO_ERR_NOT_CONVERGED", 5: "BO_ERR_LINEAR_BREAKDOWN", 6: "BO_ERR_DEVICE_TIMEOUT",
          7: "BO_ERR_STATE"}

_lib = None


class BoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libbo.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbo.so not built at {path}; run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = c_int
    L.bo_last_error.argtypes = []
    L.bo_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def call(name, *args):
    L = load()
    st = getattr(L, name)(*args)
    if st != 0:
        raise BoError(st, L.bo_last_error().decode())
    return st


def ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(c_void_p)
    if hasattr(a, "data_ptr"):  # torch tensor (device or host)
        return c_void_p(a.data_ptr())
    raise TypeError(type(a))


FLUID_KEYS = [f for f, _ in BoFluid._fields_]


def fluid_struct(fluid: dict) -> BoFluid:
    f = BoFluid()
    for k in FLUID_KEYS:
        v = fluid[k]
        if k == "rho_s":
            for q in range(3):
                f.rho_s[q] = v[q]
        else:
            setattr(f, k, float(v))
    return f


DEFAULT_NEWTON = dict(tol_mb=1e-6, tol_cnv=1e-6, tol_well=1e-6, max_newton=20, tol_lin=1e-3,
                      max_lin=500, max_cuts=8, ds_max=0.2, dp_rel_max=0.3, drs_rel_max=0.2,
                      eps_switch=1e-6, bp_overshoot=0.05, dt_init=864.0, cut_factor=0.5)


def newton_opts(**kw) -> BoNewtonOpts:
    o = dict(DEFAULT_NEWTON)
    o.update(kw)
    return BoNewtonOpts(**o)
