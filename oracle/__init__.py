"""ctypes wrapper of the CPU FP64 oracle (``oracle/bo_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain CPU reference that the CUDA
library is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path; both take their inputs from the ``synth`` generators.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bo_oracle.cpp")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FLUID_KEYS = ["g", "rho_s", "p_ref", "bw_ref", "c_w", "mu_w", "R_sb", "p_b", "Bo_slope", "c_o",
              "mu_o0", "mu_o_r", "c_mu", "p_sc", "Z", "mu_g0", "mu_g_p", "c_r", "s_wco",
              "s_orw", "s_org", "n_corey"]

# Newton / linear-solver options, in the order the oracle reads them.
DEFAULT_OPTS = {
    "tol_mb": 1e-6, "tol_cnv": 1e-6, "tol_well": 1e-6, "max_newton": 20,
    "tol_lin": 1e-3, "max_lin": 500, "max_cuts": 8,
    "ds_max": 0.2, "dp_rel_max": 0.3, "drs_rel_max": 0.2, "eps_switch": 1e-6,
    "bp_overshoot": 0.05, "dt_init": 864.0, "cut_factor": 0.5,
}
_OPT_ORDER = list(DEFAULT_OPTS.keys())


def build(force: bool = False) -> str:
    """Compile the oracle with g++ -O2 (OpenMP for the independent loops;
    one thread unless set_threads says otherwise)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_SO), exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-pthread", "-shared", "-fPIC",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        d = ctypes.c_double
        i = ctypes.c_int
        L.orc_create.restype = P
        L.orc_create.argtypes = [i, i, i, P, P, P, d, P, P, P, i, P, P, P]
        L.orc_destroy.argtypes = [P]
        L.orc_nnzb.argtypes = [P]
        L.orc_nnzb.restype = i
        L.orc_static.argtypes = [P] * 7
        L.orc_set_state.argtypes = [P] * 6
        L.orc_get_state.argtypes = [P] * 6
        L.orc_init_hydrostatic.argtypes = [P, d, d, d]
        L.orc_init_equilibrium.argtypes = [P, P]
        L.orc_begin_step.argtypes = [P]
        L.orc_assemble.argtypes = [P, d]
        L.orc_get_system.argtypes = [P] * 5
        L.orc_get_wells.argtypes = [P] * 6
        L.orc_well_rates.argtypes = [P] * 4
        L.orc_set_well_control.argtypes = [P, i, i, d]
        L.orc_norms.argtypes = [P, d, P]
        L.orc_residual_check.argtypes = [P, P, P]
        L.orc_ilu0.argtypes = [P, P, P]
        L.orc_ilu0.restype = i
        L.orc_ilu_apply.argtypes = [P, P, P]
        L.orc_apply_op.argtypes = [P, P, P]
        L.orc_solve.argtypes = [P, d, i, P, P]
        L.orc_solve.restype = i
        L.orc_dd_solve.argtypes = [P, d, i, P, P]
        L.orc_dd_solve.restype = i
        L.orc_newton_update.argtypes = [P, P, P]
        L.orc_step.argtypes = [P, d, P, P]
        L.orc_step.restype = i
        L.orc_cell_props.argtypes = [P, d, d, d, i, P]
        L.orc_get_dt_next.argtypes = [P]
        L.orc_get_dt_next.restype = d
        L.orc_set_dt_next.argtypes = [P, d]
        L.orc_set_subdomains.argtypes = [P, i, i]
        L.orc_set_threads.argtypes = [i]
        L.orc_set_threads.restype = i
        _lib = L
    return _lib


def perm3(perm, n):
    """Permeability as [3][n] (kx, ky, kz): an isotropic [n] array is repeated."""
    k = np.asarray(perm, dtype=np.float64)
    if k.size == n:
        k = np.concatenate([k.ravel()] * 3)
    if k.size != 3 * n:
        raise ValueError(f"perm must have n or 3n values, got {k.size}")
    return np.ascontiguousarray(k.reshape(-1))


def set_threads(threads: int) -> int:
    """Host threads of the oracle's independent loops (results do not depend
    on the count: every sum keeps its sequential order)."""
    return int(lib().orc_set_threads(int(threads)))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def fluid_array(fluid: dict) -> np.ndarray:
    out = []
    for k in FLUID_KEYS:
        v = fluid[k]
        out.extend(v if isinstance(v, (list, tuple)) else [v])
    return np.asarray(out, dtype=np.float64)


def opts_array(**overrides) -> np.ndarray:
    o = dict(DEFAULT_OPTS)
    o.update(overrides)
    return np.asarray([float(o[k]) for k in _OPT_ORDER], dtype=np.float64)


PROP_NAMES = ["b_w", "b_o", "b_g", "lam_w", "lam_o", "lam_g", "rho_w", "rho_o", "rho_g",
              "m_phi", "r_go", "A_w", "A_o", "A_g"]


def cell_props(fluid: dict, p, sw, x, flag) -> dict:
    """Value and (d/dp, d/dsw, d/dx) of the cell quantities at one state."""
    out = np.zeros(14 * 4)
    f = fluid_array(fluid)
    lib().orc_cell_props(_p(f), float(p), float(sw), float(x), int(flag), _p(out))
    out = out.reshape(14, 4)
    return {k: out[q] for q, k in enumerate(PROP_NAMES)}


class Oracle:
    """One black-oil model held by the oracle."""

    def __init__(self, model: dict):
        L = lib()
        self.model = model
        nx, ny, nz = model["nx"], model["ny"], model["nz"]
        self.n = nx * ny * nz
        self.nx, self.ny, self.nz = nx, ny, nz
        self._keep = []
        dx = np.ascontiguousarray(model["dx"], dtype=np.float64)
        dy = np.ascontiguousarray(model["dy"], dtype=np.float64)
        dz = np.ascontiguousarray(model["dz"], dtype=np.float64)
        perm = perm3(model["perm"], nx * ny * nz)
        poro = np.ascontiguousarray(model["poro"], dtype=np.float64)
        fl = fluid_array(model["fluid"])
        wint, wdbl, wcells = [], [], []
        for w in model["wells"]:
            kind = 0 if w["kind"] == "inj" else 1
            phase = 0 if w.get("phase", "gas") == "water" else 2
            ctl = 0 if w["control"] == "rate" else 1
            cells = [w["i"] + nx * (w["j"] + ny * k) for k in w["ks"]]
            wint += [kind, phase, ctl, len(cells)]
            wdbl += [w["target"], w["bhp_limit"], w["rw"], w["skin"]]
            wcells += cells
        self.nw = len(model["wells"])
        self.well_cells = []
        off = 0
        for q in range(self.nw):
            nc = wint[4 * q + 3]
            self.well_cells.append(wcells[off:off + nc])
            off += nc
        wint = np.asarray(wint if wint else [0], dtype=np.int32)
        wdbl = np.asarray(wdbl if wdbl else [0.0], dtype=np.float64)
        wcells_a = np.asarray(wcells if wcells else [0], dtype=np.int32)
        self.ncon = len(wcells)
        self.h = L.orc_create(nx, ny, nz, _p(dx), _p(dy), _p(dz), float(model["top_depth"]), _p(perm), _p(poro), _p(fl),
                              self.nw, _p(wint), _p(wdbl), _p(wcells_a))
        self.nnzb = L.orc_nnzb(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # -- static data --------------------------------------------------------
    def static(self):
        n = self.n
        Tx, Ty, Tz, pv, depth = (np.zeros(n) for _ in range(5))
        wi = np.zeros(max(self.ncon, 1))
        lib().orc_static(self.h, _p(Tx), _p(Ty), _p(Tz), _p(pv), _p(depth), _p(wi))
        return {"Tx": Tx, "Ty": Ty, "Tz": Tz, "pv": pv, "depth": depth, "wi": wi[:self.ncon]}

    # -- state --------------------------------------------------------------
    def set_state(self, p, sw, x, flag, bhp):
        p, sw, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (p, sw, x))
        flag = np.ascontiguousarray(flag, dtype=np.uint8)
        bhp = np.ascontiguousarray(bhp if len(bhp) else [0.0], dtype=np.float64)
        lib().orc_set_state(self.h, _p(p), _p(sw), _p(x), _p(flag), _p(bhp))

    def get_state(self):
        n = self.n
        p, sw, x = np.zeros(n), np.zeros(n), np.zeros(n)
        flag = np.zeros(n, dtype=np.uint8)
        bhp = np.zeros(max(self.nw, 1))
        lib().orc_get_state(self.h, _p(p), _p(sw), _p(x), _p(flag), _p(bhp))
        return p, sw, x, flag, bhp[:self.nw]

    def init_hydrostatic(self):
        ini = self.model["init"]
        lib().orc_init_hydrostatic(self.h, ini["p_top"], ini["sw"], ini["rgo"])

    def init_equilibrium(self, datum_depth, datum_pressure, woc, goc, rgo, swc):
        """Vertical equilibrium from a datum and the contacts (Section 2.1.3)."""
        e = np.array([datum_depth, datum_pressure, woc, goc, rgo, swc], dtype=np.float64)
        lib().orc_init_equilibrium(self.h, _p(e))

    # -- linearisation ------------------------------------------------------
    def begin_step(self):
        lib().orc_begin_step(self.h)

    def assemble(self, dt):
        lib().orc_assemble(self.h, float(dt))

    def system(self):
        """(rowptr, colind, vals[nnzb,3,3], R[n,3]) of the last assembly."""
        rp = np.zeros(self.n + 1, dtype=np.int32)
        ci = np.zeros(self.nnzb, dtype=np.int32)
        v = np.zeros(9 * self.nnzb)
        r = np.zeros(3 * self.n)
        lib().orc_get_system(self.h, _p(rp), _p(ci), _p(v), _p(r))
        return rp, ci, v.reshape(-1, 3, 3), r.reshape(-1, 3)

    def wells(self):
        """Per well: dict(Rw, Dw, B[ncon,3], C[ncon,3], control)."""
        rw = np.zeros(max(self.nw, 1))
        dw = np.zeros(max(self.nw, 1))
        B = np.zeros(max(3 * self.ncon, 1))
        C = np.zeros(max(3 * self.ncon, 1))
        ctl = np.zeros(max(self.nw, 1), dtype=np.int32)
        lib().orc_get_wells(self.h, _p(rw), _p(dw), _p(B), _p(C), _p(ctl))
        out, off = [], 0
        for q in range(self.nw):
            nc = len(self.well_cells[q])
            out.append({"Rw": rw[q], "Dw": dw[q], "B": B[3 * off:3 * (off + nc)].reshape(nc, 3),
                        "C": C[3 * off:3 * (off + nc)].reshape(nc, 3), "control": int(ctl[q])})
            off += nc
        return out

    def well_rates(self):
        """Per-well surface rates [nw, 3] (water, oil, gas; production
        positive) at the last assembly, current BHP [nw] and control [nw]."""
        nw = max(self.nw, 1)
        q, bhp = np.zeros(3 * nw), np.zeros(nw)
        ctl = np.zeros(nw, dtype=np.int32)
        lib().orc_well_rates(self.h, _p(q), _p(bhp), _p(ctl))
        return q.reshape(-1, 3)[:self.nw], bhp[:self.nw], ctl[:self.nw]

    def set_well_control(self, w, control, bhp):
        lib().orc_set_well_control(self.h, int(w), int(control), float(bhp))

    def norms(self, dt):
        out = np.zeros(7)
        lib().orc_norms(self.h, float(dt), _p(out))
        return out

    def residual_check(self, sol):
        sol = np.ascontiguousarray(sol, dtype=np.float64)
        out = np.zeros(3 * self.n + max(self.nw, 1))
        lib().orc_residual_check(self.h, _p(sol), _p(out))
        return out[:3 * self.n + self.nw]

    # -- linear solver ------------------------------------------------------
    def ilu0(self):
        lu = np.zeros(9 * self.nnzb)
        uinv = np.zeros(9 * self.n)
        st = lib().orc_ilu0(self.h, _p(lu), _p(uinv))
        if st != 0:
            raise RuntimeError("oracle ILU0: singular pivot block")
        return lu.reshape(-1, 3, 3), uinv.reshape(-1, 3, 3)

    def ilu_apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        z = np.zeros_like(r)
        lib().orc_ilu_apply(self.h, _p(r), _p(z))
        return z

    def apply_op(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        y = np.zeros_like(x)
        lib().orc_apply_op(self.h, _p(x), _p(y))
        return y

    def solve(self, tol=1e-3, maxit=500):
        """Returns (status, iterations, sol[3n + nw]); sol solves J sol = R."""
        sol = np.zeros(3 * self.n + max(self.nw, 1))
        its = np.zeros(1, dtype=np.int32)
        st = lib().orc_solve(self.h, float(tol), int(maxit), _p(sol), _p(its))
        return st, int(its[0]), sol[:3 * self.n + self.nw]

    def dd_solve(self, tol=1e-3, maxit=500):
        """solve() as K host-thread ranks, one per y slab of the block-Jacobi
        subdomains (set_subdomains(ysub), no z cuts): local rows, halo
        exchange, all-reduced inner products."""
        sol = np.zeros(3 * self.n + max(self.nw, 1))
        its = np.zeros(1, dtype=np.int32)
        st = lib().orc_dd_solve(self.h, float(tol), int(maxit), _p(sol), _p(its))
        return st, int(its[0]), sol[:3 * self.n + self.nw]

    def newton_update(self, sol, **opts):
        o = opts_array(**opts)
        s = np.ascontiguousarray(np.concatenate([sol, np.zeros(1)]), dtype=np.float64)
        lib().orc_newton_update(self.h, _p(o), _p(s))

    @property
    def dt_next(self):
        return lib().orc_get_dt_next(self.h)

    @dt_next.setter
    def dt_next(self, v):
        lib().orc_set_dt_next(self.h, float(v))

    def set_subdomains(self, ysub: int, zsub: int = 0):
        """Block-Jacobi ILU(0) over boxes of `ysub` cell rows in y and `zsub`
        cell layers in z (0: no cut in that direction)."""
        lib().orc_set_subdomains(self.h, int(ysub), int(zsub))

    def step(self, dt, **opts):
        o = opts_array(**opts)
        rep = np.zeros(5)
        st = lib().orc_step(self.h, float(dt), _p(o), _p(rep))
        return st, {"newton_its": int(rep[0]), "lin_its": int(rep[1]), "cuts": int(rep[2]),
                    "substeps": int(rep[3]), "status": int(rep[4])}
