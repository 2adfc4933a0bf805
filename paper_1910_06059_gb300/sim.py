"""Python view of one simulation object of libbo.so (marshalling only).

The method names follow the C ABI of ``include/bo.h`` without the ``bo_``
prefix.  Host arrays are NumPy; the ``*_dev`` forms take torch CUDA tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from ._lib import call, ptr


class Sim:
    """One black-oil model on the current CUDA device."""

    def __init__(self, model: dict, stream=None):
        self.model = model
        nx, ny, nz = model["nx"], model["ny"], model["nz"]
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        dx = np.ascontiguousarray(model["dx"], dtype=np.float64)
        dy = np.ascontiguousarray(model["dy"], dtype=np.float64)
        dz = np.ascontiguousarray(model["dz"], dtype=np.float64)
        h = ctypes.c_void_p()
        call("bo_create_grid", nx, ny, nz, ptr(dx), ptr(dy), ptr(dz), float(model["top_depth"]),
             ctypes.byref(h))
        self.h = h
        if stream is not None:
            self.set_stream(stream)
        self._set_properties()

    # -- setup ---------------------------------------------------------------
    def _set_properties(self):
        m = self.model
        perm = np.asarray(m["perm"], dtype=np.float64).ravel()
        if perm.size == self.n:            # isotropic: kx = ky = kz
            perm = np.concatenate([perm] * 3)
        if perm.size != 3 * self.n:
            raise ValueError(f"perm must have n or 3n values, got {perm.size}")
        perm = np.ascontiguousarray(perm)
        poro = np.ascontiguousarray(m["poro"], dtype=np.float64)
        fl = L.fluid_struct(m["fluid"])
        wells = (L.BoWell * max(1, len(m["wells"])))()
        self._cells = []
        self.well_cells = []
        for q, w in enumerate(m["wells"]):
            cells = np.asarray([w["i"] + self.nx * (w["j"] + self.ny * k) for k in w["ks"]],
                               dtype=np.int32)
            self._cells.append(cells)
            self.well_cells.append([int(c) for c in cells])
            wells[q].kind = 0 if w["kind"] == "inj" else 1
            wells[q].phase = 0 if w.get("phase", "gas") == "water" else 2
            wells[q].control = 0 if w["control"] == "rate" else 1
            wells[q].ncon = len(cells)
            wells[q].cells = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            wells[q].target = w["target"]
            wells[q].bhp_limit = w["bhp_limit"]
            wells[q].rw = w["rw"]
            wells[q].skin = w["skin"]
        self.nw = len(m["wells"])
        self.ncon = sum(len(c) for c in self._cells)
        call("bo_set_properties", self.h, ptr(perm), ptr(poro), ctypes.byref(fl),
             ctypes.cast(wells, ctypes.c_void_p), self.nw)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (legacy default)."""
        handle = getattr(stream, "cuda_stream", stream)
        call("bo_set_stream", self.h, ctypes.c_void_p(handle or 0))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            call("bo_destroy", self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- static data and state ----------------------------------------------
    def get_static(self):
        n = self.n
        Tx, Ty, Tz, pv, depth = (np.zeros(n) for _ in range(5))
        wi = np.zeros(max(self.ncon, 1))
        call("bo_get_static", self.h, ptr(Tx), ptr(Ty), ptr(Tz), ptr(pv), ptr(depth), ptr(wi))
        return {"Tx": Tx, "Ty": Ty, "Tz": Tz, "pv": pv, "depth": depth, "wi": wi[:self.ncon]}

    def init_hydrostatic(self):
        ini = self.model["init"]
        call("bo_init_hydrostatic", self.h, float(ini["p_top"]), float(ini["sw"]), float(ini["rgo"]))

    def init_equilibrium(self, datum_depth, datum_pressure, woc, goc, rgo, swc):
        """Vertical equilibrium from a datum and the contacts (bo_init_equilibrium)."""
        e = (ctypes.c_double * 6)(datum_depth, datum_pressure, woc, goc, rgo, swc)
        call("bo_init_equilibrium", self.h, e)

    def set_state(self, p, sw, x, flag, bhp):
        p, sw, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (p, sw, x))
        flag = np.ascontiguousarray(flag, dtype=np.uint8)
        bhp = np.ascontiguousarray(bhp if len(bhp) else [0.0], dtype=np.float64)
        call("bo_set_state", self.h, ptr(p), ptr(sw), ptr(x), ptr(flag), ptr(bhp))

    def get_state(self, out=None):
        """(p, sw, x, flag, bhp) as host arrays; out: five preallocated
        contiguous arrays (float64 [n] x 3, uint8 [n], float64 [max(nw, 1)])
        to read into instead of new ones (e.g. pinned host buffers)."""
        n = self.n
        if out is None:
            p, sw, x = np.zeros(n), np.zeros(n), np.zeros(n)
            flag = np.zeros(n, dtype=np.uint8)
            bhp = np.zeros(max(self.nw, 1))
        else:
            p, sw, x, flag, bhp = out
            for a, dt in zip(out, (np.float64,) * 3 + (np.uint8, np.float64)):
                if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("get_state(out=...): wrong dtype or non-contiguous array")
            if min(p.size, sw.size, x.size, flag.size) < n or bhp.size < max(self.nw, 1):
                raise ValueError("get_state(out=...): arrays too small")
        call("bo_get_state", self.h, ptr(p), ptr(sw), ptr(x), ptr(flag), ptr(bhp))
        return p, sw, x, flag, bhp[:self.nw]

    def set_state_dev(self, p, sw, x, flag, bhp):
        call("bo_set_state_dev", self.h, ptr(p), ptr(sw), ptr(x), ptr(flag), ptr(bhp))

    def get_state_dev(self, p, sw, x, flag, bhp):
        call("bo_get_state_dev", self.h, ptr(p), ptr(sw), ptr(x), ptr(flag), ptr(bhp))

    # -- linearisation -------------------------------------------------------
    def begin_step(self):
        call("bo_begin_step", self.h)

    def assemble(self, dt):
        call("bo_assemble", self.h, float(dt))

    def norms(self, dt):
        out = np.zeros(7)
        call("bo_norms", self.h, float(dt), ptr(out))
        return out

    def system(self):
        """(rowptr, colind, vals[nnzb,3,3], R[n,3]) of the last assembly."""
        nnzb = ctypes.c_int()
        call("bo_get_system", self.h, None, None, None, None, ctypes.byref(nnzb))
        rp = np.zeros(self.n + 1, dtype=np.int32)
        ci = np.zeros(nnzb.value, dtype=np.int32)
        v = np.zeros(9 * nnzb.value)
        r = np.zeros(3 * self.n)
        call("bo_get_system", self.h, ptr(rp), ptr(ci), ptr(v), ptr(r), None)
        return rp, ci, v.reshape(-1, 3, 3), r.reshape(-1, 3)

    def wells(self):
        nw = max(self.nw, 1)
        rw, dw = np.zeros(nw), np.zeros(nw)
        B = np.zeros(max(3 * self.ncon, 1))
        C = np.zeros(max(3 * self.ncon, 1))
        ctl = np.zeros(nw, dtype=np.int32)
        call("bo_get_wells", self.h, ptr(rw), ptr(dw), ptr(B), ptr(C), ptr(ctl))
        out, off = [], 0
        for q in range(self.nw):
            nc = len(self.well_cells[q])
            out.append({"Rw": rw[q], "Dw": dw[q], "B": B[3 * off:3 * (off + nc)].reshape(nc, 3),
                        "C": C[3 * off:3 * (off + nc)].reshape(nc, 3), "control": int(ctl[q])})
            off += nc
        return out

    # -- well model ----------------------------------------------------------
    @property
    def well_model(self):
        """"reduced" (one unknown per rate well) or "standard" (four unknowns
        per well, cross-flow, wellbore storage)."""
        v = ctypes.c_int()
        call("bo_get_well_model", self.h, ctypes.byref(v))
        return {q: k for k, q in L.WELL_MODEL.items()}[v.value]

    def set_sweep_ctas_per_sm(self, k):
        """Persistent CTAs of the FP64 sweeps per SM (1 or 2)."""
        call("bo_set_sweep_ctas_per_sm", self.h, int(k))

    def set_well_model(self, name, storage=True):
        """Select the well model; the well unknowns start at the next
        set_state / init_hydrostatic / init_equilibrium."""
        call("bo_set_well_model", self.h, L.WELL_MODEL[name], 1 if storage else 0)

    def std_wells(self, blocks=True):
        """Full standard wells: per well dict(B [ncon,4,3], C [ncon,3,4],
        D [4,4], Rw [4]) of the last assembly (blocks=True) and the current
        unknowns xw [4] = (Q_t, F_w, F_g, p_bhp)."""
        nw, nc = max(self.nw, 1), max(self.ncon, 1)
        B, C = np.zeros(12 * nc), np.zeros(12 * nc)
        D, Rw, xw = np.zeros(16 * nw), np.zeros(4 * nw), np.zeros(4 * nw)
        if blocks:
            call("bo_get_std_wells", self.h, ptr(B), ptr(C), ptr(D), ptr(Rw), ptr(xw))
        else:
            call("bo_get_std_wells", self.h, None, None, None, None, ptr(xw))
        out, off = [], 0
        for q in range(self.nw):
            k = len(self.well_cells[q])
            d = {"xw": xw[4 * q:4 * q + 4].copy()}
            if blocks:
                d.update(B=B[12 * off:12 * (off + k)].reshape(k, 4, 3),
                         C=C[12 * off:12 * (off + k)].reshape(k, 3, 4),
                         D=D[16 * q:16 * q + 16].reshape(4, 4), Rw=Rw[4 * q:4 * q + 4].copy())
            out.append(d)
            off += k
        return out

    def well_rates(self):
        """Per-well surface rates [nw, 3] (water, oil, gas; m^3/s, production
        positive) at the last assembly, with the current BHP [nw] and control
        [nw] (0 rate, 1 BHP)."""
        nw = max(self.nw, 1)
        q, bhp = np.zeros(3 * nw), np.zeros(nw)
        ctl = np.zeros(nw, dtype=np.int32)
        call("bo_get_well_rates", self.h, ptr(q), ptr(bhp), ptr(ctl))
        return q.reshape(-1, 3)[:self.nw], bhp[:self.nw], ctl[:self.nw]

    # -- linear solver -------------------------------------------------------
    def factor(self):
        dinv = np.zeros(9 * self.n)
        call("bo_factor", self.h, ptr(dinv))
        return dinv.reshape(-1, 3, 3)

    def precond_apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        z = np.zeros_like(r)
        call("bo_precond_apply", self.h, ptr(r), ptr(z))
        return z

    def apply_op(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        y = np.zeros_like(x)
        call("bo_apply_op", self.h, ptr(x), ptr(y))
        return y

    def solve(self, tol=1e-3, maxit=500, report=False):
        """Returns (status, iterations, sol[3n + nw]); sol solves J sol = R.
        With report=True a fourth item gives the restarts, the true
        relative residual ||b - Op x|| / ||b|| and the fallback mask (1: repeated
        without the learned stage, 2: repeated with the FP64 sweeps)."""
        o = L.BoSolveOpts(tol=float(tol), max_it=int(maxit))
        rep = L.BoSolveReport()
        nwv = 4 * self.nw if self.well_model == "standard" else self.nw
        sol = np.zeros(3 * self.n + max(nwv, 1))
        call("bo_solve", self.h, ctypes.byref(o), ctypes.byref(rep), ptr(sol))
        out = (rep.status, rep.iterations, sol[:3 * self.n + nwv])
        if report:
            return out + ({"restarts": rep.restarts, "rel_res": rep.rel_res,
                           "fallback": rep.fallback},)
        return out

    def dd_solve(self, tol=1e-3, maxit=500):
        """solve() as K subdomains (the y slabs of `subdomains`): subdomain-
        local vectors with ghost rows, device halo copies, all-reduced inner
        products.  Returns (status, iterations, sol[3n + nw])."""
        o = L.BoSolveOpts(tol=float(tol), max_it=int(maxit))
        rep = L.BoSolveReport()
        sol = np.zeros(3 * self.n + max(self.nw, 1))
        call("bo_dd_solve", self.h, ctypes.byref(o), ctypes.byref(rep), ptr(sol))
        return rep.status, rep.iterations, sol[:3 * self.n + self.nw]

    def newton_update(self, **opts):
        o = L.newton_opts(**opts)
        call("bo_newton_update", self.h, ctypes.byref(o))

    def step(self, dt, raise_on_fail=False, **opts):
        """One report step; returns (status, report dict)."""
        o = L.newton_opts(**opts)
        rep = L.BoStepReport()
        Lb = L.load()
        st = Lb.bo_step(self.h, float(dt), ctypes.byref(o), ctypes.byref(rep))
        if st != 0 and (raise_on_fail or st != 4):
            raise L.BoError(st, Lb.bo_last_error().decode())
        return st, {"newton_its": rep.newton_its, "lin_its": rep.lin_its, "cuts": rep.cuts,
                    "substeps": rep.substeps, "status": rep.status, "mb": list(rep.mb),
                    "cnv": list(rep.cnv), "well_res": rep.well_res,
                    "ms_assemble": rep.ms_assemble, "ms_solve": rep.ms_solve,
                    "ms_update": rep.ms_update}

    @property
    def dt_next(self):
        v = ctypes.c_double()
        call("bo_get_step_control", self.h, ctypes.byref(v))
        return v.value

    @dt_next.setter
    def dt_next(self, v):
        call("bo_set_step_control", self.h, float(v))

    @property
    def precision(self):
        """"fp64" or "mixed" (FP32 ILU(0) factors and sweeps)."""
        v = ctypes.c_int()
        call("bo_get_precision", self.h, ctypes.byref(v))
        return {q: k for k, q in L.PRECISION.items()}[v.value]

    @precision.setter
    def precision(self, name):
        call("bo_set_precision", self.h, L.PRECISION[name])

    @property
    def preconditioner(self):
        """"ilu0" (block ILU(0)) or "cpr" (two-stage CPR with AMG pressure stage)."""
        v = ctypes.c_int()
        call("bo_get_preconditioner", self.h, ctypes.byref(v))
        return {q: k for k, q in L.PRECONDITIONER.items()}[v.value]

    @preconditioner.setter
    def preconditioner(self, name):
        call("bo_set_preconditioner", self.h, L.PRECONDITIONER[name])

    @property
    def solve_schedule(self):
        """"tiled" (wavefront-tiled kernels over the GPU) or "block" (the whole
        ILU(0)-BiCGStab solve in one launch of one CTA, for small models)."""
        v = ctypes.c_int()
        call("bo_get_solve_schedule", self.h, ctypes.byref(v))
        return {q: k for k, q in L.SCHEDULE.items()}[v.value]

    @solve_schedule.setter
    def solve_schedule(self, name):
        call("bo_set_solve_schedule", self.h, L.SCHEDULE[name])

    def cpr_hierarchy(self):
        """(sizes per level, aggregation maps of levels 0 .. L-2)."""
        nl = ctypes.c_int()
        sizes = np.zeros(16, dtype=np.int32)
        call("bo_cpr_hierarchy", self.h, 16, ctypes.byref(nl), ptr(sizes), None)
        L_ = nl.value
        agg = np.zeros(max(1, int(sizes[:L_ - 1].sum())), dtype=np.int32)
        call("bo_cpr_hierarchy", self.h, 16, ctypes.byref(nl), ptr(sizes), ptr(agg))
        maps, off = [], 0
        for l in range(L_ - 1):
            maps.append(agg[off:off + sizes[l]].copy())
            off += sizes[l]
        return [int(v) for v in sizes[:L_]], maps

    def cpr_pressure_system(self):
        """(w [n, 3], ap [n, 7]) of the last factorisation with CPR."""
        w = np.zeros(3 * self.n)
        ap = np.zeros(7 * self.n)
        call("bo_cpr_pressure_system", self.h, ptr(w), ptr(ap))
        return w.reshape(-1, 3), ap.reshape(-1, 7)

    def cpr_vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        call("bo_cpr_vcycle", self.h, ptr(b), ptr(x))
        return x

    @property
    def subdomains(self):
        """Block-Jacobi slab height in y (0: no cut in y)."""
        return self._subdomains()[0]

    @subdomains.setter
    def subdomains(self, ysub):
        call("bo_set_subdomains", self.h, int(ysub), self._subdomains()[1])

    @property
    def subdomains_z(self):
        """Block-Jacobi slab height in z (0: no cut in z)."""
        return self._subdomains()[1]

    @subdomains_z.setter
    def subdomains_z(self, zsub):
        call("bo_set_subdomains", self.h, self._subdomains()[0], int(zsub))

    def _subdomains(self):
        y, z = ctypes.c_int(), ctypes.c_int()
        call("bo_get_subdomains", self.h, ctypes.byref(y), ctypes.byref(z))
        return y.value, z.value

    # -- learned preconditioner stage ----------------------------------------
    def learn_set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        call("bo_learn_set_params", self.h, ptr(theta), int(theta.size))

    def learn_get_params(self):
        theta = np.zeros(L.LEARN_NPARAM)
        call("bo_learn_get_params", self.h, ptr(theta), L.LEARN_NPARAM)
        return theta

    @property
    def learn_engine(self):
        """"tcgen05" (default) or "mma_sync": the tensor-core kernel of the network."""
        v = ctypes.c_int()
        call("bo_learn_get_engine", self.h, ctypes.byref(v))
        return {0: "mma_sync", 1: "tcgen05"}[v.value]

    @learn_engine.setter
    def learn_engine(self, name):
        call("bo_learn_set_engine", self.h, {"mma_sync": 0, "tcgen05": 1}[name])

    def learn_collect(self, max_systems, samples=16):
        """Keep the next max_systems linear systems with their first `samples`
        residuals for offline training (0: stop collecting)."""
        call("bo_learn_collect", self.h, int(max_systems), int(samples))

    def learn_set_info(self):
        """(kept systems, kept residuals) of the offline set."""
        a, b = ctypes.c_int(), ctypes.c_int()
        call("bo_learn_set_info", self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def learn_train_offline(self, epochs=1, lr=1e-3):
        """Adam over every kept residual on its own system; returns the mean
        loss of the first and of the last pass."""
        f, l = ctypes.c_double(), ctypes.c_double()
        call("bo_learn_train_offline", self.h, int(epochs), float(lr), ctypes.byref(f),
             ctypes.byref(l))
        return f.value, l.value

    def learn_enable(self, on=True):
        call("bo_learn_enable", self.h, 1 if on else 0)

    def learn_online(self, samples=16, epochs=1, lr=1e-3, on=True):
        """Train after every later linear solve on its first `samples`
        BiCGStab residuals (on=False turns it off)."""
        if not on:
            call("bo_learn_online", self.h, None)
            return
        o = L.BoLearnOpts(samples=int(samples), epochs=int(epochs), lr=float(lr))
        call("bo_learn_online", self.h, ctypes.byref(o))

    def learn_guard(self, probe):
        """A/B window of the stage (bo_learn_guard)."""
        call("bo_learn_guard", self.h, int(probe))

    def learn_report(self):
        r = L.BoLearnReport()
        call("bo_learn_get_report", self.h, ctypes.byref(r))
        return {k: getattr(r, k) for k, _ in L.BoLearnReport._fields_}

    def learn_delta(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        d = np.zeros_like(r)
        call("bo_learn_delta", self.h, ptr(r), ptr(d))
        return d

    def learn_loss_grad(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        loss = ctypes.c_double()
        g = np.zeros(L.LEARN_NPARAM)
        call("bo_learn_loss_grad", self.h, ptr(r), ctypes.byref(loss), ptr(g))
        return loss.value, g

    # -- timing --------------------------------------------------------------
    def set_timing(self, enabled: bool):
        call("bo_set_timing", self.h, 1 if enabled else 0)

    @property
    def launches(self):
        """Kernels launched for this object so far (bo_get_launch_count)."""
        v = ctypes.c_longlong()
        call("bo_get_launch_count", self.h, ctypes.byref(v))
        return v.value

    def timing(self):
        k = 16
        names = (ctypes.c_char * 32 * k)()
        ms = np.zeros(k)
        cnt = np.zeros(k, dtype=np.int64)
        count = ctypes.c_int()
        call("bo_get_timing", self.h, k, ctypes.cast(names, ctypes.c_void_p), ptr(ms), ptr(cnt),
             ctypes.byref(count))
        return {bytes(names[q]).split(b"\0")[0].decode(): (float(ms[q]), int(cnt[q]))
                for q in range(count.value)}
