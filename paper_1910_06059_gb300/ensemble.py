"""Python view of a batched ensemble of libbo.so models (marshalling only).

The ensemble steps its members concurrently on one GPU from a native pool
of workers with one CUDA stream each (``bo_ensemble_*`` in include/bo.h).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from ._lib import call
from .sim import Sim


class Ensemble:
    """Independent models stepped together; members are ``Sim`` objects."""

    def __init__(self, models=None, streams: int = 8, sims=None):
        """models: model dicts (members created and owned here), or sims:
        existing Sim objects (not owned; close them yourself)."""
        self._own = sims is None
        self.members = [Sim(m) for m in models] if sims is None else list(sims)
        arr = (ctypes.c_void_p * len(self.members))(*[s.h.value for s in self.members])
        h = ctypes.c_void_p()
        call("bo_ensemble_create", arr, len(self.members), int(streams), ctypes.byref(h))
        self.h = h
        self.cells = sum(s.n for s in self.members)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            call("bo_ensemble_destroy", self.h)
            self.h = None
        if getattr(self, "_own", False):
            for s in getattr(self, "members", []):
                s.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_hydrostatic(self):
        for s in self.members:
            s.init_hydrostatic()

    @property
    def schedule(self):
        w, lf = ctypes.c_int(), ctypes.c_int()
        call("bo_ensemble_get_schedule", self.h, ctypes.byref(w), ctypes.byref(lf))
        return {"streams": w.value, "largest_first": bool(lf.value)}

    def set_schedule(self, streams: int, largest_first: bool = True):
        call("bo_ensemble_set_schedule", self.h, int(streams), 1 if largest_first else 0)

    def step(self, dt, raise_on_fail=True, **opts):
        """One report step of every member; returns (statuses, reports)."""
        o = L.newton_opts(**opts)
        n = len(self.members)
        reps = (L.BoStepReport * n)()
        sts = (ctypes.c_int * n)()
        lib = L.load()
        st = lib.bo_ensemble_step(self.h, float(dt), ctypes.byref(o), reps, sts)
        if st != 0 and raise_on_fail:
            raise L.BoError(st, lib.bo_last_error().decode())
        out = [{"newton_its": r.newton_its, "lin_its": r.lin_its, "cuts": r.cuts,
                "substeps": r.substeps} for r in reps]
        return list(sts), out

    def autotune_precond(self, dt_probe, **opts):
        """Preconditioner per size class (members up to the median size, the
        larger ones) from a probe step of each of the four combinations;
        returns the probe times and the choice."""
        o = L.newton_opts(**opts)
        sec = np.zeros(4)
        ks, kl = ctypes.c_int(), ctypes.c_int()
        call("bo_ensemble_autotune_precond", self.h, float(dt_probe), ctypes.byref(o),
             sec.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ks), ctypes.byref(kl))
        names = {v: k for k, v in L.PRECONDITIONER.items()}
        combos = [("ilu0", "ilu0"), ("ilu0", "cpr"), ("cpr", "ilu0"), ("cpr", "cpr")]
        return {"probe_s": {f"small {a}, large {b}": float(t) for (a, b), t in zip(combos, sec)},
                "chosen": {"small": names[ks.value], "large": names[kl.value]}}

    def autotune_schedule(self, dt_probe, **opts):
        """Solve schedule of the members up to the median size ("tiled" or
        "block") and the worker count (current or four times it, at most
        256) from a probe step of each of the four combinations; returns the
        probe times and the choice."""
        o = L.newton_opts(**opts)
        sec = np.zeros(4)
        ks, ws = ctypes.c_int(), ctypes.c_int()
        w0 = self.schedule["streams"]
        call("bo_ensemble_autotune_schedule", self.h, float(dt_probe), ctypes.byref(o),
             sec.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ks), ctypes.byref(ws))
        names = {v: k for k, v in L.SCHEDULE.items()}
        labels = ["small tiled, workers w", "small block, workers w",
                  "small tiled, workers 4w", "small block, workers 4w"]
        return {"probe_s": {k: float(t) for k, t in zip(labels, sec)},
                "chosen": {"small": names[ks.value], "streams": int(ws.value)},
                "workers_before": w0}

    def last_step_ms(self):
        """Device time (CUDA events) of the last step, in ms (-1: not measured)."""
        v = ctypes.c_double()
        call("bo_ensemble_last_step_ms", self.h, ctypes.byref(v))
        return v.value

    def autotune(self, dt_probe, candidates=(1, 2, 4, 8, 16, 32), **opts):
        """Pick the worker count and order by timing a probe step of each
        candidate (states restored after each probe); returns the probe times."""
        o = L.newton_opts(**opts)
        cand = (ctypes.c_int * len(candidates))(*candidates)
        sec = np.zeros(2 * len(candidates))
        call("bo_ensemble_autotune", self.h, float(dt_probe), ctypes.byref(o), cand,
             len(candidates), sec.ctypes.data_as(ctypes.c_void_p))
        return {"largest_first": dict(zip(candidates, sec[:len(candidates)].tolist())),
                "given_order": dict(zip(candidates, sec[len(candidates):].tolist())),
                "chosen": self.schedule}
