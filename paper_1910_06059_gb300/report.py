"""Run log of a simulation: one JSON line per report step.

A reservoir simulator reports, per report step, its time, step length,
Newton and linear iteration counts, time-step cuts, convergence measures and
the wells' rates and bottom-hole pressures (the well curves that the paper's
Section 3 compares between simulators).  ``StepLog`` assembles that line from ``bo_step``'s
report and the well production report (``bo_get_well_rates``); it only
formats what the library returns.
"""
from __future__ import annotations

import json

DAY = 86400.0


def step_record(t_end, dt, status, rep, rates, bhp, control, names):
    """The JSON-ready record of one report step (SI units; times in days and
    seconds, surface rates in m^3/day, production positive)."""
    wells = []
    for q, name in enumerate(names):
        wells.append({
            "name": name,
            "control": "rate" if int(control[q]) == 0 else "bhp",
            "bhp_pa": float(bhp[q]),
            "q_water_m3_day": float(rates[q][0]) * DAY,
            "q_oil_m3_day": float(rates[q][1]) * DAY,
            "q_gas_m3_day": float(rates[q][2]) * DAY,
        })
    return {
        "t_days": t_end / DAY,
        "dt_days": dt / DAY,
        "status": int(status),
        "newton_its": int(rep["newton_its"]),
        "lin_its": int(rep["lin_its"]),
        "cuts": int(rep["cuts"]),
        "substeps": int(rep["substeps"]),
        "mb": [float(v) for v in rep["mb"]],
        "cnv": [float(v) for v in rep["cnv"]],
        "well_res": float(rep["well_res"]),
        "ms": {"assemble": float(rep["ms_assemble"]), "solve": float(rep["ms_solve"]),
               "update": float(rep["ms_update"])},
        "wells": wells,
    }


class StepLog:
    """Steps a ``Sim`` report step by report step and writes one JSON line
    per step to ``out`` (a path or an open text file)."""

    def __init__(self, sim, out, t0=0.0, well_names=None):
        self.sim = sim
        self.t = float(t0)
        self.names = list(well_names) if well_names is not None else [
            f"{w['kind']}{q}" for q, w in enumerate(sim.model["wells"])]
        self._own = isinstance(out, str)
        self.out = open(out, "a") if self._own else out

    def step(self, dt, **opts):
        """One report step; returns (status, record).  A failed step (status
        != 0) is logged with the time left where it started."""
        status, rep = self.sim.step(dt, **opts)
        if status == 0:
            self.t += dt
        rates, bhp, control = self.sim.well_rates()
        rec = step_record(self.t, dt, status, rep, rates, bhp, control, self.names)
        self.out.write(json.dumps(rec) + "\n")
        self.out.flush()
        return status, rec

    def close(self):
        if self._own:
            self.out.close()
