"""The per-step JSON run log (paper_1910_06059_gb300/report.py) on a stand-in
simulator object: no GPU, the formatting and bookkeeping only."""
from __future__ import annotations

import io
import json

import numpy as np

from paper_1910_06059_gb300.report import StepLog, step_record


class _FakeSim:
    model = {"wells": [{"kind": "inj"}, {"kind": "prod"}]}

    def __init__(self, statuses):
        self.statuses = list(statuses)

    def step(self, dt, **opts):
        st = self.statuses.pop(0)
        return st, {"newton_its": 7, "lin_its": 300, "cuts": 1 if st else 0, "substeps": 3,
                    "mb": [1e-8, 2e-8, 3e-8], "cnv": [1e-7, 2e-7, 3e-7], "well_res": 1e-9,
                    "ms_assemble": 1.5, "ms_solve": 20.0, "ms_update": 0.5}

    def well_rates(self):
        return (np.array([[-1e-3, 0.0, 0.0], [2e-5, 1e-3, 5e-2]]), np.array([3.0e7, 2.0e7]),
                np.array([0, 1], dtype=np.int32))


def test_step_log_lines():
    out = io.StringIO()
    log = StepLog(_FakeSim([0, 4, 0]), out, well_names=["I1", "P1"])
    day = 86400.0
    for _ in range(3):
        log.step(10 * day)
    lines = [json.loads(s) for s in out.getvalue().splitlines()]
    assert [r["t_days"] for r in lines] == [10.0, 10.0, 20.0]   # a failed step does not advance
    assert [r["status"] for r in lines] == [0, 4, 0] and lines[1]["cuts"] == 1
    w = lines[0]["wells"]
    assert [x["name"] for x in w] == ["I1", "P1"] and [x["control"] for x in w] == ["rate", "bhp"]
    assert np.isclose(w[0]["q_water_m3_day"], -1e-3 * day) and np.isclose(w[1]["q_gas_m3_day"], 5e-2 * day)
    assert w[1]["bhp_pa"] == 2.0e7
    assert lines[0]["ms"] == {"assemble": 1.5, "solve": 20.0, "update": 0.5}


def test_step_record_default_names():
    rec = step_record(86400.0, 86400.0, 0, _FakeSim([0]).step(1.0)[1],
                      *_FakeSim([]).well_rates(), names=["a", "b"])
    assert rec["dt_days"] == 1.0 and len(rec["wells"]) == 2
    log = StepLog(_FakeSim([0]), io.StringIO())
    assert log.names == ["inj0", "prod1"]
