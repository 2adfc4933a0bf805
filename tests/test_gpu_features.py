"""Checkpoint/restart, the run log and failure detection on the GPU path."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1910_06059_gb300.build import build
    build()


def test_restart_from_checkpoint_is_bitwise_identical():
    """State + carried sub-step length are the whole checkpoint: continuing
    from a restored checkpoint repeats the uninterrupted run bit for bit."""
    from paper_1910_06059_gb300 import Sim
    m = synth.config0()
    g = Sim(m)
    g.init_hydrostatic()
    for _ in range(2):
        g.step(m["dt"], raise_on_fail=True)
    snap = g.get_state()
    snap_dt = g.dt_next
    for _ in range(2):
        g.step(m["dt"], raise_on_fail=True)
    first = g.get_state()
    h = Sim(m)                      # a fresh object, as after a restart
    h.set_state(*snap)
    h.dt_next = snap_dt
    for _ in range(2):
        h.step(m["dt"], raise_on_fail=True)
    second = h.get_state()
    for a, b in zip(first, second):
        assert np.array_equal(a, b)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A device wait on a flag nothing sets runs out (about a second), is
    reported as BO_ERR_DEVICE_TIMEOUT, and the context stays usable."""
    import ctypes
    from paper_1910_06059_gb300 import Sim, _lib
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    g = Sim(m)
    lib = _lib.load()
    sec = ctypes.c_double(-1.0)
    st = lib.bo_selftest_bounded_wait(g.h, ctypes.byref(sec))
    assert st == 6, lib.bo_last_error().decode()          # BO_ERR_DEVICE_TIMEOUT
    assert 0.05 < sec.value < 30.0
    # the object and the context still work
    g.init_hydrostatic()
    st2, rep = g.step(synth.DAY)
    assert st2 == 0


def test_step_log_reports_the_library_values():
    """The JSON run log carries bo_step's counters and the well production
    report of the converged state, one line per report step."""
    import io
    import json
    from paper_1910_06059_gb300 import Sim
    from paper_1910_06059_gb300.report import StepLog
    m = synth.config0()
    g = Sim(m)
    g.init_hydrostatic()
    out = io.StringIO()
    log = StepLog(g, out)
    recs = [log.step(m["dt"])[1] for _ in range(2)]
    lines = [json.loads(s) for s in out.getvalue().splitlines()]
    assert lines == recs and [r["t_days"] for r in lines] == [30.0, 60.0]
    rates, bhp, control = g.well_rates()
    last = lines[-1]["wells"]
    for q in range(len(last)):
        assert np.isclose(last[q]["q_gas_m3_day"], rates[q, 2] * 86400.0, rtol=1e-15)
        assert last[q]["bhp_pa"] == bhp[q]
    assert all(r["status"] == 0 and r["newton_its"] > 0 for r in lines)
