"""Equilibration from a datum and the contacts (bo_init_equilibrium) against
the oracle's (orc_init_equilibrium), through the C ABI.

Both integrate the same RK4 steps; they differ only in rounding and in the
exp of the device and host libraries, so pressures agree to 1e-12 relative
and saturations, dissolved ratios and phase flags exactly (no cell sits at
its bubble point in these inputs).  A Newton step from the equilibrated
state then meets the same 1e-6 state bar as the plain path."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
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


def _model():
    # 12 layers of 10 ft under 2500 m: contacts inside the column
    return synth.small_model(6, 5, 12, wells="5spot", dz=10.0)


@pytest.mark.parametrize("datum", [2512.0, 2503.0, 2530.0])   # oil, gas, water zone
def test_equilibrium_vs_oracle(datum):
    from paper_1910_06059_gb300 import Sim
    m = _model()
    g, o = Sim(m), oracle.Oracle(m)
    e = (datum, 26.0e6, 2525.0, 2506.0, 120.0, 0.15)
    g.init_equilibrium(*e)
    o.init_equilibrium(*e)
    pg, swg, xg, fg, bg = g.get_state()
    po, swo, xo, fo, bo = o.get_state()
    assert np.max(np.abs(pg - po) / po) <= 1e-12
    assert np.array_equal(fg, fo) and np.array_equal(swg, swo) and np.array_equal(xg, xo)
    assert len(set(fo.tolist())) == 2          # both phase states present
    assert np.allclose(bg, bo, rtol=1e-12)


def test_newton_step_from_equilibrium():
    from paper_1910_06059_gb300 import Sim
    m = _model()
    g, o = Sim(m), oracle.Oracle(m)
    e = (2512.0, 26.0e6, 2525.0, 2506.0, 120.0, 0.15)
    g.init_equilibrium(*e)
    o.init_equilibrium(*e)
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10, max_cuts=0)
    for days in (0.01, 0.1):
        dt = days * synth.DAY
        g.dt_next = dt
        o.dt_next = dt
        stg, rg = g.step(dt, **tight)
        sto, ro = o.step(dt, **tight)
        assert stg == 0 and sto == 0, (days, rg, ro)
        pg, swg, xg, fg, bg = g.get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo)
        assert np.max(np.abs(pg - po) / po) <= 1e-6
        assert np.max(np.abs(swg - swo)) <= 1e-6


def test_equilibrium_rejects_bad_input():
    from paper_1910_06059_gb300 import Sim, _lib as L
    import ctypes
    g = Sim(_model())
    bad = (ctypes.c_double * 6)(2512.0, 26.0e6, 2500.0, 2506.0, 120.0, 0.15)   # GOC below WOC
    assert L.load().bo_init_equilibrium(g.h, bad) == 1
