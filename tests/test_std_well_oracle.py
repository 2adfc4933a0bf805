"""Pins of the full standard-well oracle (oracle/std_well.py; Section 2.2.1:
four unknowns per well, cross-flow, wellbore storage): without cross-flow
and storage it reaches the reduced well's solution (two independent
formulations of the same equations); with cross-flow it conserves every
component across the reservoir, the connections and the wellbore."""
from __future__ import annotations

import numpy as np

import oracle
import synth
from helpers import _well, make_model
from oracle.std_well import StandardWellModel


def test_full_well_without_crossflow_equals_the_reduced_well():
    """A rate-controlled water injector (every connection injecting) and a
    BHP producer (every connection producing), no storage: the four-unknown
    wells and the BHP-only reduced wells give the same states, BHPs and
    surface rates after each report step."""
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    m["wells"] = m["wells"][:2]
    red = oracle.Oracle(m)
    red.init_hydrostatic()
    full = StandardWellModel(m, storage=False)
    full.set_state(*red.get_state())
    tight = dict(tol_mb=1e-11, tol_cnv=1e-11, tol_well=1e-11, tol_lin=1e-12, max_cuts=0)
    for days in (0.1, 0.5):
        dt = days * synth.DAY
        red.dt_next = dt
        st, rep = red.step(dt, **tight)
        ok, its = full.step(dt, tol=1e-11)
        assert st == 0 and ok, (rep, its)
        pr, swr, xr, fr, br = red.get_state()
        pf, swf, xf, ff, bf = full.get_state()
        assert np.array_equal(fr, ff)
        assert np.max(np.abs(pf - pr) / pr) <= 1e-12
        assert np.max(np.abs(swf - swr)) <= 1e-12
        assert np.max(np.abs(xf - xr) / np.abs(xr).clip(1e-300)) <= 1e-12
        assert np.allclose(bf, br, rtol=1e-12, atol=0)
        q_red = red.well_rates()[0]
        q_full = np.array([full._Q(w["x"]) for w in full.wells])
        assert np.allclose(q_full, q_red, rtol=1e-9, atol=1e-12 * np.abs(q_red).max())


def _crossflow_column(storage):
    """A BHP producer perforating the top and bottom cells of a column whose
    middle cell seals them apart; the top is above the BHP and produces, the
    bottom is below it and takes the wellbore mixture back."""
    perm = np.array([300.0, 1e-9, 300.0]) * synth.MD
    wells = [_well(0, 0, [0, 2], "prod", "bhp", 4000 * synth.PSI, 4000 * synth.PSI)]
    m = make_model(1, 1, 3, perm, 0.2, wells, dx=50.0, dy=50.0, dz=5.0)
    m["fluid"]["g"] = 0.0
    s = StandardWellModel(m, storage=storage)
    p = np.array([5000.0, 4500.0, 3500.0]) * synth.PSI
    s.set_state(p, np.full(3, 0.3), np.full(3, 150.0), np.ones(3, np.uint8),
                np.array([4000 * synth.PSI]))
    return m, s


def _masses(m, s):
    pv = s.o.static()["pv"]
    p, sw, x, fl = s.cells()
    M = np.zeros(3)
    for c in range(s.n):
        cp = oracle.cell_props(m["fluid"], p[c], sw[c], x[c], fl[c])
        M += pv[c] * np.array([cp["A_w"][0], cp["A_o"][0], cp["A_g"][0]])
    return M


def test_crossflow_conserves_every_component():
    for storage in (False, True):
        m, s = _crossflow_column(storage)
        M0 = _masses(m, s)
        w = s.wells[0]
        A0 = s._storage(w, w["x"])
        dt = 0.2 * synth.DAY
        ok, its = s.step(dt, tol=1e-12)
        assert ok, its
        p, sw, x, fl = s.cells()
        q = s._well_rates(w, p, sw, x, fl, w["x"][3])
        Q = s._Q(w["x"])
        # the top connection produces, the bottom one takes fluid back
        assert np.all(q[0] > 0) and np.all(q[1] < 0)
        # ... with the wellbore's composition
        assert np.allclose(q[1] / q[1].sum(), Q / Q.sum(), rtol=1e-12)
        # wellbore: what the connections deliver leaves at the surface or is stored
        scale = np.abs(q).sum(axis=0)
        dA = s._storage(w, w["x"]) - A0
        assert np.all(np.abs(q.sum(axis=0) - Q - dA / dt) <= 1e-12 * scale)
        if storage:
            assert np.abs(dA).max() > 0
        # reservoir: its component masses fall by what the connections take
        assert np.all(np.abs(_masses(m, s) - M0 + q.sum(axis=0) * dt) <= 1e-10 * scale * dt)


def test_the_reduced_well_has_no_crossflow():
    """The same column with the reduced well: the bottom connection does not
    take fluid back (reverse flow is set to zero), so the two models differ
    exactly where the standard well's cross-flow acts."""
    m, s = _crossflow_column(False)
    red = oracle.Oracle(m)
    red.set_state(*s.get_state())
    red.dt_next = 0.2 * synth.DAY
    st, _ = red.step(0.2 * synth.DAY, tol_mb=1e-12, tol_cnv=1e-12, tol_lin=1e-12, max_cuts=0)
    assert st == 0
    s.step(0.2 * synth.DAY, tol=1e-12)
    p_red = red.get_state()[0]
    p_full = s.get_state()[0]
    assert abs(p_full[2] - p_red[2]) > 1e3     # the bottom cell gained fluid only with cross-flow
    assert abs(p_full[0] - p_red[0]) / p_red[0] < 1e-2


def test_exact_well_jacobian_against_central_differences():
    """The dual-number Jacobian of the well terms (``assemble``) against
    central differences of the plain residual (``assemble_fd``): producing
    and cross-flowing connections with storage, a rate-controlled injector
    and BHP producers, and a rate-controlled producer.  Central differences
    of step 1e-6 carry errors near 1e-9 relative; the bar is 1e-6 on every
    entry above 1e-9 of the largest in its row."""
    cases = []
    m, s = _crossflow_column(True)
    cases.append((s, 0.2 * synth.DAY))
    m2 = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    red = oracle.Oracle(m2)
    red.init_hydrostatic()
    s2 = StandardWellModel(m2, storage=True)
    s2.set_state(*red.get_state())
    cases.append((s2, 0.5 * synth.DAY))
    m3 = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    m3["wells"][1] = dict(m3["wells"][1], control="rate", target=200 * synth.STB / synth.DAY)
    red3 = oracle.Oracle(m3)
    red3.init_hydrostatic()
    s3 = StandardWellModel(m3, storage=True)
    s3.set_state(*red3.get_state())
    cases.append((s3, 0.5 * synth.DAY))
    for s, dt in cases:
        s.o.begin_step()
        s._begin_wells()
        J, R = s.assemble(dt)
        Jf, Rf = s.assemble_fd(dt)
        assert np.array_equal(R, Rf)
        row = np.abs(Jf).max(axis=1, keepdims=True)
        big = np.abs(Jf) > 1e-9 * row
        err = np.abs(J - Jf) / np.maximum(np.abs(Jf), 1e-300)
        assert err[big].max() <= 1e-6, err[big].max()
        assert np.all(np.abs(J[~big]) <= 1e-8 * np.broadcast_to(row, J.shape)[~big])
