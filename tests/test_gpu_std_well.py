"""Full standard well on the GPU against the oracle (Section 2.2.1: Q_t, F_w,
F_g, p_bhp per well, cross-flow, wellbore storage; Eq. wellequation's Schur
complement with a 4x4 D_w).  Needs a GB300.

Bars:
  well unknowns after initialisation        1e-12 relative
  B_w, C_w, D_w per entry                   1e-12, an entry judged against
                                            max(|oracle|, 1e-3 * the largest
                                            entry of the same unknown and the
                                            same kind of equation in the well)
  R_w                                       1e-12 of the terms it sums
  cell residual and Jacobian                as for the reduced well (1e-12)
  linear solution (tight solve)             1e-9 relative per unknown family
  Newton states (tolerance 1e-10)           pressure 1e-6 relative, saturations
                                            1e-6 absolute, well unknowns and
                                            surface rates 1e-6 relative
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import bcsr_to_dense, family_close, vec_close
from oracle.std_well import StandardWellModel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1910_06059_gb300.build import build
    build()


def _crossflow_5spot():
    """A 7x7x4 five-spot whose second layer seals the top from the bottom and
    whose two lower layers start 25% below hydrostatic pressure: producers
    take fluid from the top layers and give part of it back to the bottom
    ones (cross-flow), the water injector injects at a rate target."""
    m = synth.small_model(7, 7, 4, wells="5spot", dz=4.0)
    perm = np.asarray(m["perm"]).reshape(4, 49).copy()
    perm[1] = 1e-6 * synth.MD
    m["perm"] = perm.reshape(-1)
    red = oracle.Oracle(m)
    red.init_hydrostatic()
    p, sw, x, fl, bhp = red.get_state()
    p = p.copy()
    p.reshape(4, 49)[2:] *= 0.75
    return m, (p, sw, x, fl, bhp)


def _rate_producer():
    """The small five-spot with its first producer under an oil-rate target."""
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    m["wells"][1] = dict(m["wells"][1], control="rate", target=200 * synth.STB / synth.DAY)
    red = oracle.Oracle(m)
    red.init_hydrostatic()
    return m, red.get_state()


def _hydrostatic(make):
    def f():
        m = make()
        red = oracle.Oracle(m)
        red.init_hydrostatic()
        return m, red.get_state()
    return f


CASES = {
    "crossflow_5spot_7x7x4": _crossflow_5spot,
    "rate_producer_6x5x4": _rate_producer,
    "gas_7x6x5": _hydrostatic(lambda: synth.small_model(7, 6, 5, wells="gas", dz=5.0)),
    "config0": _hydrostatic(synth.config0),
}


def _pair(name, storage=True):
    m, st = CASES[name]()
    from paper_1910_06059_gb300 import Sim
    g = Sim(m)
    g.set_well_model("standard", storage=storage)
    assert g.well_model == "standard"
    g.set_state(*st)
    o = StandardWellModel(m, storage=storage)
    o.set_state(*st)
    return m, g, o


def _family_err(a, b, kinds_axis, kinds):
    """Max error of blocks b[..., r, c] judged against max(|b|, 1e-3 * max |b|
    over every block and every row of the same kind, same column)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    err = 0.0
    for rows in kinds:
        sl = [slice(None)] * b.ndim
        sl[kinds_axis] = rows
        bb, aa = b[tuple(sl)], a[tuple(sl)]
        red = tuple(q for q in range(bb.ndim) if q != bb.ndim - 1)
        fam = np.abs(bb).max(axis=red, keepdims=True)
        scale = np.maximum(np.abs(bb), 1e-3 * fam)
        scale = np.where(scale == 0, 1.0, scale)
        err = max(err, float((np.abs(aa - bb) / scale).max()))
    return err


def _oracle_blocks(o, dt):
    n = o.n
    J, R = o.assemble(dt)
    out = []
    for k, w in enumerate(o.wells):
        col = 3 * n + 4 * k
        B = np.array([J[col:col + 4, 3 * c:3 * c + 3] for c in w["cells"]])
        C = np.array([J[3 * c:3 * c + 3, col:col + 4] for c in w["cells"]])
        blk = o.well_blocks(k, dt)
        out.append({"B": B, "C": C, "D": J[col:col + 4, col:col + 4].copy(),
                    "Rw": R[col:col + 4].copy(), "q": blk["q"], "x": w["x"].copy()})
    return J, R, out


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("storage", [True, False])
def test_std_well_blocks(name, storage):
    m, g, o = _pair(name, storage)
    for a, b in zip(g.std_wells(blocks=False), o.wells):
        assert np.allclose(a["xw"], b["x"], rtol=1e-12, atol=1e-300), (a["xw"], b["x"])
    dt = 0.5 * synth.DAY
    g.begin_step()
    g.assemble(dt)
    o.o.begin_step()
    o._begin_wells()
    J, R, ob = _oracle_blocks(o, dt)
    n = o.n
    # cell rows: residual and Jacobian with the connection terms
    rpg, cig, vg, Rg = g.system()
    rpo, cio, vo, _ = o.o.system()
    Jc = J[:3 * n, :3 * n]
    vo2 = np.array([Jc[3 * i:3 * i + 3, 3 * cio[q]:3 * cio[q] + 3]
                    for i in range(n) for q in range(rpo[i], rpo[i + 1])])
    assert family_close(vg, vo2, rpo) <= 1e-12
    Ro = R[:3 * n].reshape(n, 3)
    scale = np.maximum(np.abs(Ro), 1e-3 * np.abs(Ro).max(axis=0))
    assert np.max(np.abs(Rg - Ro) / scale) <= 1e-12
    for k, (a, b) in enumerate(zip(g.std_wells(), ob)):
        assert np.allclose(a["xw"], b["x"], rtol=1e-12, atol=0)
        assert _family_err(a["B"], b["B"], 1, [[0, 1, 2], [3]]) <= 1e-12, ("B", k)
        assert _family_err(a["C"], b["C"], 1, [[0, 1, 2]]) <= 1e-12, ("C", k)
        assert _family_err(a["D"][None], b["D"][None], 1, [[0, 1, 2], [3]]) <= 1e-12, ("D", k)
        # R_w sums storage, surface rates and connection rates: judge it
        # against the size of those terms
        terms = np.abs(b["q"]).sum(axis=0) + np.abs(o._Q(b["x"])) + \
            np.abs(o._storage(o.wells[k], b["x"]) - o.wells[k]["A0"]) / dt
        assert np.all(np.abs(a["Rw"][:3] - b["Rw"][:3]) <= 1e-12 * np.maximum(terms.max(), 1e-300))
        w = o.wells[k]
        tscale = max(abs(w["spec"]["target"]), abs(w["spec"]["bhp_limit"]), np.abs(o._Q(b["x"])).max())
        assert abs(a["Rw"][3] - b["Rw"][3]) <= 1e-12 * tscale, ("Rw3", k)
    # the convergence measures (reservoir MB/CNV with the well terms, well residual)
    ng = g.norms(dt)
    mb, cnv, wres = o.norms(dt, R)
    assert np.allclose(ng[3:6], cnv, rtol=1e-11, atol=0)
    assert ng[6] == pytest.approx(wres, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("name", list(CASES))
def test_std_well_linear_solution(name):
    """One tight BiCGStab solve of the well-reduced system, well unknowns
    recovered by x_w = D_w^-1 (R_w - B_w x_r), against the oracle's dense
    solve of the unreduced system."""
    m, g, o = _pair(name)
    dt = 0.1 * synth.DAY
    g.begin_step()
    g.assemble(dt)
    o.o.begin_step()
    o._begin_wells()
    J, R = o.assemble(dt)
    dx = np.linalg.solve(J, R)
    st, its, sol = g.solve(tol=1e-13, maxit=1000)
    assert st == 0, its
    n = o.n
    # the GPU solution solves the oracle's unreduced system
    res = J @ sol - R
    for a in range(3):
        assert np.abs(res[a:3 * n:3]).max() <= 1e-9 * np.abs(R[a:3 * n:3]).max(), a
    # per unknown family: 1e-9 of the family's largest update, plus 1e-11 of
    # the variable's own size (an update family far below its variable's
    # size, like the r_go updates of an undersaturated state over a short
    # step, is rounding noise of the solve on both sides)
    p, sw, x, fl = o.cells()
    natural = [np.abs(p).max(), 1.0, max(np.abs(x).max(), 1.0)]
    for v in range(3):
        a, b = sol[v:3 * n:3], dx[v:3 * n:3]
        bar = 1e-9 * np.abs(b).max() + 1e-11 * natural[v]
        assert np.abs(a - b).max() <= bar, (v, np.abs(a - b).max(), bar)
    for k in range(o.nw):
        a, b = sol[3 * n + 4 * k:3 * n + 4 * k + 4], dx[3 * n + 4 * k:3 * n + 4 * k + 4]
        scale = np.array([abs(o.wells[k]["x"][0]) + abs(b[0]), 1.0, 1.0, abs(o.wells[k]["x"][3])])
        assert np.all(np.abs(a - b) <= 1e-9 * scale), (k, a, b)


def _gpu_newton(g, dt, tol, max_newton=30):
    g.begin_step()
    for it in range(max_newton + 1):
        g.assemble(dt)
        nrm = g.norms(dt)
        if nrm.max() <= tol:
            return True, it
        if it == max_newton:
            return False, it
        st, _, _ = g.solve(tol=1e-12, maxit=1000)
        assert st == 0
        g.newton_update()
    return False, max_newton


@pytest.mark.parametrize("name", ["crossflow_5spot_7x7x4", "config0", "rate_producer_6x5x4"])
def test_std_well_newton_parity(name):
    """Sub-steps of 0.1, 0.5 and 2 days, each one Newton solve to 1e-10 on
    both sides (the same iteration: chop, switching, well update)."""
    m, g, o = _pair(name)
    crossflow_seen = False
    for days in (0.1, 0.5, 2.0):
        dt = days * synth.DAY
        okg, itg = _gpu_newton(g, dt, 1e-10)
        oko, ito = o.step(dt, tol=1e-10)
        assert okg and oko, (itg, ito)
        assert abs(itg - ito) <= 1
        pg, swg, xg, fg, bg = g.get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo)
        assert np.max(np.abs(pg - po) / po) <= 1e-6
        assert np.max(np.abs(swg - swo)) <= 1e-6
        sat = fo == 0
        assert np.max(np.abs(xg[sat] - xo[sat]), initial=0.0) <= 1e-6
        assert np.max(np.abs(xg[~sat] - xo[~sat]) / xo[~sat].clip(1e-300), initial=0.0) <= 1e-6
        assert np.allclose(bg, bo, rtol=1e-6)
        qg, _, ctl = g.well_rates()
        for k, (a, w) in enumerate(zip(g.std_wells(blocks=False), o.wells)):
            scale = np.array([abs(w["x"][0]), 1.0, 1.0, abs(w["x"][3])])
            assert np.all(np.abs(a["xw"] - w["x"]) <= 1e-6 * scale), (k, a["xw"], w["x"])
            Q = o._Q(w["x"])
            assert np.allclose(qg[k], Q, rtol=1e-6, atol=1e-6 * np.abs(Q).max())
            assert ctl[k] == w["control"]
            p, sw, x, fl = o.cells()
            q = o._well_rates(w, p, sw, x, fl, w["x"][3])
            if not w["inj"] and (q.sum(axis=1) < 0).any():
                crossflow_seen = True
    if name == "crossflow_5spot_7x7x4":
        assert crossflow_seen


def test_std_well_report_steps_and_model_switch():
    """bo_step with the full standard well: report steps converge with
    sub-stepping and cuts; switching back to the reduced well restores its
    results bit for bit."""
    m, st = _crossflow_5spot()
    from paper_1910_06059_gb300 import Sim
    ref = Sim(m)
    ref.set_state(*st)
    s0, r0 = ref.step(synth.DAY)
    g = Sim(m)
    g.set_well_model("standard")
    g.set_state(*st)
    for _ in range(3):
        s, rep = g.step(2 * synth.DAY)
        assert s == 0, rep
    g.set_well_model("reduced")
    assert g.well_model == "reduced"
    g.set_state(*st)
    g.dt_next = 0.0
    ref_state = ref.get_state()
    s1, r1 = g.step(synth.DAY)
    assert s0 == s1 == 0
    assert r0["newton_its"] == r1["newton_its"] and r0["lin_its"] == r1["lin_its"]
    for a, b in zip(g.get_state(), ref_state):
        assert np.array_equal(a, b)
