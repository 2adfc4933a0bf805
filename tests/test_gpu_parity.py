"""GPU-vs-oracle parity through the C ABI (needs a GB300).

Tolerances:
  static data, hydrostatic state       1e-13 relative
  residual and Jacobian, per entry     1e-12 relative, an entry judged against
                                       max(|oracle|, 1e-3 * largest entry of the
                                       same unknown family in its block row)
  ILU(0) pivot inverses                1e-10 relative (same floor)
  preconditioner / operator applies    1e-11 relative to the vector's max
  linear solution (tight solve)        1e-9 relative per unknown family
  Newton states (tight tolerances)     pressure 1e-6 relative, saturations 1e-6 absolute
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import family_close, vec_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1910_06059_gb300.build import build
    build()


def Sim(m):
    from paper_1910_06059_gb300 import Sim as _S
    return _S(m)


MODELS = {
    "small_5spot": lambda: synth.small_model(6, 5, 4, wells="5spot", dz=4.0),
    "ragged_33x17x9": lambda: synth.small_model(33, 17, 9, wells="5spot", dz=3.0),
    "gas_7x6x5": lambda: synth.small_model(7, 6, 5, wells="gas", dz=5.0),
    "config0": synth.config0,
    "aniso_9x8x6": lambda: synth.anisotropic(synth.small_model(9, 8, 6, wells="5spot", dz=4.0),
                                             seed=1),
}


def _pair(name, seed=0, frac_sat=0.5):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    st = synth.random_state(m, seed_member=seed, frac_sat=frac_sat)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    p, sw, x, fl, bhp = [a.copy() for a in st]
    st2 = (p * 1.003, sw + 0.004, x, fl, bhp)
    g.set_state(*st2)
    o.set_state(*st2)
    return m, g, o


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(MODELS))
def test_static_data(name):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    sg, so = g.get_static(), o.static()
    for k in ("Tx", "Ty", "Tz", "pv", "depth", "wi"):
        assert vec_close(sg[k], so[k]) <= 1e-13, k


@pytest.mark.parametrize("name", ["small_5spot", "config0"])
def test_hydrostatic_initial_state(name):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.init_hydrostatic()
    o.init_hydrostatic()
    pg, swg, xg, fg, bg = g.get_state()
    po, swo, xo, fo, bo = o.get_state()
    assert np.max(np.abs(pg - po) / po) <= 1e-13
    assert np.array_equal(fg, fo) and np.array_equal(swg, swo) and np.array_equal(xg, xo)
    assert np.array_equal(bg, bo)


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("frac_sat", [0.0, 0.5, 1.0])
def test_assembly_parity(name, frac_sat):
    m, g, o = _pair(name, seed=3, frac_sat=frac_sat)
    dt = 3 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    rpg, cig, vg, Rg = g.system()
    rpo, cio, vo, Ro = o.system()
    assert np.array_equal(rpg, rpo) and np.array_equal(cig, cio)
    assert family_close(vg, vo, rpo) <= 1e-12
    # residual: per equation, floor by the row's flux scale
    scale = np.maximum(np.abs(Ro), 1e-3 * np.abs(Ro).max(axis=0))
    assert np.max(np.abs(Rg - Ro) / scale) <= 1e-12
    wg, wo = g.wells(), o.wells()
    for a, b in zip(wg, wo):
        assert a["control"] == b["control"]
        for k in ("Rw", "Dw"):
            assert abs(a[k] - b[k]) <= 1e-12 * max(abs(b[k]), abs(b["Dw"]) * 1e5, 1e-300), k
        for k in ("B", "C"):
            assert vec_close(a[k], b[k]) <= 1e-12, k
    ng, no = g.norms(dt), o.norms(dt)
    assert np.allclose(ng[3:], no[3:], rtol=1e-12, atol=0)
    # MB_a = (dt Bavg_a / PV_tot) |sum R_a| is a cancelling sum: its rounding
    # is bounded by the same factor times 1e-12 * sum |R_a|, where the factor
    # follows from CNV_a = dt Bavg_a max |R_a| / pv.
    pv = o.static()["pv"]
    factor = no[3:6] / (np.abs(Ro) / pv[:, None]).max(axis=0) / pv.sum()
    assert np.all(np.abs(ng[:3] - no[:3]) <= 1e-12 * factor * np.abs(Ro).sum(axis=0) + 1e-15 * no[:3])


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9", "config0"])
def test_ilu0_and_operator_parity(name):
    m, g, o = _pair(name, seed=5)
    dt = 2 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    dinv = g.factor()
    rp, ci, vals, _ = o.system()
    lu, uinv = o.ilu0()
    assert family_close(dinv, uinv, np.arange(o.n + 1), per_equation=False) <= 1e-10
    rng = np.random.default_rng(11)
    r = rng.standard_normal(3 * o.n)
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    for v in range(3):
        assert vec_close(zg[v::3], zo[v::3]) <= 1e-11
    x = rng.standard_normal(3 * o.n) * np.tile([1e5, 0.1, 1.0], o.n)
    yg, yo = g.apply_op(x), o.apply_op(x)
    for v in range(3):
        assert vec_close(yg[v::3], yo[v::3]) <= 1e-11


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9", "gas_7x6x5"])
def test_bicgstab_solution_parity(name):
    # random states with a long step give systems that ILU0-BiCGStab does not
    # solve (the oracle stalls too); a short step keeps them well conditioned
    m, g, o = _pair(name, seed=7)
    dt = 0.1 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    stg, itg, solg = g.solve(tol=1e-12, maxit=500)
    sto, ito, solo = o.solve(tol=1e-12, maxit=500)
    assert stg == 0 and sto == 0
    # rounding makes long BiCGStab runs drift by a few iterations; the
    # solution is unique and is what must agree
    assert abs(itg - ito) <= max(2, 0.05 * ito)
    n = o.n
    for v in range(3):
        assert vec_close(solg[v:3 * n:3], solo[v:3 * n:3]) <= 1e-9
    assert np.allclose(solg[3 * n:], solo[3 * n:], rtol=1e-9, atol=1e-9 * np.abs(solo[3 * n:]).max())
    # the GPU solution solves the oracle's unreduced system
    chk = o.residual_check(solg)
    assert np.max(np.abs(chk[:3 * n])) <= 1e-9 * np.abs(o.system()[3]).max()


def test_bicgstab_iteration_limit_and_status():
    m, g, o = _pair("ragged_33x17x9", seed=2)
    g.assemble(synth.DAY)
    o.assemble(synth.DAY)
    stg, itg, _ = g.solve(tol=1e-14, maxit=3)
    sto, ito, _ = o.solve(tol=1e-14, maxit=3)
    assert stg == sto == 1 and itg == ito == 3


@pytest.mark.parametrize("name,steps,dt_days", [("small_5spot", 3, 2.0), ("gas_7x6x5", 3, 5.0),
                                                ("aniso_9x8x6", 3, 2.0), ("config0", 10, 30.0)])
def test_newton_steps_parity(name, steps, dt_days):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.init_hydrostatic()
    o.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10)
    for s in range(steps):
        stg, rg = g.step(dt_days * synth.DAY, **tight)
        sto, ro = o.step(dt_days * synth.DAY, **tight)
        assert stg == 0 and sto == 0, (s, rg, ro)
        pg, swg, xg, fg, bg = g.get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo), s
        assert np.max(np.abs(pg - po) / po) <= 1e-6, s
        assert np.max(np.abs(swg - swo)) <= 1e-6, s
        sat = fo == 0
        assert np.max(np.abs(xg[sat] - xo[sat]), initial=0.0) <= 1e-6, s
        assert np.max(np.abs(xg[~sat] - xo[~sat]) / xo[~sat].clip(1e-300), initial=0.0) <= 1e-6, s
        assert np.allclose(bg, bo, rtol=1e-6)


@pytest.mark.parametrize("name", ["small_5spot", "gas_7x6x5", "config0"])
def test_well_rates_parity(name):
    """Per-well surface rates (bo_get_well_rates): at an assembled state they
    match the oracle's to rounding (the connection terms match at 1e-12, the
    sums differ in order); after Newton steps at tight tolerances every
    rate-controlled well meets its target and the rates match the oracle's
    to the tolerance of the states (pressure 1e-6 relative, acting on
    drawdowns of about 1e-2 of the pressure)."""
    m, g, o = _pair(name, seed=4)
    dt = 2 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    qg, bg, cg = g.well_rates()
    qo, bo, co = o.well_rates()
    assert qg.shape == qo.shape == (len(m["wells"]), 3)
    assert np.array_equal(cg, co) and np.array_equal(bg, bo)
    for w in range(len(qo)):
        floor = 1e-3 * np.abs(qo[w]).max() + 1e-300
        assert np.all(np.abs(qg[w] - qo[w]) <= 1e-11 * np.maximum(np.abs(qo[w]), floor)), w
    g2, o2 = Sim(m), oracle.Oracle(m)
    g2.init_hydrostatic()
    o2.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10)
    for _ in range(2):
        stg, _ = g2.step(dt, **tight)
        sto, _ = o2.step(dt, **tight)
        assert stg == 0 and sto == 0
    qg, bg, cg = g2.well_rates()
    qo, bo, co = o2.well_rates()
    assert np.array_equal(cg, co)
    for w, well in enumerate(m["wells"]):
        if cg[w] == 0:   # rate control: the controlled surface rate meets its target
            a = 0 if well["phase"] == "water" else 2
            ctl = -qg[w, a] if well["kind"] == "inj" else qg[w, 1]
            assert abs(ctl - well["target"]) <= 1e-8 * well["target"], w
        floor = 1e-3 * np.abs(qo[w]).max() + 1e-300
        assert np.all(np.abs(qg[w] - qo[w]) <= 1e-3 * np.maximum(np.abs(qo[w]), floor)), w


def test_step_restores_state_on_failure():
    """A report step that cannot converge returns BO_ERR_NOT_CONVERGED and
    leaves the state exactly as it was (host-side fault injection: a
    one-iteration Newton budget with no cuts)."""
    m = MODELS["small_5spot"]()
    g = Sim(m)
    g.init_hydrostatic()
    before = g.get_state()
    st, rep = g.step(10 * synth.DAY, max_newton=0, max_cuts=0)
    assert st == 4
    after = g.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_full_size_config1_sampled_assembly_and_solve():
    """Config 1 at full size (1.12M cells): every residual entry and the
    Jacobian rows of sampled cells match the oracle; the GPU's linear
    solution at tol 1e-3 satisfies the oracle's own operator."""
    m = synth.config1()
    g, o = Sim(m), oracle.Oracle(m)
    st = synth.random_state(m, seed_member=1)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    st2 = (st[0] * 1.002, st[1] + 0.003, st[2], st[3], st[4])
    g.set_state(*st2)
    o.set_state(*st2)
    dt = 10 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    rpg, cig, vg, Rg = g.system()
    rpo, cio, vo, Ro = o.system()
    scale = np.maximum(np.abs(Ro), 1e-3 * np.abs(Ro).max(axis=0))
    assert np.max(np.abs(Rg - Ro) / scale) <= 1e-12
    rng = np.random.default_rng(5)
    cells = np.unique(np.concatenate([rng.choice(o.n, 4000, replace=False),
                                      np.concatenate(o.well_cells)]))
    idx = np.concatenate([np.arange(rpo[c], rpo[c + 1]) for c in cells])
    sub_rp = np.concatenate([[0], np.cumsum(rpo[cells + 1] - rpo[cells])])
    assert family_close(vg[idx], vo[idx], sub_rp) <= 1e-12
    # random states of this heterogeneous model give systems ILU0-BiCGStab
    # does not solve; the linear solve is checked on the physical initial state
    g.init_hydrostatic()
    o.init_hydrostatic()
    g.begin_step()
    o.begin_step()
    dt = 1.0 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    Ro = o.system()[3]
    stg, itg, solg = g.solve(tol=1e-3, maxit=500)
    assert stg == 0
    n = o.n
    b = Ro.reshape(-1).copy()
    # reduced right-hand side from the oracle's well terms
    for q, w in enumerate(o.wells()):
        if w["control"] == 0:
            for con, c in enumerate(o.well_cells[q]):
                b[3 * c:3 * c + 3] -= w["C"][con] * (w["Rw"] / w["Dw"])
    res = b - o.apply_op(solg[:3 * n])
    assert np.linalg.norm(res) <= 1.0001e-3 * np.linalg.norm(b)
