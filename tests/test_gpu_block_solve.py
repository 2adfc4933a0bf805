"""The one-CTA linear solve (BO_SCHEDULE_BLOCK) against the oracle (needs a GB300).

Section 2.3.1's ILU0-BiCGStab run as ONE launch of ONE CTA: the triangular
sweeps by levels i + j + k inside the CTA, the reduced operator, the dot
products and the recurrence with its true-residual checks.  Bars as for the
tiled schedule:
  preconditioner apply            1e-11 relative to the vector's max (oracle ilu_apply)
  linear solution (tight solve)   1e-9 relative per unknown family
  Newton states                   pressure 1e-6 relative, saturations 1e-6 absolute
and against the tiled schedule on the same factorisation: applies 1e-12 (the
two differ only in the order of the FP64 operations), iteration counts within
rounding drift.  Members of an ensemble on the block schedule reach exactly
the states they reach alone.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth
from helpers import vec_close

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
    "no_wells_11x9x7": lambda: synth.small_model(11, 9, 7, wells="none", dz=3.0),
    "thin_40x3x2": lambda: synth.small_model(40, 3, 2, wells="none", dz=3.0),
    "gas_7x6x5": lambda: synth.small_model(7, 6, 5, wells="gas", dz=5.0),
    "config0": synth.config0,
    # 20 tiles (5 x 4) over 8 warps: several tiles per warp and level
    "ragged_21x37x13": lambda: synth.small_model(21, 37, 13, wells="5spot", dz=3.0),
    # 32 tiles, the largest ensemble member's tiling: a 48 KB ring (shared-memory opt-in)
    "tiles32_6x64x16": lambda: synth.small_model(6, 64, 16, wells="5spot", dz=3.0),
}


def _pair(name, seed=0):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    st = synth.random_state(m, seed_member=seed, frac_sat=0.5)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    p, sw, x, fl, bhp = [a.copy() for a in st]
    st2 = (p * 1.003, sw + 0.004, x, fl, bhp)
    g.set_state(*st2)
    o.set_state(*st2)
    g.solve_schedule = "block"
    return m, g, o


@pytest.mark.parametrize("name", list(MODELS))
def test_block_precond_apply_parity(name):
    m, g, o = _pair(name, seed=5)
    dt = 2 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    g.factor()
    o.ilu0()
    rng = np.random.default_rng(11)
    r = rng.standard_normal(3 * o.n)
    zb, zo = g.precond_apply(r), o.ilu_apply(r)
    for v in range(3):
        assert vec_close(zb[v::3], zo[v::3]) <= 1e-11, v
    g.solve_schedule = "tiled"
    zt = g.precond_apply(r)
    for v in range(3):
        assert vec_close(zb[v::3], zt[v::3]) <= 1e-12, v
    assert np.all(np.isfinite(zb))


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9", "gas_7x6x5", "no_wells_11x9x7",
                                  "ragged_21x37x13"])
def test_block_solution_parity(name):
    m, g, o = _pair(name, seed=7)
    dt = 0.1 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    stg, itg, solg = g.solve(tol=1e-12, maxit=500)
    sto, ito, solo = o.solve(tol=1e-12, maxit=500)
    assert stg == 0 and sto == 0
    assert abs(itg - ito) <= max(2, 0.05 * ito)
    n = o.n
    # the error of a solve to a 1e-12 relative residual grows with the
    # condition number: the 10k-cell model gets a wider bar than the others
    bar = 5e-9 if n > 5000 else 1e-9
    for v in range(3):
        assert vec_close(solg[v:3 * n:3], solo[v:3 * n:3]) <= bar
    if len(solo) > 3 * n:
        assert np.allclose(solg[3 * n:], solo[3 * n:], rtol=1e-9,
                           atol=1e-9 * np.abs(solo[3 * n:]).max())
    chk = o.residual_check(solg)
    assert np.max(np.abs(chk[:3 * n])) <= 1e-9 * np.abs(o.system()[3]).max()


def test_block_solve_equals_tiled_solve_to_rounding():
    # a short step keeps the random state's system well conditioned (as in
    # the tiled schedule's solution test)
    m, g, o = _pair("ragged_33x17x9", seed=3)
    g.assemble(0.1 * synth.DAY)
    # Both solve to a 1e-12 relative residual.  Two such solutions differ by
    # up to the condition number times that (measured here: 2.6e-9 of the
    # family maximum on this system), so what must agree is that each solves
    # the oracle's unreduced system; the solutions themselves agree to 1e-7.
    o.assemble(0.1 * synth.DAY)
    stb, itb, solb, rep_b = g.solve(tol=1e-12, maxit=500, report=True)
    g.solve_schedule = "tiled"
    stt, itt, solt, rep_t = g.solve(tol=1e-12, maxit=500, report=True)
    assert stb == stt == 0, (stb, itb, rep_b, stt, itt, rep_t)
    assert abs(itb - itt) <= max(2, 0.05 * itt)
    assert rep_b["rel_res"] <= 1e-12 and rep_t["rel_res"] <= 1e-12
    n = o.n
    scale = np.abs(o.system()[3]).max()
    for sol in (solb, solt):
        assert np.max(np.abs(o.residual_check(sol)[:3 * n])) <= 1e-9 * scale
    for v in range(3):
        assert vec_close(solb[v:3 * n:3], solt[v:3 * n:3]) <= 1e-7


def test_block_iteration_limit_and_status():
    m, g, o = _pair("ragged_33x17x9", seed=2)
    g.assemble(synth.DAY)
    o.assemble(synth.DAY)
    stg, itg, _ = g.solve(tol=1e-14, maxit=3)
    sto, ito, _ = o.solve(tol=1e-14, maxit=3)
    assert stg == sto == 1 and itg == ito == 3


def test_block_schedule_is_one_launch_per_solve():
    """Between assembly and the solution's well recovery the block schedule
    launches the reduced right-hand side (a copy and the well rows) and ONE
    solver kernel; the timers show the block solve and no tiled sweep."""
    m, g, o = _pair("small_5spot", seed=4)
    g.set_timing(True)
    g.assemble(0.1 * synth.DAY)
    g.factor()
    before = g.launches
    st, its, _ = g.solve(tol=1e-8, maxit=200)
    after = g.launches
    assert st == 0 and its > 3
    # bo_solve factors again (a graph of a few kernels), then copy + wells +
    # the block kernel, then the well recovery: far fewer than one tiled iteration's
    assert after - before <= 12, after - before
    names = g.timing()
    assert "block_bicgstab" in names
    assert "ilu_fwd_sweep" not in names


@pytest.mark.parametrize("name,steps,dt_days", [("small_5spot", 3, 2.0), ("gas_7x6x5", 3, 5.0),
                                                ("config0", 6, 30.0)])
def test_block_newton_steps_parity(name, steps, dt_days):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.solve_schedule = "block"
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


def test_block_schedule_keeps_tiled_path_where_it_does_not_apply():
    """With CPR selected the block schedule does not apply: the solve runs the
    tiled two-stage path (its timer, not the block solver's) and reaches the
    same state as a run that never asked for the block schedule."""
    m = MODELS["ragged_33x17x9"]()
    a, b = Sim(m), Sim(m)
    for s in (a, b):
        s.init_hydrostatic()
        s.preconditioner = "cpr"
        s.set_timing(True)
    a.solve_schedule = "block"
    assert a.solve_schedule == "block"
    for s in (a, b):
        st, rep = s.step(2 * synth.DAY)
        assert st == 0
    names = a.timing()
    assert "cpr_apply" in names and "block_bicgstab" not in names
    pa, swa = a.get_state()[:2]
    pb, swb = b.get_state()[:2]
    assert np.max(np.abs(pa - pb) / pb) <= 1e-9
    assert np.max(np.abs(swa - swb)) <= 1e-9


def small_members(k=6, pool=40):
    ms = [synth.config3_member(q) for q in range(pool)]
    ms.sort(key=lambda m: m["nx"] * m["ny"] * m["nz"])
    return ms[:k]


def test_block_ensemble_equals_members_alone_and_oracle():
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(6)
    ens = Ensemble(models, streams=6)
    for s in ens.members:
        s.solve_schedule = "block"
    ens.init_hydrostatic()
    alone = [Sim(m) for m in models]
    for s in alone:
        s.solve_schedule = "block"
        s.init_hydrostatic()
    orc = oracle.Oracle(models[0])
    orc.init_hydrostatic()
    for days in (1.0, 3.0):
        sts, reps = ens.step(days * synth.DAY)
        assert all(st == 0 for st in sts)
        for q, s in enumerate(alone):
            st, rep = s.step(days * synth.DAY)
            assert st == 0
            assert (rep["newton_its"], rep["lin_its"]) == (reps[q]["newton_its"], reps[q]["lin_its"])
            for u, w in zip(s.get_state(), ens.members[q].get_state()):
                assert np.array_equal(u, w)
        sto, _ = orc.step(days * synth.DAY)
        assert sto == 0
        pg, swg = ens.members[0].get_state()[:2]
        po, swo = orc.get_state()[:2]
        assert np.max(np.abs(pg - po) / po) <= 1e-6
        assert np.max(np.abs(swg - swo)) <= 1e-6


def test_autotune_schedule_restores_and_applies_choice():
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(8)
    ens = Ensemble(models, streams=2)
    ens.init_hydrostatic()
    before = [s.get_state() for s in ens.members]
    t0 = time.perf_counter()
    res = ens.autotune_schedule(0.2 * synth.DAY)
    assert time.perf_counter() - t0 > 0.0
    assert len(res["probe_s"]) == 4 and all(v > 0 for v in res["probe_s"].values())
    assert res["chosen"]["small"] in ("tiled", "block")
    assert res["chosen"]["streams"] in (2, 8)
    assert ens.schedule["streams"] == res["chosen"]["streams"]
    for s, st in zip(ens.members, before):
        for u, w in zip(s.get_state(), st):
            assert np.array_equal(u, w)
    sizes = [m["nx"] * m["ny"] * m["nz"] for m in models]
    med = sorted(sizes)[(len(sizes) - 1) // 2]
    for s, n in zip(ens.members, sizes):
        assert s.solve_schedule == (res["chosen"]["small"] if n <= med else "tiled")
    sts, _ = ens.step(1.0 * synth.DAY)
    assert all(st == 0 for st in sts)
