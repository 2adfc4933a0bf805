"""Mixed precision against the FP64 oracle (needs a GB300).

In mixed precision the ILU(0) factors are stored in FP32 and both
triangular sweeps run in FP32; assembly, the operator, the Krylov vectors,
the true-residual check and the Newton test stay FP64.

Tolerances:
  FP32 preconditioner apply vs the oracle's FP64 apply   1e-4 relative to the
      vector's max per unknown family, and at least 1e-9 (the FP32 sweeps ran)
  linear solve                                           the oracle's operator
      gives ||b - Op x|| <= tol ||b|| (FP64 true residual)
  Newton states (tight tolerances)                       pressure 1e-6 relative,
      saturations and r_go 1e-6 absolute / relative, as for the FP64 path
"""
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


def Sim(m, precision="mixed"):
    from paper_1910_06059_gb300 import Sim as _S
    s = _S(m)
    s.precision = precision
    return s


def vec_close(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


MODELS = {
    "small_5spot": lambda: synth.small_model(6, 5, 4, wells="5spot", dz=4.0),
    "ragged_33x17x9": lambda: synth.small_model(33, 17, 9, wells="5spot", dz=3.0),
    "gas_7x6x5": lambda: synth.small_model(7, 6, 5, wells="gas", dz=5.0),
    "config0": synth.config0,
}


def _pair(name, seed=0, precision="mixed"):
    m = MODELS[name]()
    g, o = Sim(m, precision), oracle.Oracle(m)
    st = synth.random_state(m, seed_member=seed, frac_sat=0.5)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    p, sw, x, fl, bhp = [a.copy() for a in st]
    st2 = (p * 1.003, sw + 0.004, x, fl, bhp)
    g.set_state(*st2)
    o.set_state(*st2)
    return m, g, o


def _reduced_rhs(o):
    b = o.system()[3].reshape(-1).copy()
    for q, w in enumerate(o.wells()):
        if w["control"] == 0:
            for con, c in enumerate(o.well_cells[q]):
                b[3 * c:3 * c + 3] -= w["C"][con] * (w["Rw"] / w["Dw"])
    return b


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9", "config0"])
def test_fp32_precond_apply_vs_oracle(name):
    m, g, o = _pair(name, seed=5)
    dt = 2 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    g.factor()
    o.ilu0()
    rng = np.random.default_rng(11)
    r = rng.standard_normal(3 * o.n)
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    errs = [vec_close(zg[v::3], zo[v::3]) for v in range(3)]
    assert max(errs) <= 1e-4, errs
    assert max(errs) >= 1e-9, errs   # FP32 rounding is visible: the FP32 sweeps ran


@pytest.mark.parametrize("name", ["ragged_33x17x9", "config0"])
def test_fp32_precond_apply_on_initial_residual(name):
    """The Newton residual at the undersaturated initial state: the pivot
    blocks are ill-conditioned there (pressure and r_go columns), so applying
    an FP32-rounded explicit D^-1 loses the small unknown families to
    cancellation.  Pressure and water saturation must match the FP64 oracle
    per family; the r_go family of the exact result is numerically zero here
    (all cells undersaturated, ~1e-12 against updates of order 1), so it is
    judged by its effect in the equations: the apply's error mapped through
    the operator must be small against the residual."""
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.init_hydrostatic()
    o.init_hydrostatic()
    g.begin_step()
    o.begin_step()
    dt = 0.1 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    g.factor()
    o.ilu0()
    r = o.system()[3].reshape(-1).copy()
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    errs = [vec_close(zg[v::3], zo[v::3]) for v in range(2)]
    assert max(errs) <= 1e-4, errs
    op_err = np.linalg.norm(o.apply_op(zg - zo)) / np.linalg.norm(r)
    assert op_err <= 1e-5, op_err


def test_precision_switch_keeps_fp64_path_bitwise():
    """FP64 -> mixed -> FP64 gives the same FP64 results bit for bit."""
    m, g, o = _pair("ragged_33x17x9", seed=3, precision="fp64")
    g.assemble(synth.DAY)
    g.factor()
    r = np.random.default_rng(2).standard_normal(3 * g.n)
    z64 = g.precond_apply(r)
    g.precision = "mixed"
    assert g.precision == "mixed"
    z32 = g.precond_apply(r)         # factors converted at the switch
    assert not np.array_equal(z32, z64)
    g.precision = "fp64"
    assert g.precision == "fp64"
    assert np.array_equal(g.precond_apply(r), z64)
    from paper_1910_06059_gb300 import _lib as L
    Lb = L.load()
    assert Lb.bo_set_precision(g.h, 7) == 1   # BO_ERR_INVALID_ARG


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9", "gas_7x6x5"])
def test_mixed_solve_true_residual(name):
    m, g, o = _pair(name, seed=7)
    dt = 0.1 * synth.DAY
    g.assemble(dt)
    o.assemble(dt)
    for tol in (1e-3, 1e-10):
        st, its, sol, rep = g.solve(tol=tol, maxit=500, report=True)
        assert st == 0, (tol, its, rep)
        assert rep["rel_res"] <= tol
        b = _reduced_rhs(o)
        res = b - o.apply_op(sol[:3 * o.n])
        assert np.linalg.norm(res) <= tol * (1 + 1e-6) * np.linalg.norm(b) + 1e-300


def test_failed_fp32_solve_is_repeated_with_fp64_sweeps():
    """A solve whose FP32 attempt runs out of iterations is repeated with the
    FP64 factors and sweeps (zero initial guess, a fresh iteration budget):
    it converges, reports fallback 2, and its solution is the FP64 solver's.
    The mixed solver afterwards gives its own result again (the face buffers
    are back in FP32)."""
    m = MODELS["ragged_33x17x9"]()
    g, h = Sim(m, "mixed"), Sim(m, "fp64")
    st = synth.random_state(m, seed_member=7, frac_sat=0.5)
    p, sw, x, fl, bhp = [a.copy() for a in st]
    for s in (g, h):
        s.set_state(*st)
        s.begin_step()
        s.set_state(p * 1.003, sw + 0.004, x, fl, bhp)
        s.assemble(0.1 * synth.DAY)
    tol = 1e-10
    s64, n64, x64, r64 = h.solve(tol=tol, maxit=500, report=True)
    s32, n32, x32, r32 = g.solve(tol=tol, maxit=500, report=True)
    assert s64 == 0 and s32 == 0 and r64["fallback"] == 0 and r32["fallback"] == 0
    if n32 <= n64:
        pytest.skip(f"the FP32 sweeps need no more iterations here ({n32} vs {n64})")
    sf, nf, xf, rf = g.solve(tol=tol, maxit=n64, report=True)
    assert sf == 0 and rf["fallback"] == 2 and rf["rel_res"] <= tol, (nf, rf)
    assert nf > n64
    assert vec_close(xf, x64) <= 1e-13
    s2, n2, x2, r2 = g.solve(tol=tol, maxit=500, report=True)
    assert s2 == 0 and r2["fallback"] == 0 and n2 == n32
    assert vec_close(x2, x32) <= 1e-13


# Report steps of growing length, each taken as one Newton solve (no adaptive
# sub-steps, no cuts), so both sides solve the same discrete equations and
# the comparison measures the precision of the solver alone.
SCHEDULE_DAYS = [0.01, 0.05, 0.2, 0.5, 1.0, 2.0]


@pytest.mark.parametrize("name", ["small_5spot", "gas_7x6x5", "config0"])
def test_mixed_newton_steps_vs_oracle(name):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.init_hydrostatic()
    o.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10, max_cuts=0)
    worst = 0.0
    for s, days in enumerate(SCHEDULE_DAYS):
        dt = days * synth.DAY
        g.dt_next = dt
        o.dt_next = dt
        stg, rg = g.step(dt, **tight)
        sto, ro = o.step(dt, **tight)
        assert stg == 0 and sto == 0, (s, rg, ro)
        assert rg["substeps"] == ro["substeps"] == 1
        pg, swg, xg, fg, bg = g.get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo), s
        err_p = np.max(np.abs(pg - po) / po)
        err_s = np.max(np.abs(swg - swo))
        sat = fo == 0
        err_x = max(np.max(np.abs(xg[sat] - xo[sat]), initial=0.0),
                    np.max(np.abs(xg[~sat] - xo[~sat]) / xo[~sat].clip(1e-300), initial=0.0))
        assert err_p <= 1e-6 and err_s <= 1e-6 and err_x <= 1e-6, (s, err_p, err_s, err_x)
        assert np.allclose(bg, bo, rtol=1e-6)
        worst = max(worst, err_p, err_s, err_x)
    print(f"{name}: largest state error of the mixed-precision path vs the FP64 oracle {worst:.2e}")


def test_mixed_vs_fp64_on_grf_100x100x50():
    """The 100x100x50 Gaussian-random-field model at full size: report steps
    taken as single Newton solves at tight tolerances reach the same state in
    both precisions.  The steps stay short (the first hours of depletion below
    the bubble point), where one Newton solve per step converges in FP64."""
    m = synth.config2()
    states = {}
    for prec in ("fp64", "mixed"):
        g = Sim(m, prec)
        g.init_hydrostatic()
        for days in (0.01, 0.02, 0.04):
            g.dt_next = days * synth.DAY
            st, rep = g.step(days * synth.DAY, tol_mb=1e-9, tol_cnv=1e-9, tol_well=1e-9,
                             tol_lin=1e-8, max_cuts=0)
            assert st == 0 and rep["substeps"] == 1, (prec, days, rep)
        states[prec] = g.get_state()
        g.close()
    p64, sw64, x64, f64, b64 = states["fp64"]
    p32, sw32, x32, f32, b32 = states["mixed"]
    assert np.max(np.abs(p32 - p64) / p64) <= 1e-6
    assert np.max(np.abs(sw32 - sw64)) <= 1e-6
    same = f64 == f32
    assert same.mean() > 0.999
    sat = same & (f64 == 0)
    assert np.max(np.abs(x32[sat] - x64[sat]), initial=0.0) <= 1e-6
