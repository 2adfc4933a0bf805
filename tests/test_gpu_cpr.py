"""CPR two-stage preconditioner on the GPU against the CPU oracle
(oracle/cpr.py; Section 2.3.1: CPR with algebraic multigrid for the pressure
for large cases).  Needs a GB300.

  aggregation hierarchy            identical integer maps
  quasi-IMPES weights, A_p         1e-12 relative per entry (floor: 1e-3 of the
                                   cell's largest entry)
  one V-cycle                      1e-10 relative to the vector's max
  two-stage apply                  1e-9 relative to the vector's max, per family:
                                   the V-cycle's difference carried through
                                   S and the ILU(0) stage (whose own apply
                                   differs by up to 1e-10 on these
                                   conditionings, see test_gpu_subdomains.py)
  linear solve                     converges; the solution solves the oracle's system
  Newton states (tight)            pressure 1e-6 relative, saturations 1e-6 absolute
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import vec_close
from oracle.cpr import (AMG, CPR, diagonal_blocks, pressure_matrix, quasi_impes_weights,
                        transmissibility_laplacian)

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
    "layered_20x30x20": lambda: synth.layered_model(20, 30, 20, config=1, name="layered 20x30x20"),
    "ragged_33x17x9": lambda: synth.small_model(33, 17, 9, wells="5spot", dz=3.0),
}


def _oracle_hierarchy(o):
    st = o.static()
    L = transmissibility_laplacian(st["Tx"], st["Ty"], st["Tz"], o.nx, o.ny, o.nz)
    return AMG(L).P


def _maps(Ps):
    return [np.asarray(P.tocsr().indices, dtype=np.int64) for P in Ps]


@pytest.fixture(scope="module", params=list(MODELS))
def system(request):
    """GPU and oracle at the same assembled state (hydrostatic start, a
    10-day step: the wells' pressure pulse), CPR factorised on the GPU."""
    m = MODELS[request.param]()
    g, o = Sim(m), oracle.Oracle(m)
    g.preconditioner = "cpr"
    o.init_hydrostatic()
    st = o.get_state()
    g.set_state(*st)
    for s in (g, o):
        s.begin_step()
        s.assemble(10 * synth.DAY)
    g.factor()
    o.ilu0()
    rp, ci, vals, _ = o.system()
    Ps = _oracle_hierarchy(o)
    yield request.param, m, g, o, (rp, ci, vals), Ps
    g.close()


def test_cpr_hierarchy_matches_the_oracle(system):
    name, m, g, o, _, Ps = system
    sizes, maps = g.cpr_hierarchy()
    om = _maps(Ps)
    assert sizes[0] == o.n
    assert len(maps) == len(om), (sizes, [len(x) for x in om])
    for l, (a, b) in enumerate(zip(maps, om)):
        assert np.array_equal(a, b), l
    assert sizes[-1] <= 200 or len(sizes) == 12


def test_cpr_weights_and_pressure_matrix(system):
    name, m, g, o, (rp, ci, vals), _ = system
    w_g, ap_g = g.cpr_pressure_system()
    w_o = quasi_impes_weights(diagonal_blocks(rp, ci, vals))
    floor = 1e-3 * np.abs(w_o).max(axis=1, keepdims=True)
    assert np.max(np.abs(w_g - w_o) / np.maximum(np.abs(w_o), floor)) <= 1e-12
    Ap = pressure_matrix(rp, ci, vals, w_o).tocsr()
    n, nx, ny = o.n, m["nx"], m["ny"]
    ap_o = np.zeros((n, 7))
    offs = {0: 0, -1: 1, 1: 2, -nx: 3, nx: 4, -nx * ny: 5, nx * ny: 6}
    for c in range(n):
        for q in range(Ap.indptr[c], Ap.indptr[c + 1]):
            ap_o[c, offs[Ap.indices[q] - c]] = Ap.data[q]
    floor = 1e-3 * np.abs(ap_o).max(axis=1, keepdims=True)
    assert np.max(np.abs(ap_g - ap_o) / np.maximum(np.abs(ap_o), floor)) <= 1e-12


def _fixed_amg(rp, ci, vals, Ps):
    w = quasi_impes_weights(diagonal_blocks(rp, ci, vals))
    return AMG(pressure_matrix(rp, ci, vals, w), prolongators=Ps)


def test_cpr_vcycle_matches_the_oracle(system):
    name, m, g, o, (rp, ci, vals), Ps = system
    b = np.random.default_rng(41).standard_normal(o.n)
    xg = g.cpr_vcycle(b)
    xo = _fixed_amg(rp, ci, vals, Ps).vcycle(b)
    assert vec_close(xg, xo) <= 1e-10


def test_cpr_two_stage_apply_matches_the_oracle(system):
    name, m, g, o, (rp, ci, vals), Ps = system
    fixed = _fixed_amg(rp, ci, vals, Ps)
    cpr = CPR(rp, ci, vals, o.apply_op, o.ilu_apply, pressure_solve=fixed.vcycle)
    r = np.random.default_rng(43).standard_normal(3 * o.n) * np.tile([1.0, 1e-3, 1e-2], o.n)
    zg = g.precond_apply(r)
    zo = cpr(r)
    for v in range(3):
        assert vec_close(zg[v::3], zo[v::3]) <= 1e-9, v


def test_cpr_solve_reaches_the_oracle_system(system):
    """BiCGStab with CPR on the GPU converges in far fewer iterations than
    with ILU(0), and its solution solves the oracle's well-coupled system."""
    name, m, g, o, (rp, ci, vals), Ps = system
    st, its_cpr, sol = g.solve(tol=1e-8, maxit=500)
    assert st == 0
    chk = o.residual_check(sol)
    assert np.max(np.abs(chk[:3 * o.n])) <= 1e-6 * np.abs(o.system()[3]).max()
    g.preconditioner = "ilu0"
    g.factor()
    st2, its_ilu, _ = g.solve(tol=1e-8, maxit=500)
    g.preconditioner = "cpr"
    g.factor()
    print(f"{name}: BiCGStab iterations to 1e-8, CPR {its_cpr}, ILU(0) {its_ilu}")
    assert st2 != 0 or its_cpr < its_ilu


def test_cpr_newton_states_match_the_oracle():
    """Report steps with CPR on the GPU against the oracle's Newton with
    ILU(0), both at tight tolerances: the preconditioner changes the path of
    the linear solves, not the converged Newton states."""
    m = synth.small_model(7, 6, 5, wells="gas", dz=5.0)
    g, o = Sim(m), oracle.Oracle(m)
    g.preconditioner = "cpr"
    g.init_hydrostatic()
    o.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10)
    for s in range(3):
        stg, rg = g.step(5 * synth.DAY, **tight)
        sto, ro = o.step(5 * synth.DAY, **tight)
        assert stg == 0 and sto == 0, (s, rg, ro)
        pg, swg, xg, fg, bg = g.get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo), s
        assert np.max(np.abs(pg - po) / po) <= 1e-6, s
        assert np.max(np.abs(swg - swo)) <= 1e-6, s
        sat = fo == 0
        assert np.max(np.abs(xg[sat] - xo[sat]), initial=0.0) <= 1e-6, s
    g.close()
