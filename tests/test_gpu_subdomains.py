"""Block-Jacobi ILU(0) over slabs in y, in z and boxes of both
(bo_set_subdomains) against the oracle's block-Jacobi ILU(0)
(orc_set_subdomains), through the C ABI.

Bars: applies at 1e-10 relative (FP64), FP32 applies at 1e-4, Newton states
at 1e-6 with tight tolerances, pivot inverses at 1e-8.  The pivot blocks of
these random states have Skeel condition numbers |D^-1||D| up to ~1e7, so
two FP64 computations of D^-1 that sum in different orders (the GPU's fused
wavefront and the oracle's natural-order elimination) may differ by about
cond x 1.1e-16 ~ 1e-9 relative in an entry; measured 4.4e-10 on the 33x17x9
model.  The applies carry those differences through the two triangular
sweeps: measured up to 1.1e-11 of the vector's largest entry (16x24x13
boxes); a dropped or misplaced coupling block gives errors of order one."""
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


MODELS = {
    # ny = 17: slabs of 8, 8, 1 rows (a ragged last slab and a ragged last tile)
    "ragged_33x17x9": (lambda: synth.small_model(33, 17, 9, wells="5spot", dz=3.0), (8, 0)),
    # ny = 40: slabs of 16, 16, 8 rows, two tiles per slab
    "slabs_12x40x6": (lambda: synth.small_model(12, 40, 6, wells="5spot", dz=3.0), (16, 0)),
    # nz = 22: slabs of 8, 8, 6 layers in z, a ragged last tile (2 of 4 layers)
    "zslabs_20x9x22": (lambda: synth.small_model(20, 9, 22, wells="5spot", dz=2.0), (0, 8)),
    # boxes: 3 slabs in y times 4 in z (4, 4, 4, 1 layers: a one-layer slab)
    "boxes_16x24x13": (lambda: synth.small_model(16, 24, 13, wells="5spot", dz=2.0), (8, 4)),
}


def _box(m, sub):
    """Subdomain index of every cell (natural order) for slab heights sub."""
    c = np.arange(m["nx"] * m["ny"] * m["nz"])
    j, k = (c // m["nx"]) % m["ny"], c // (m["nx"] * m["ny"])
    sy = j // sub[0] if sub[0] else 0 * j
    sz = k // sub[1] if sub[1] else 0 * k
    return sy + m["ny"] * sz


def _pair(name, seed=5, dt_days=2.0, precision="fp64"):
    from paper_1910_06059_gb300 import Sim
    mk, sub = MODELS[name]
    m = mk()
    g, o = Sim(m), oracle.Oracle(m)
    g.precision = precision
    g.subdomains, g.subdomains_z = sub
    o.set_subdomains(*sub)
    st = synth.random_state(m, seed_member=seed, frac_sat=0.5)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    g.assemble(dt_days * synth.DAY)
    o.assemble(dt_days * synth.DAY)
    return m, g, o, sub


@pytest.mark.parametrize("name", list(MODELS))
def test_block_jacobi_factors_and_apply(name):
    m, g, o, sub = _pair(name)
    assert (g.subdomains, g.subdomains_z) == sub
    dinv = g.factor()
    lu, uinv = o.ilu0()
    assert family_close(dinv, uinv, np.arange(o.n + 1), per_equation=False) <= 1e-8
    r = np.random.default_rng(11).standard_normal(3 * o.n)
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    for v in range(3):
        assert vec_close(zg[v::3], zo[v::3]) <= 1e-10
    # a residual on one subdomain (the second slab, or the second box) stays there
    box = _box(m, sub)
    mid = box == np.unique(box)[1]
    r2 = (r.reshape(-1, 3) * mid[:, None]).reshape(-1)
    z2 = g.precond_apply(r2).reshape(-1, 3)
    assert np.all(z2[~mid] == 0.0) and np.abs(z2[mid]).max() > 0


@pytest.mark.parametrize("name", list(MODELS))
def test_block_jacobi_fp32_apply(name):
    m, g, o, sub = _pair(name, precision="mixed")
    g.factor()
    o.ilu0()
    r = np.random.default_rng(12).standard_normal(3 * o.n)
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    errs = [vec_close(zg[v::3], zo[v::3]) for v in range(3)]
    assert max(errs) <= 1e-4, errs


def test_switching_back_to_one_domain():
    m, g, o, sub = _pair("boxes_16x24x13")
    g.factor()
    g.subdomains, g.subdomains_z = 0, 0
    o.set_subdomains(0, 0)
    dinv = g.factor()
    lu, uinv = o.ilu0()
    assert family_close(dinv, uinv, np.arange(o.n + 1), per_equation=False) <= 1e-8
    r = np.random.default_rng(3).standard_normal(3 * o.n)
    zg, zo = g.precond_apply(r), o.ilu_apply(r)
    for v in range(3):
        assert vec_close(zg[v::3], zo[v::3]) <= 1e-10
    from paper_1910_06059_gb300 import _lib as L
    assert L.load().bo_set_subdomains(g.h, 12, 0) == 1   # not a multiple of 8
    assert L.load().bo_set_subdomains(g.h, 8, 6) == 1    # not a multiple of 4
    assert (g.subdomains, g.subdomains_z) == (0, 0)


@pytest.mark.parametrize("name", list(MODELS))
def test_newton_steps_with_block_jacobi(name):
    from paper_1910_06059_gb300 import Sim
    mk, sub = MODELS[name]
    m = mk()
    g, o = Sim(m), oracle.Oracle(m)
    g.subdomains, g.subdomains_z = sub
    o.set_subdomains(*sub)
    g.init_hydrostatic()
    o.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10, max_cuts=0)
    for days in (0.01, 0.05, 0.2, 1.0):
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
