"""Pins of the oracle's domain-decomposed solve (Section 2.5: one host
thread per subdomain -- the y slabs of the block-Jacobi preconditioner --
with its own rows, its own ILU(0) block, a halo exchange before every
operator product and all-reduced inner products).

With one subdomain the decomposed solve must be the single-domain solve bit
for bit (the same arithmetic in the same order: a plausible mistake in the
local numbering, the local factorisation or the well terms breaks it).  With
K > 1 subdomains only the grouping of the inner products' sums differs, so
the decomposed solve must reach the tolerance in about as many iterations
and must solve the same unreduced system (a missing or misplaced halo row,
or a partial sum left out of an all-reduce, does not)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth


def _system(m, dt_days=1.0):
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.begin_step()
    o.assemble(dt_days * synth.DAY)
    return o


MODELS = {
    "layered_12x32x6": lambda: synth.layered_model(12, 32, 6, config=1),
    "ragged_11x27x5": lambda: synth.small_model(11, 27, 5, wells="5spot", dz=3.0),
}


@pytest.mark.parametrize("name", list(MODELS))
def test_one_subdomain_is_the_single_domain_solve(name):
    m = MODELS[name]()
    o = _system(m)
    o.set_subdomains(m["ny"], 0)   # one slab: no cut
    s1, i1, x1 = o.solve(tol=1e-10, maxit=500)
    s2, i2, x2 = o.dd_solve(tol=1e-10, maxit=500)
    assert s1 == s2 == 0 and i1 == i2
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("ysub", [8, 16])
def test_subdomains_solve_the_same_system(name, ysub):
    m = MODELS[name]()
    o = _system(m)
    o.set_subdomains(ysub, 0)
    s1, i1, x1 = o.solve(tol=1e-10, maxit=500)
    s2, i2, x2 = o.dd_solve(tol=1e-10, maxit=500)
    assert s1 == s2 == 0
    assert abs(i1 - i2) <= max(3, 0.15 * i1), (i1, i2)
    n = o.n
    R = o.system()[3]
    for x in (x1, x2):
        chk = o.residual_check(x)
        assert np.max(np.abs(chk[:3 * n])) <= 1e-8 * np.abs(R).max()
    # the pressure updates, the best-determined family, agree closely
    assert np.abs(x1[0:3 * n:3] - x2[0:3 * n:3]).max() <= 1e-6 * np.abs(x1[0:3 * n:3]).max()
