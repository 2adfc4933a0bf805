"""Pins of the CPR oracle (oracle/cpr.py), the two-stage preconditioner that
Section 2.3.1 names for large cases: quasi-IMPES decoupling, the pressure
matrix, the aggregation AMG and the two-stage composition, each against a
property the mathematics fixes; and its effect on BiCGStab on a Newton system
of the layered workload's generator."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from helpers import bcsr_to_dense
from oracle.cpr import (AMG, CPR, aggregate, bicgstab, diagonal_blocks, pressure_matrix,
                        quasi_impes_weights, strength, transmissibility_laplacian)


def _reduced_rhs(o):
    b = o.system()[3].reshape(-1).copy()
    for q, w in enumerate(o.wells()):
        if w["control"] == 0:
            for con, c in enumerate(o.well_cells[q]):
                b[3 * c:3 * c + 3] -= w["C"][con] * (w["Rw"] / w["Dw"])
    return b


@pytest.fixture(scope="module")
def small_system():
    """A Newton system of a small lognormal model at a random SAT/USAT state."""
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    o = oracle.Oracle(m)
    o.set_state(*synth.random_state(m, seed_member=2, frac_sat=0.5))
    o.begin_step()
    o.assemble(2 * synth.DAY)
    rp, ci, vals, _ = o.system()
    return o, rp, ci, vals


@pytest.fixture(scope="module")
def layered_system():
    """The first Newton system of a 20x30x20 model of the layered generator
    from its hydrostatic state (a 10-day step: the wells' pressure pulse)."""
    m = synth.layered_model(20, 30, 20, config=1, name="layered 20x30x20")
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.begin_step()
    o.assemble(10 * synth.DAY)
    o.ilu0()
    rp, ci, vals, _ = o.system()
    return o, rp, ci, vals


def _aniso_laplacian(nx, ny, nz, ax, ay, az):
    """7-point finite-difference Laplacian with Dirichlet ends (SPD M-matrix)."""
    def d1(k, a):
        return a * sp.diags([-np.ones(k - 1), 2 * np.ones(k), -np.ones(k - 1)], [-1, 0, 1])
    ix, iy, iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(iz, sp.kron(iy, d1(nx, ax))) + sp.kron(iz, sp.kron(d1(ny, ay), ix))
            + sp.kron(d1(nz, az), sp.kron(iy, ix))).tocsr()


def test_quasi_impes_weights_decouple_the_diagonal_block(small_system):
    o, rp, ci, vals = small_system
    D = diagonal_blocks(rp, ci, vals)
    w = quasi_impes_weights(D)
    wd = np.einsum("ce,cev->cv", w, D)
    assert np.allclose(wd[:, 0], 1.0, rtol=0, atol=1e-12)
    scale = np.abs(w[:, :, None] * D).max(axis=(1, 2))
    assert np.all(np.abs(wd[:, 1:]) <= 1e-12 * scale[:, None])


def test_pressure_matrix_is_the_weighted_pressure_column(small_system):
    """A_p = W^T A E_p, checked against the dense Jacobian."""
    o, rp, ci, vals = small_system
    w = quasi_impes_weights(diagonal_blocks(rp, ci, vals))
    Ap = pressure_matrix(rp, ci, vals, w).toarray()
    A = bcsr_to_dense(rp, ci, vals, o.n)
    W = np.zeros((o.n, 3 * o.n))
    for c in range(o.n):
        W[c, 3 * c:3 * c + 3] = w[c]
    Ep = np.zeros((3 * o.n, o.n))
    Ep[3 * np.arange(o.n), np.arange(o.n)] = 1.0
    ref = W @ A @ Ep
    assert np.allclose(Ap, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_amg_on_an_anisotropic_laplacian():
    """On an SPD M-matrix (the textbook case, strong coupling in z) the
    V-cycle contracts the error, and as a BiCGStab preconditioner it reaches
    the direct solution."""
    A = _aniso_laplacian(16, 20, 12, 1.0, 4.0, 100.0)
    amg = AMG(A)
    assert len(amg.A) >= 3 and amg.A[-1].shape[0] <= 200
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    x = np.zeros_like(b)
    res = [np.linalg.norm(b)]
    for _ in range(10):
        x = x + amg.vcycle(b - A @ x)
        res.append(np.linalg.norm(b - A @ x))
    assert res[-1] / res[0] <= 0.9 ** 10, res
    x, its, ok = bicgstab(lambda v: A @ v, b, amg.vcycle, tol=1e-11, maxit=200)
    xd = spla.spsolve(A.tocsc(), b)
    assert ok and np.allclose(x, xd, rtol=1e-8, atol=1e-8 * np.abs(xd).max()), its


def test_aggregation_keeps_coarse_operators_diagonally_dominant(layered_system):
    """Plain aggregation of a matrix with positive diagonal, non-positive
    off-diagonals and non-negative row sums keeps all three properties on
    every coarse level (sums of rows over an aggregate)."""
    o, rp, ci, vals = layered_system
    Ap = pressure_matrix(rp, ci, vals, quasi_impes_weights(diagonal_blocks(rp, ci, vals)))
    off = Ap - sp.diags(Ap.diagonal())
    rs = np.asarray(Ap.sum(axis=1)).ravel()
    assert off.data.max() <= 0 and rs.min() >= -1e-4 * Ap.diagonal().max()
    amg = AMG(Ap)
    for Al in amg.A[1:]:
        d = Al.diagonal()
        offl = (Al - sp.diags(d)).tocsr()
        offl.eliminate_zeros()
        rsl = np.asarray(Al.sum(axis=1)).ravel()
        assert d.min() > 0
        assert offl.data.max() <= 1e-12 * d.max()
        assert rsl.min() >= -1e-4 * d.max()
    # every node in exactly one aggregate, aggregate indices contiguous
    agg = aggregate(strength(Ap, 0.25))
    assert agg.min() == 0 and len(np.unique(agg)) == agg.max() + 1


def test_exact_second_stage_makes_the_two_stage_method_exact(small_system):
    """x1 + S^-1 (r - S x1) = S^-1 r whatever the first stage gives."""
    o, rp, ci, vals = small_system
    A = bcsr_to_dense(rp, ci, vals, o.n)
    cpr = CPR(rp, ci, vals, lambda v: A @ v, lambda v: np.linalg.solve(A, v))
    r = np.random.default_rng(3).standard_normal(3 * o.n)
    z = cpr(r)
    ref = np.linalg.solve(A, r)
    assert np.allclose(z, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
    assert np.abs(cpr.first_stage(r)).max() > 0


def test_exact_pressure_stage_clears_the_weighted_residual(small_system):
    """With an exact pressure solve, the residual after the first stage has
    no weighted pressure component: w_c^T (r - A x1)_c = 0 for every cell."""
    o, rp, ci, vals = small_system
    A = bcsr_to_dense(rp, ci, vals, o.n)
    w = quasi_impes_weights(diagonal_blocks(rp, ci, vals))
    lu = spla.splu(pressure_matrix(rp, ci, vals, w).tocsc())
    cpr = CPR(rp, ci, vals, lambda v: A @ v, lambda v: v, pressure_solve=lu.solve)
    r = np.random.default_rng(4).standard_normal(3 * o.n)
    r2 = (r - A @ cpr.first_stage(r)).reshape(-1, 3)
    rp_ = np.einsum("ce,ce->c", w, r.reshape(-1, 3))
    assert np.abs(np.einsum("ce,ce->c", w, r2)).max() <= 1e-10 * np.abs(rp_).max()


def test_cpr_cuts_bicgstab_iterations_on_the_layered_pressure_pulse(layered_system):
    """On the first Newton system of the layered generator (dominated by the
    wells' pressure pulse) CPR with one AMG V-cycle needs a small fraction of
    ILU(0)'s BiCGStab iterations; both solutions meet the tolerance."""
    o, rp, ci, vals = layered_system
    b = _reduced_rhs(o)
    op = o.apply_op
    x0, n_ilu, ok0 = bicgstab(op, b, o.ilu_apply, tol=1e-3, maxit=2000)
    x1, n_cpr, ok1 = bicgstab(op, b, CPR(rp, ci, vals, op, o.ilu_apply), tol=1e-3, maxit=2000)
    print(f"BiCGStab iterations at 1e-3: ILU(0) {n_ilu}, CPR {n_cpr}")
    assert ok0 and ok1
    for x in (x0, x1):
        assert np.linalg.norm(b - op(x)) <= 1.01e-3 * np.linalg.norm(b)
    assert n_cpr * 4 <= n_ilu


def test_fixed_hierarchy_from_the_transmissibilities(layered_system):
    """Aggregates built once from the transmissibility Laplacian carry each
    Newton system's pressure matrix: the Galerkin coarse operators of a
    piecewise-constant P keep aggregated row sums, (P^T A P) 1 = P^T (A 1),
    and CPR with that fixed hierarchy still needs a small fraction of
    ILU(0)'s iterations on the pressure pulse."""
    o, rp, ci, vals = layered_system
    st = o.static()
    L = transmissibility_laplacian(st["Tx"], st["Ty"], st["Tz"], o.nx, o.ny, o.nz)
    Ps = AMG(L).P
    assert len(Ps) >= 2
    Ap = pressure_matrix(rp, ci, vals, quasi_impes_weights(diagonal_blocks(rp, ci, vals)))
    fixed = AMG(Ap, prolongators=Ps)
    ones = np.ones(Ap.shape[0])
    rs = Ap @ ones
    for P, Ac in zip(Ps, fixed.A[1:]):
        assert np.allclose(Ac @ np.ones(Ac.shape[0]), P.T @ rs, rtol=1e-12,
                           atol=1e-12 * np.abs(rs).max())
        rs = P.T @ rs
    b = _reduced_rhs(o)
    op = o.apply_op
    _, n_ilu, _ = bicgstab(op, b, o.ilu_apply, tol=1e-3, maxit=2000)
    cpr = CPR(rp, ci, vals, op, o.ilu_apply, pressure_solve=fixed.vcycle)
    _, n_cpr, ok = bicgstab(op, b, cpr, tol=1e-3, maxit=2000)
    assert ok and n_cpr * 4 <= n_ilu, (n_cpr, n_ilu)


def test_cpr_absorbs_the_iteration_cost_of_block_jacobi_boxes():
    """With the ILU(0) stage cut into 8x8 boxes (Section 2.5's block-Jacobi,
    the form that shortens the GPU wavefront), ILU(0) alone needs many more
    iterations than in one domain, CPR needs fewer than half of ILU(0)'s and
    loses less to the boxes (a system of the layered generator after a
    2-day report step)."""
    m = synth.layered_model(20, 32, 24, config=1, name="layered 20x32x24")
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    st, rep = o.step(2 * synth.DAY)
    assert st == 0, rep
    o.begin_step()
    o.assemble(m["dt"] / 4)
    rp, ci, vals, _ = o.system()
    b = _reduced_rhs(o)
    op = o.apply_op
    its = {}
    for sub in ((0, 0), (8, 8)):
        o.set_subdomains(*sub)
        o.ilu0()
        _, n_ilu, ok0 = bicgstab(op, b, o.ilu_apply, tol=1e-3, maxit=3000)
        _, n_cpr, ok1 = bicgstab(op, b, CPR(rp, ci, vals, op, o.ilu_apply), tol=1e-3, maxit=3000)
        assert ok0 and ok1
        its[sub] = (n_ilu, n_cpr)
    print("BiCGStab iterations (ILU(0), CPR), one domain and 8x8 boxes:", its)
    (i1, c1), (ib, cb) = its[(0, 0)], its[(8, 8)]
    assert 2 * cb <= ib
    assert cb / c1 < ib / i1
