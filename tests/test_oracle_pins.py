"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to something fixed independently:
finite differences, closed-form solutions of the continuous equations,
conservation, equilibrium, textbook linear-algebra identities, dense LU, and
a published well-index value.  A dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
import synth
from helpers import bcsr_to_dense, entrywise_rel_ok, make_model, _well

PSI = synth.PSI
MD = synth.MD
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Transmissibility (Appendix B): T_ij must reproduce steady Darcy flow through
# two homogeneous half-cells in series (exact for piecewise-constant k).
# ---------------------------------------------------------------------------
def test_transmissibility_series_darcy():
    k1, k2 = 50 * MD, 800 * MD
    dx = np.array([12.0, 30.0])
    dy, dz = 7.0, 3.0
    m = make_model(2, 1, 1, [k1, k2], 0.2, [], dx=dx, dy=dy, dz=dz)
    o = oracle.Oracle(m)
    st = o.static()
    area = dy * dz
    # Series resistance of the continuous problem v = -k grad p between the
    # two cell centres: (dx1/2)/(k1 A) + (dx2/2)/(k2 A).
    resistance = (dx[0] / 2) / (k1 * area) + (dx[1] / 2) / (k2 * area)
    assert st["Tx"][0] == pytest.approx(1.0 / resistance, rel=1e-14)
    assert st["Tx"][1] == 0.0  # boundary face: no flow (Section 2.1.3)
    # Pore volume and cell-centre depth.
    assert st["pv"][1] == pytest.approx(0.2 * dx[1] * dy * dz, rel=1e-15)
    assert st["depth"][0] == pytest.approx(2500.0 + dz / 2, rel=1e-15)


def test_transmissibility_vertical_uses_layer_thickness():
    m = make_model(1, 1, 3, [100 * MD, 100 * MD, 400 * MD], 0.2, [], dx=5.0, dy=8.0,
                   dz=np.array([1.0, 2.0, 4.0]))
    st = oracle.Oracle(m).static()
    area = 5.0 * 8.0
    for k, (h1, h2, k1, k2) in enumerate([(1.0, 2.0, 100, 100), (2.0, 4.0, 100, 400)]):
        res = (h1 / 2) / (k1 * MD * area) + (h2 / 2) / (k2 * MD * area)
        assert st["Tz"][k] == pytest.approx(1 / res, rel=1e-14)
    assert np.allclose(st["depth"], 2500.0 + np.array([0.5, 2.0, 5.0]))


# ---------------------------------------------------------------------------
# Peaceman well index against the published equivalent radius.
# ---------------------------------------------------------------------------
def test_peaceman_equivalent_radius_square_block():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "peaceman_1978.txt"))
            if l.strip() and not l.startswith("#")]
    ref = {r[0]: (float(r[1]), float(r[2])) for r in rows}
    val, tol = ref["ro_over_dx_square"]
    k, h, dx, rw = 150 * MD, 6.0, 40.0, 0.1
    w = _well(0, 0, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI, rw=rw)
    m = make_model(1, 1, 1, k, 0.2, [w], dx=dx, dy=dx, dz=h)
    wi = oracle.Oracle(m).static()["wi"][0]
    # Steady radial flow q = 2 pi k h dp / (mu ln(r_o/r_w)) defines r_o from WI.
    ro = rw * math.exp(2 * math.pi * k * h / wi)
    assert abs(ro / dx - val) <= tol


def _single_cell_wi(kx, ky, dx, dy, h, rw):
    w = _well(0, 0, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI, rw=rw)
    m = make_model(1, 1, 1, 1.0, 0.2, [w], dx=dx, dy=dy, dz=h)
    m["perm"] = np.array([kx, ky, 0.1 * kx])
    return oracle.Oracle(m).static()["wi"][0]


def test_peaceman_anisotropic_coordinate_transform():
    """Peaceman's anisotropic index follows from the isotropic one by the
    stretch x' = x a, y' = y / a, a = (ky/kx)^(1/4), which turns the rock
    isotropic with k = sqrt(kx ky), the block into dx a by dy / a and the well
    circle into an ellipse of semi-axes r_w a and r_w / a, whose equivalent
    circle for steady radial flow has radius r_w (a + 1/a) / 2.  The
    anisotropic index must equal the isotropic index of that stretched
    problem; with dy = dx sqrt(ky/kx) the stretched block is square and r_o
    must be the published 0.198 of its side."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "peaceman_1978.txt"))
            if l.strip() and not l.startswith("#")]
    ref = {r[0]: (float(r[1]), float(r[2])) for r in rows}
    val, tol = ref["ro_over_dx_square"]
    h, rw = 6.0, 0.1
    for kx, ky, dx, dy in [(150 * MD, 15 * MD, 40.0, 25.0), (20 * MD, 300 * MD, 30.0, 70.0),
                           (80 * MD, 60 * MD, 100.0, 10.0)]:
        a = (ky / kx) ** 0.25
        k = math.sqrt(kx * ky)
        wi = _single_cell_wi(kx, ky, dx, dy, h, rw)
        wi_iso = _single_cell_wi(k, k, dx * a, dy / a, h, rw * (a + 1 / a) / 2)
        assert wi == pytest.approx(wi_iso, rel=1e-13)
        # the square stretched block against the published equivalent radius
        dy_sq = dx * math.sqrt(ky / kx)
        wi_sq = _single_cell_wi(kx, ky, dx, dy_sq, h, rw)
        ro = rw * (a + 1 / a) / 2 * math.exp(2 * math.pi * k * h / wi_sq)
        assert abs(ro / (dx * a) - val) <= tol
    # the anisotropic form meets the isotropic one as ky -> kx
    wi0 = _single_cell_wi(150 * MD, 150 * MD, 40.0, 25.0, h, rw)
    wi1 = _single_cell_wi(150 * MD, 150 * MD * (1 + 1e-9), 40.0, 25.0, h, rw)
    assert wi1 == pytest.approx(wi0, rel=1e-8)
    # swapping kx and ky swaps the roles of dx and dy
    assert _single_cell_wi(150 * MD, 15 * MD, 40.0, 25.0, h, rw) == pytest.approx(
        _single_cell_wi(15 * MD, 150 * MD, 25.0, 40.0, h, rw), rel=1e-13)


# ---------------------------------------------------------------------------
# Cell properties: AD derivatives against central differences; end points of
# the relative permeability curves; continuity at the bubble point.
# ---------------------------------------------------------------------------
def _fd_props(fluid, y, flag, h):
    base = oracle.cell_props(fluid, *y, flag)
    out = {}
    for v in range(3):
        yp = list(y); ym = list(y)
        yp[v] += h[v]; ym[v] -= h[v]
        fp = oracle.cell_props(fluid, *yp, flag)
        fm = oracle.cell_props(fluid, *ym, flag)
        for k in base:
            out.setdefault(k, np.zeros(3))[v] = (fp[k][0] - fm[k][0]) / (2 * h[v])
    return base, out


@pytest.mark.parametrize("flag", [0, 1])
def test_cell_props_ad_vs_fd(flag):
    fluid = synth.fluid_params()
    rng = np.random.default_rng(1)
    for _ in range(25):
        sw = rng.uniform(0.15, 0.55)
        if flag == 0:
            y = (rng.uniform(2500, 6000) * PSI, sw, rng.uniform(0.05, 0.8 - sw))
        else:
            y = (rng.uniform(4100, 6000) * PSI, sw, rng.uniform(50, 170))
        h = (1e-6 * y[0], 1e-7, 1e-7 if flag == 0 else 1e-5)
        base, fd = _fd_props(fluid, y, flag, h)
        for k in base:
            ad = base[k][1:]
            scale = max(np.abs(ad).max(), np.abs(fd[k]).max(), 1e-300)
            # derivatives of a smooth function: per-quantity relative agreement
            assert np.abs(ad - fd[k]).max() <= 1e-7 * scale + 1e-300, (k, ad, fd[k])


def test_relperm_end_points():
    f = synth.fluid_params()
    swco, sorw, sorg = f["s_wco"], f["s_orw"], f["s_org"]
    p = 5000 * PSI
    # connate water, no gas: water immobile, oil at its end point k_ro = 1
    c = oracle.cell_props(f, p, swco, 100.0, 1)
    assert c["lam_w"][0] == 0.0
    assert c["lam_o"][0] * f["mu_o0"] > 0
    mu_o = f["mu_o0"]  # oil mobility times viscosity gives k_ro; recover mu from a zero-krw state
    # residual oil in the water system: oil immobile (k_ro = k_row(s_orw) = 0 with s_g = 0)
    c = oracle.cell_props(f, p, 1.0 - sorw, 100.0, 1)
    assert c["lam_o"][0] == 0.0
    # maximum water saturation 1 - s_orw gives k_rw = 1: lam_w = 1/mu_w
    assert c["lam_w"][0] == pytest.approx(1.0 / f["mu_w"], rel=1e-15)
    # no gas saturation: gas immobile
    c = oracle.cell_props(f, 3000 * PSI, 0.3, 0.0, 0)
    assert c["lam_g"][0] == 0.0
    # gas at 1 - s_wco - s_org in the gas system: k_rg = 1
    c = oracle.cell_props(f, 3000 * PSI, swco, 1 - swco - sorg, 0)
    assert c["lam_g"][0] * (f["mu_g0"] * (1 + 3000 * PSI / f["mu_g_p"])) == pytest.approx(1.0, rel=1e-14)
    # ... and the oil in that state is at its residual: k_rog = 0, and with
    # s_w = s_wco the segregation weights put all weight on k_rog (Eq. gwseg)
    assert c["lam_o"][0] == 0.0
    del mu_o


def test_segregation_model_weights():
    """Eq. (gwseg) is a weighted mean: with s_w = s_wco the oil relperm equals
    the gas-oil curve, with s_g = 0 it equals the water-oil curve, and in
    between it lies between the two."""
    f = synth.fluid_params()
    f["s_org"] = 0.2  # make the water-oil and gas-oil curves differ
    p = 3000 * PSI
    so = 0.55
    # pure gas-oil (s_w = s_wco): k_ro = k_rog(s_o)
    a = oracle.cell_props(f, p, f["s_wco"], 1 - f["s_wco"] - so, 0)
    # pure water-oil (s_g = 0): k_ro = k_row(s_o)
    b = oracle.cell_props(f, p, 1 - so, 0.0, 0)
    mixed = oracle.cell_props(f, p, 0.25, 1 - 0.25 - so, 0)
    lo, hi = sorted([a["lam_o"][0], b["lam_o"][0]])
    assert lo <= mixed["lam_o"][0] <= hi
    # equal weights give the arithmetic mean of the two curves
    sg = (1 - so - f["s_wco"]) / 2
    eq = oracle.cell_props(f, p, f["s_wco"] + sg, sg, 0)
    assert eq["lam_o"][0] == pytest.approx(0.5 * (a["lam_o"][0] + b["lam_o"][0]), rel=1e-13)


def test_properties_continuous_at_saturation_boundary():
    """At r_go = r_s(p) the saturated (x = s_g = 0) and undersaturated
    (x = r_go) descriptions are the same fluid (Section 2.1.2, 2.1.6)."""
    f = synth.fluid_params()
    for p in (1500 * PSI, 3000 * PSI, 4000 * PSI):
        sat = oracle.cell_props(f, p, 0.3, 0.0, 0)
        rs = sat["r_go"][0]
        usat = oracle.cell_props(f, p, 0.3, rs, 1)
        for k in ("b_o", "rho_o", "lam_o", "A_o", "A_g", "A_w", "b_w", "b_g"):
            assert usat[k][0] == pytest.approx(sat[k][0], rel=1e-13), k
        # the saturated dissolved ratio grows with pressure
        assert sat["r_go"][1] > 0


# ---------------------------------------------------------------------------
# Full Jacobian (cells, faces, wells) against central finite differences.
# ---------------------------------------------------------------------------
def _residual_vector(o, state, dt):
    o.set_state(*state)
    o.assemble(dt)
    _, _, _, R = o.system()
    wl = o.wells()
    return R.reshape(-1).copy(), np.array([w["Rw"] for w in wl])


@pytest.mark.parametrize("frac_sat", [0.0, 0.5, 1.0])
def test_jacobian_ad_vs_fd(frac_sat):
    m = synth.small_model(4, 3, 3, wells="5spot", dz=4.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=int(frac_sat * 10), frac_sat=frac_sat)
    o.set_state(*st)
    o.begin_step()
    # perturb the state away from the step start so accumulation is active
    p, sw, x, fl, bhp = [a.copy() for a in st]
    p *= 1.01
    sw += 0.01
    state = (p, sw, x, fl, bhp)
    dt = 5 * synth.DAY
    o.set_state(*state)
    o.assemble(dt)
    rp, ci, vals, R0 = o.system()
    J = bcsr_to_dense(rp, ci, vals, o.n)
    wl = o.wells()
    n = o.n
    rng = np.random.default_rng(3)
    cells = rng.choice(n, size=8, replace=False)
    wcells = [c for cs in o.well_cells for c in cs]
    cells = np.unique(np.concatenate([cells, wcells[:4]]))
    def fd_column(c, v, h):
        def central(hh):
            yp = [a.copy() for a in (p, sw, x)]
            ym = [a.copy() for a in (p, sw, x)]
            yp[v][c] += hh
            ym[v][c] -= hh
            Rp, Wp = _residual_vector(o, (*yp, fl, bhp), dt)
            Rm, Wm = _residual_vector(o, (*ym, fl, bhp), dt)
            return (Rp - Rm) / (2 * hh), (Wp - Wm) / (2 * hh)
        # Richardson extrapolation of the central difference: O(h^4) error
        r1, w1 = central(h)
        r2, w2 = central(h / 2)
        return (4 * r2 - r1) / 3, (4 * w2 - w1) / 3

    for c in cells:
        for v in range(3):
            y = [p, sw, x][v]
            h = 1e-4 * abs(y[c]) if v == 0 or (v == 2 and fl[c] == 1) else 1e-4
            col_fd, wfd = fd_column(c, v, h)
            col_ad = J[:, 3 * c + v]
            # each entry against its own size, floored by the largest entry of
            # the same unknown family in its row (pressure columns are per Pa)
            fam = np.abs(J[:, v::3]).max(axis=1)
            scale = np.maximum(np.abs(col_ad), 1e-3 * fam)
            nz = scale > 0
            err = np.abs(col_fd - col_ad)[nz] / scale[nz]
            assert err.max() <= 1e-7, (c, v, err.max())
            # well equations: B entries
            for q, w in enumerate(wl):
                if w["control"] != 0 or c not in o.well_cells[q]:
                    continue
                con = o.well_cells[q].index(c)
                assert wfd[q] == pytest.approx(w["B"][con, v], rel=1e-7,
                                               abs=1e-7 * np.abs(w["B"][:, v]).max())
    # BHP column: C and D of the rate-controlled wells
    for q, w in enumerate(wl):
        if w["control"] != 0:
            continue
        def central(hh):
            bp = bhp.copy(); bm = bhp.copy()
            bp[q] += hh; bm[q] -= hh
            Rp, Wp = _residual_vector(o, (p, sw, x, fl, bp), dt)
            Rm, Wm = _residual_vector(o, (p, sw, x, fl, bm), dt)
            return (Rp - Rm) / (2 * hh), (Wp[q] - Wm[q]) / (2 * hh)
        h = 1e-4 * bhp[q]
        r1, d1 = central(h)
        r2, d2 = central(h / 2)
        fdC = ((4 * r2 - r1) / 3).reshape(-1, 3)[o.well_cells[q]]
        assert np.allclose(fdC, w["C"], rtol=1e-7, atol=1e-7 * np.abs(w["C"]).max())
        assert (4 * d2 - d1) / 3 == pytest.approx(w["Dw"], rel=1e-7)


# ---------------------------------------------------------------------------
# Conservation: in a closed reservoir the fluxes cancel and every Newton step
# conserves each component's surface volume.
# ---------------------------------------------------------------------------
def _component_masses(o):
    f = o.model["fluid"]
    pv = o.static()["pv"]
    p, sw, x, fl, _ = o.get_state()
    M = np.zeros(3)
    for c in range(o.n):
        cp = oracle.cell_props(f, p[c], sw[c], x[c], fl[c])
        M += pv[c] * np.array([cp["A_w"][0], cp["A_o"][0], cp["A_g"][0]])
    return M


def test_flux_terms_cancel_in_closed_reservoir():
    m = synth.small_model(5, 4, 3, wells="none", dz=6.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=4)
    o.set_state(*st)
    o.begin_step()
    o.assemble(synth.DAY)
    _, _, _, R = o.system()
    # state == step start: accumulation is zero, so the residual is flux only
    flux_scale = np.abs(R).max()
    assert flux_scale > 0
    assert np.all(np.abs(R.sum(axis=0)) <= 1e-12 * flux_scale * o.n)


def test_convergence_norms_closed_form():
    """MB and CNV (Section 2.3's tolerance-mb / tolerance-cnv) on two cells
    that exchange nothing (permeability 1e-30 m^2): each residual is the
    accumulation change (PV/dt)(A(p) - A(p0)) with A from the closed forms of
    the fluid and rock (water b_w exponential in p, live oil b_o at its r_go,
    m_phi exponential in p), B_avg is the mean of 1/b over the cells at the
    current state, MB sums the residual and divides by the summed pore
    volume, CNV takes the largest residual per pore volume."""
    from math import exp
    wells = []
    m = make_model(2, 1, 1, 1e-30, 0.2, wells, dx=10.0, dy=20.0, dz=5.0)
    m["poro"] = np.array([0.15, 0.3])
    F = m["fluid"]
    o = oracle.Oracle(m)
    p0 = np.array([3000.0, 3500.0]) * PSI
    p1 = np.array([3100.0, 3420.0]) * PSI
    sw = np.array([0.3, 0.45])
    r = np.array([100.0, 140.0])                  # undersaturated: p > p_b r / R_sb
    fl = np.ones(2, np.uint8)
    o.set_state(p0, sw, r, fl, np.zeros(1))
    o.begin_step()
    o.set_state(p1, sw, r, fl, np.zeros(1))
    dt = 3.0 * synth.DAY
    o.assemble(dt)
    nrm = o.norms(dt)

    def b_w(p):
        return F["bw_ref"] * exp(F["c_w"] * (p - F["p_ref"]))

    def b_o(p, rr):
        return exp(F["c_o"] * (p - F["p_b"] * rr / F["R_sb"])) / (1.0 + F["Bo_slope"] * rr)

    def b_g(p):
        return p / (F["p_sc"] * F["Z"])

    def acc(p, s, rr):
        mphi = exp(F["c_r"] * (p - F["p_ref"]))
        return np.array([mphi * b_w(p) * s, mphi * b_o(p, rr) * (1 - s),
                         mphi * rr * b_o(p, rr) * (1 - s)])

    pv = m["poro"] * 10.0 * 20.0 * 5.0
    R = np.array([pv[i] / dt * (acc(p1[i], sw[i], r[i]) - acc(p0[i], sw[i], r[i]))
                  for i in range(2)])                                    # [cell][w, o, g]
    binv = np.array([[1 / b_w(p1[i]), 1 / b_o(p1[i], r[i]), 1 / b_g(p1[i])] for i in range(2)])
    bavg = binv.mean(axis=0)
    mb = dt * bavg * np.abs(R.sum(axis=0)) / pv.sum()
    cnv = dt * bavg * np.max(np.abs(R) / pv[:, None], axis=0)
    assert np.allclose(nrm[0:3], mb, rtol=1e-11, atol=0), (nrm[0:3], mb)
    assert np.allclose(nrm[3:6], cnv, rtol=1e-11, atol=0), (nrm[3:6], cnv)
    assert nrm[6] == 0.0


def test_mass_conservation_per_step():
    m = synth.small_model(5, 4, 3, wells="none", dz=6.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=5)
    o.set_state(*st)
    M0 = _component_masses(o)
    for _ in range(3):
        status, rep = o.step(2 * synth.DAY, tol_mb=1e-13, tol_cnv=1e-11, tol_lin=1e-12)
        assert status == 0, rep
        M1 = _component_masses(o)
        assert np.all(np.abs(M1 - M0) <= 1e-10 * M0), (M1 - M0) / M0
        M0 = M1


# ---------------------------------------------------------------------------
# Hydrostatic equilibrium (Section 2.1.3, Eq. head): the initial column
# matches the continuous ODE dp/dz = rho(p) g, and a closed reservoir with
# immobile water and no gas stays at rest.
# ---------------------------------------------------------------------------
def test_hydrostatic_column_matches_ode():
    from scipy.integrate import solve_ivp
    nz, dz = 60, 5.0
    m = make_model(1, 1, nz, 100 * MD, 0.2, [], dz=dz)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    p, *_ = o.get_state()
    f = m["fluid"]
    r = m["init"]["rgo"]
    sw = m["init"]["sw"]
    rho = lambda pp: oracle.cell_props(f, pp, sw, r, 1)["rho_o"][0]
    sol = solve_ivp(lambda z, y: [f["g"] * rho(y[0])], (0, dz * (nz - 1)), [p[0]],
                    rtol=1e-13, atol=1e-6, dense_output=True)
    z = dz * np.arange(nz)
    ref = sol.sol(z)[0]
    # trapezoidal discretisation error is O(dz^2 rho'') -- negligible here
    assert np.max(np.abs(p - ref) / ref) < 1e-10
    assert p[0] == m["init"]["p_top"]
    assert np.all(np.diff(p) > 0)  # pressure increases with depth


def test_closed_reservoir_at_rest_stays_at_rest():
    m = synth.small_model(4, 3, 6, wells="none", dz=3.0)
    m["init"]["sw"] = m["fluid"]["s_wco"]  # immobile water, no free gas
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    s0 = o.get_state()
    for _ in range(10):
        # rounding leaves CNV near 1e-12, four orders below the 1e-6 tolerance
        status, rep = o.step(30 * synth.DAY, tol_mb=1e-10, tol_cnv=1e-10)
        assert status == 0
        assert rep["newton_its"] == 0 and rep["lin_its"] == 0
    s1 = o.get_state()
    assert np.allclose(s1[0], s0[0], rtol=1e-12, atol=0)
    assert np.array_equal(s1[3], s0[3])
    o.begin_step()
    o.assemble(30 * synth.DAY)
    _, _, vals, R = o.system()
    # residual is rounding-level against the flux scale T * lambda * b * p
    st = o.static()
    scale = st["Tz"].max() * 1e3 * m["init"]["p_top"]
    assert np.abs(R).max() <= 1e-13 * scale


# ---------------------------------------------------------------------------
# 1-D incompressible single-phase flow between a BHP injector and a BHP
# producer: the discrete solution is the exact steady Darcy solution
# (Appendix B: v_ij = T_ij (p_i - p_j) / mu); pressure is linear within each
# homogeneous stretch and the rate follows the series resistance.
# ---------------------------------------------------------------------------
def test_1d_incompressible_linear_profile():
    N = 12
    rng = np.random.default_rng(7)
    perm = np.exp(np.log(200 * MD) + 0.5 * rng.standard_normal(N))
    dx, dy, dz = 15.0, 10.0, 4.0
    pL, pR = 5000 * PSI, 4000 * PSI
    wells = [_well(0, 0, [0], "inj", "bhp", pL, pL, phase="water"),
             _well(N - 1, 0, [0], "prod", "bhp", pR, pR)]
    fluid = {"g": 0.0, "c_w": 0.0, "c_r": 0.0, "s_orw": 0.0}
    m = make_model(N, 1, 1, perm, 0.25, wells, fluid=fluid, dx=dx, dy=dy, dz=dz)
    o = oracle.Oracle(m)
    n = N
    p0 = np.full(n, 0.5 * (pL + pR))
    o.set_state(p0, np.ones(n), np.zeros(n), np.zeros(n, np.uint8), np.array([pL, pR]))
    status, rep = o.step(10 * synth.DAY, tol_mb=1e-13, tol_cnv=1e-12, tol_lin=1e-13)
    assert status == 0 and rep["newton_its"] == 1
    p, sw, x, fl, _ = o.get_state()
    assert np.all(sw == 1.0) and np.all(x == 0.0)
    mu = m["fluid"]["mu_w"]
    wi = o.static()["wi"]
    area = dy * dz
    res = [mu / wi[0]]
    for i in range(N - 1):
        res.append(mu * ((dx / 2) / (perm[i] * area) + (dx / 2) / (perm[i + 1] * area)))
    res.append(mu / wi[1])
    q = (pL - pR) / sum(res)
    ref = pL - q * np.cumsum(res)[:-1]
    assert np.max(np.abs(p - ref)) <= 1e-9 * pL


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_1d_incompressible_anisotropic_chain(axis):
    """The same steady Darcy chain laid along x, y or z of an anisotropic
    rock: only the permeability along the chain enters its resistances (the
    other two components are made 50x larger and 50x smaller to expose a
    mix-up), and the profile is the series solution of Appendix B."""
    N = 10
    rng = np.random.default_rng(11)
    kc = np.exp(np.log(150 * MD) + 0.5 * rng.standard_normal(N))
    h = {"x": 15.0, "y": 12.0, "z": 3.0}
    pL, pR = 5000 * PSI, 4000 * PSI
    dims = {"x": (N, 1, 1), "y": (1, N, 1), "z": (1, 1, N)}[axis]
    if axis == "x":
        wells = [_well(0, 0, [0], "inj", "bhp", pL, pL, phase="water"),
                 _well(N - 1, 0, [0], "prod", "bhp", pR, pR)]
    elif axis == "y":
        wells = [_well(0, 0, [0], "inj", "bhp", pL, pL, phase="water"),
                 _well(0, N - 1, [0], "prod", "bhp", pR, pR)]
    else:
        wells = [_well(0, 0, [0], "inj", "bhp", pL, pL, phase="water"),
                 _well(0, 0, [N - 1], "prod", "bhp", pR, pR)]
    fluid = {"g": 0.0, "c_w": 0.0, "c_r": 0.0, "s_orw": 0.0}
    m = make_model(*dims, 1.0, 0.25, wells, fluid=fluid, dx=h["x"], dy=h["y"], dz=h["z"])
    comp = {"x": 0, "y": 1, "z": 2}[axis]
    perm = np.empty((3, N))
    for d in range(3):
        perm[d] = kc * (1.0 if d == comp else (50.0 if d == (comp + 1) % 3 else 0.02))
    m["perm"] = perm.reshape(-1)
    o = oracle.Oracle(m)
    p0 = np.full(N, 0.5 * (pL + pR))
    o.set_state(p0, np.ones(N), np.zeros(N), np.zeros(N, np.uint8), np.array([pL, pR]))
    status, rep = o.step(10 * synth.DAY, tol_mb=1e-13, tol_cnv=1e-12, tol_lin=1e-13)
    assert status == 0 and rep["newton_its"] == 1
    p = o.get_state()[0]
    mu = m["fluid"]["mu_w"]
    wi = o.static()["wi"]
    area = {"x": h["y"] * h["z"], "y": h["x"] * h["z"], "z": h["x"] * h["y"]}[axis]
    half = h[axis] / 2
    res = [mu / wi[0]]
    for i in range(N - 1):
        res.append(mu * (half / (kc[i] * area) + half / (kc[i + 1] * area)))
    res.append(mu / wi[1])
    q = (pL - pR) / sum(res)
    ref = pL - q * np.cumsum(res)[:-1]
    assert np.max(np.abs(p - ref)) <= 1e-9 * pL


# ---------------------------------------------------------------------------
# 1-D waterflood against the Buckley-Leverett solution: incompressible water
# and undersaturated oil, no gravity, a rate-controlled water injector in the
# first cell and a BHP producer in the last.  With the Corey curves and
# viscosities of Sections 2.1.5-2.1.6 the fractional flow is
# f(S) = (k_rw/mu_w) / (k_rw/mu_w + k_ro/mu_o); water of saturation S travels
# at f'(S) times the injected pore volumes, and the front carries the shock
# saturation S_f of the Welge tangent f'(S_f) (S_f - S_wc) = f(S_f) - f(S_wc).
# The implicit upwind discretisation converges to this profile as the cells
# and the time steps shrink together; a mistake in the fluxes, the upwinding,
# the relative permeabilities or the viscosities changes the limit.
# ---------------------------------------------------------------------------
def _waterflood(N, L=200.0, area=100.0, poro=0.2, q=1e-3, days=11.0):
    fluid = {"g": 0.0, "c_w": 0.0, "c_r": 0.0, "c_o": 0.0, "c_mu": 0.0}
    wells = [_well(0, 0, [0], "inj", "rate", q, 9000 * PSI, phase="water"),
             _well(N - 1, 0, [0], "prod", "bhp", 4800 * PSI, 4800 * PSI)]
    m = make_model(N, 1, 1, 1000 * MD, poro, wells, fluid=fluid, dx=L / N, dy=10.0,
                   dz=area / 10.0)
    F = m["fluid"]
    o = oracle.Oracle(m)
    o.set_state(np.full(N, 5000 * PSI), np.full(N, F["s_wco"]), np.full(N, F["R_sb"]),
                np.ones(N, np.uint8), np.array([5200 * PSI, 4800 * PSI]))   # undersaturated
    dt = 10.0 / N * synth.DAY          # time steps shrink with the cells (fixed CFL)
    steps = int(round(days * synth.DAY / dt))
    for _ in range(steps):
        st, rep = o.step(dt)
        assert st == 0, rep
    sw = o.get_state()[1]
    assert np.all(o.get_state()[3] == 1)            # the oil stays undersaturated
    # injected pore volumes in reservoir water volume (B_w = 1 / bw_ref here)
    X = q / F["bw_ref"] * steps * dt / (area * poro)
    return F, sw, L / N, X


def _bl_fractional_flow(F):
    swc, sor, nc = F["s_wco"], F["s_orw"], F["n_corey"]
    mu_w = F["mu_w"]
    mu_o = F["mu_o0"] / (1.0 + F["mu_o_r"] * F["R_sb"])

    def f(S):
        se = min(max((S - swc) / (1.0 - swc - sor), 0.0), 1.0)
        kw, ko = se ** nc, (1.0 - se) ** nc
        return (kw / mu_w) / (kw / mu_w + ko / mu_o)

    def df(S, h=1e-7):
        return (f(S + h) - f(S - h)) / (2 * h)
    return f, df


def test_waterflood_converges_to_buckley_leverett():
    from scipy.optimize import brentq
    errs = []
    for N in (100, 200, 400):
        F, sw, dx, X = _waterflood(N)
        f, df = _bl_fractional_flow(F)
        swc = F["s_wco"]
        Sf = brentq(lambda S: df(S) * (S - swc) - (f(S) - f(swc)), swc + 0.05,
                    1.0 - F["s_orw"] - 1e-6)
        xc = (np.arange(N) + 0.5) * dx

        def crossing(level):   # where the (decreasing) profile passes level
            i = int(np.nonzero(sw < level)[0][0])
            return xc[i - 1] + (sw[i - 1] - level) / (sw[i - 1] - sw[i]) * dx
        x_front = X * df(Sf)
        pts = [(crossing(0.5 * (Sf + swc)), x_front)]                 # the shock
        pts += [(crossing(S), X * df(S)) for S in (0.6, 0.65, 0.7, 0.75, 0.8)]  # the fan
        errs.append(max(abs(a - b) for a, b in pts) / x_front)
    # first-order upwinding: the error falls steadily with refinement
    assert errs[1] <= 0.7 * errs[0] and errs[2] <= 0.7 * errs[1], errs
    assert errs[2] <= 0.035, errs


# ---------------------------------------------------------------------------
# Linear algebra: ILU(0) identity on the pattern, exactness in 1-D, and the
# Schur-reduced BiCGStab solve against dense LU of the full system.
# ---------------------------------------------------------------------------
def _assembled_small(nx, ny, nz, wells="5spot", seed=0, frac_sat=0.5):
    m = synth.small_model(nx, ny, nz, wells=wells, dz=4.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=seed, frac_sat=frac_sat)
    o.set_state(*st)
    o.begin_step()
    p, sw, x, fl, bhp = [a.copy() for a in st]
    o.set_state(p * 1.005, sw, x, fl, bhp)
    o.assemble(2 * synth.DAY)
    return o


def test_ilu0_product_matches_matrix_on_pattern():
    o = _assembled_small(4, 3, 3)
    rp, ci, vals, _ = o.system()
    lu, uinv = o.ilu0()
    n = o.n
    L = np.eye(3 * n)
    U = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            j = ci[q]
            if j < i:
                L[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[q]
            else:
                U[3 * i:3 * i + 3, 3 * j:3 * j + 3] = lu[q]
        d = [q for q in range(rp[i], rp[i + 1]) if ci[q] == i][0]
        # the stored inverse of the pivot block (columns scale as 1/Pa, 1, 1)
        ok, err = entrywise_rel_ok(uinv[i], np.linalg.inv(lu[d]), 1e-10)
        assert ok, err
    A = bcsr_to_dense(rp, ci, vals, n)
    P = L @ U
    mask = bcsr_to_dense(rp, ci, np.ones_like(vals), n) > 0
    # LU backward-error bound: |A - LU| <= c eps (|L| |U|) entry by entry
    bound = np.abs(L) @ np.abs(U)
    assert np.all(np.abs(P - A)[mask] <= 1024 * np.finfo(float).eps * bound[mask])
    # the ILU apply is the exact inverse of L U
    r = np.random.default_rng(0).standard_normal(3 * n)
    z = o.ilu_apply(r)
    assert np.allclose(P @ z, r, rtol=0, atol=1e-9 * np.abs(r).max())


def test_ilu0_is_exact_block_lu_in_1d():
    m = synth.small_model(9, 1, 1, wells="none")
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=2)
    o.set_state(*st)
    o.begin_step()
    o.set_state(st[0] * 1.01, *st[1:])
    o.assemble(synth.DAY)
    rp, ci, vals, R = o.system()
    A = bcsr_to_dense(rp, ci, vals, o.n)
    r = np.random.default_rng(1).standard_normal(3 * o.n)
    o.ilu0()
    z = o.ilu_apply(r)
    assert np.allclose(A @ z, r, rtol=0, atol=1e-10 * np.abs(r).max())
    status, its, sol = o.solve(tol=1e-10, maxit=10)
    assert status == 0 and its == 1
    assert np.allclose(A @ sol, R.reshape(-1), rtol=0, atol=1e-9 * np.abs(R).max())


@pytest.mark.parametrize("seed,frac_sat", [(0, 0.5), (1, 0.0), (2, 1.0)])
def test_schur_bicgstab_matches_dense_lu(seed, frac_sat):
    o = _assembled_small(4, 3, 2, seed=seed, frac_sat=frac_sat)
    rp, ci, vals, R = o.system()
    n = o.n
    A = bcsr_to_dense(rp, ci, vals, n)
    wl = o.wells()
    rate = [q for q, w in enumerate(wl) if w["control"] == 0]
    assert rate, "test needs a rate-controlled well"
    N = 3 * n + len(rate)
    J = np.zeros((N, N))
    J[:3 * n, :3 * n] = A
    rhs = np.zeros(N)
    rhs[:3 * n] = R.reshape(-1)
    for k, q in enumerate(rate):
        w = wl[q]
        for con, c in enumerate(o.well_cells[q]):
            J[3 * c:3 * c + 3, 3 * n + k] = w["C"][con]
            J[3 * n + k, 3 * c:3 * c + 3] = w["B"][con]
        J[3 * n + k, 3 * n + k] = w["Dw"]
        rhs[3 * n + k] = w["Rw"]
    ref = np.linalg.solve(J, rhs)
    status, its, sol = o.solve(tol=1e-13, maxit=300)
    assert status == 0
    full = np.concatenate([sol[:3 * n], sol[3 * n:][rate]])
    scale = np.abs(ref).reshape(-1)
    # compare per unknown family (pressure, s_w, x, bhp) at its own scale
    for v in range(3):
        a, b = full[v:3 * n:3], ref[v:3 * n:3]
        assert np.max(np.abs(a - b)) <= 1e-8 * np.abs(b).max()
    assert np.allclose(full[3 * n:], ref[3 * n:], rtol=1e-8)
    # the oracle's residual check of the unreduced system agrees
    chk = o.residual_check(sol)
    assert np.max(np.abs(chk[:3 * n])) <= 1e-9 * np.abs(R).max()
    del scale


def test_newton_update_chop_and_switching_cases():
    """The Newton update's safeguards of Section 2.3 on hand-made cases, one
    per cell of a row (the update is cell-local): a pressure step past 30% of
    p is cut to 30%; saturation steps are scaled together to at most 0.2; a
    dissolved-gas step is cut to 0.2 R_sb; a gas saturation that would turn
    negative makes the cell undersaturated at r_go = r_s(p); an r_go above
    r_s(p) makes it saturated with s_g = 0; an undersaturated cell's pressure
    stops 5% below the saturation pressure of its r_go (and the cell then
    switches); s_w stays in [0, 1]."""
    n = 6
    m = make_model(n, 1, 1, 100 * MD, 0.2, [])
    F = m["fluid"]
    o = oracle.Oracle(m)
    rs = lambda p: F["R_sb"] * p / F["p_b"]           # r_s(p), linear (Section 2.1.4)
    SAT, USAT = 0, 1
    p = np.array([3000, 3000, 5000, 4000, 2500, 5000], float) * PSI
    sw = np.array([0.3, 0.3, 0.2, 0.2, 0.2, 0.95])
    x = np.array([0.05, 0.2, 150.0, 170.0, 100.0, 150.0])
    fl = np.array([SAT, SAT, USAT, USAT, USAT, USAT], np.uint8)
    o.set_state(p, sw, x, fl, np.zeros(1))
    dy = np.zeros((n, 3))
    dy[0] = [0.5 * p[0], 0.05, -0.1]     # dp cut to 0.3 p; s_g -> -0.05: switch
    dy[1] = [0.0, 0.5, -0.25]            # scaled by 0.4: ds_w 0.2, ds_g -0.1
    dy[2] = [0.0, 0.0, 100.0]            # dr cut to 36
    dy[3] = [0.0, 0.0, 20.0]             # r_go 190 > r_s = 180: switch
    dy[4] = [-600 * PSI, 0.0, 0.0]       # stops at 0.95 p_sat(100), then switches
    dy[5] = [0.0, 0.1, 0.0]              # s_w 1.05 -> 1
    o.newton_update(-dy.reshape(-1))     # the update is dy = -sol
    pn, swn, xn, fln, _ = o.get_state()
    p0 = 1.3 * p[0]
    assert np.isclose(pn[0], p0, rtol=1e-15) and fln[0] == USAT
    assert np.isclose(xn[0], rs(p0), rtol=1e-14) and np.isclose(swn[0], 0.35)
    assert fln[1] == SAT and np.isclose(swn[1], 0.5) and np.isclose(xn[1], 0.1)
    assert fln[2] == USAT and np.isclose(xn[2], 150.0 + 0.2 * F["R_sb"])
    assert fln[3] == SAT and xn[3] == 0.0 and np.isclose(swn[3], 0.2)
    assert np.isclose(pn[4], 0.95 * F["p_b"] * 100.0 / F["R_sb"], rtol=1e-14)
    # below its saturation pressure the cell holds more gas than r_s(p): saturated, s_g = 0
    assert fln[4] == SAT and xn[4] == 0.0
    assert swn[5] == 1.0
    assert np.array_equal(pn[[1, 2, 3, 5]], p[[1, 2, 3, 5]])


def test_newton_converges_fast_near_solution():
    """Near the solution the Newton iteration with exact linear solves
    converges quadratically (Eq. linsystem): once the scaled residual is
    small, each iteration roughly squares it."""
    m = synth.small_model(5, 4, 3, wells="5spot", dz=4.0)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.step(0.5 * synth.DAY)  # settle the wells
    o.step(0.5 * synth.DAY)
    o.begin_step()
    dt = 0.05 * synth.DAY
    hist = []
    for it in range(12):
        o.assemble(dt)
        nrm = o.norms(dt)
        hist.append(max(nrm[3:6]))
        if hist[-1] < 1e-12:
            break
        st, its, sol = o.solve(tol=1e-14, maxit=300)
        o.newton_update(sol)
    assert hist[-1] < 1e-10, hist
    # the first iterate below 1e-2 and its successor: quadratic reduction
    k = next(q for q, v in enumerate(hist) if v < 1e-2)
    assert k + 1 < len(hist), hist
    assert hist[k + 1] <= 10 * hist[k] ** 1.8, hist


def test_block_jacobi_ilu0_is_exact_per_subdomain_in_1d():
    """Block-Jacobi ILU(0) (Section 2.5: one ILU(0) block per subdomain) on a
    column of cells in y: each subdomain's matrix is block tridiagonal, so its
    ILU(0) is its exact LU and the preconditioner is the inverse of the
    block-diagonal part of A (a dense solve per subdomain)."""
    m = make_model(1, 12, 1, 1e-13, 0.2, [], dy=15.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=3, frac_sat=0.5)
    o.set_state(*st)
    o.begin_step()
    o.assemble(0.5 * synth.DAY)
    rp, ci, v, R = o.system()
    D = bcsr_to_dense(rp, ci, v, o.n)
    o.set_subdomains(4)
    o.ilu0()
    r = np.random.default_rng(1).standard_normal(3 * o.n)
    z = o.ilu_apply(r)
    for k in range(3):
        sl = slice(12 * k, 12 * (k + 1))          # 4 cells x 3 unknowns
        zk = np.linalg.solve(D[sl, sl], r[sl])
        assert np.allclose(z[sl], zk, rtol=1e-10, atol=1e-10 * np.abs(zk).max())
    # without subdomains the same column is one block tridiagonal system
    o.set_subdomains(0)
    o.ilu0()
    assert np.allclose(o.ilu_apply(r), np.linalg.solve(D, r), rtol=1e-9,
                       atol=1e-9 * np.abs(np.linalg.solve(D, r)).max())


def test_block_jacobi_ilu0_stays_in_its_subdomain():
    """A residual supported on one slab gives a preconditioned vector
    supported on that slab only (no coupling between subdomains in M)."""
    m = synth.small_model(5, 12, 3, wells="5spot", dz=3.0)
    o = oracle.Oracle(m)
    o.set_state(*synth.random_state(m, seed_member=2, frac_sat=0.5))
    o.begin_step()
    o.assemble(0.5 * synth.DAY)
    o.set_subdomains(4)
    o.ilu0()
    n = o.n
    j = (np.arange(n) // 5) % 12
    r = np.zeros((n, 3))
    r[j // 4 == 1] = np.random.default_rng(2).standard_normal(((j // 4 == 1).sum(), 3))
    z = o.ilu_apply(r.reshape(-1)).reshape(n, 3)
    assert np.all(z[j // 4 != 1] == 0.0)
    assert np.abs(z[j // 4 == 1]).max() > 0


def test_block_jacobi_ilu0_is_exact_per_z_slab_in_1d():
    """The same exactness on a column of cells in z (gravity and the z faces
    enter the blocks): slabs of 4 layers, the last one ragged (3 layers)."""
    m = make_model(1, 1, 11, 1e-13, 0.2, [], dz=3.0)
    o = oracle.Oracle(m)
    o.set_state(*synth.random_state(m, seed_member=4, frac_sat=0.5))
    o.begin_step()
    o.assemble(0.5 * synth.DAY)
    rp, ci, v, R = o.system()
    D = bcsr_to_dense(rp, ci, v, o.n)
    o.set_subdomains(0, 4)
    o.ilu0()
    r = np.random.default_rng(6).standard_normal(3 * o.n)
    z = o.ilu_apply(r)
    for lo, hi in ((0, 4), (4, 8), (8, 11)):
        sl = slice(3 * lo, 3 * hi)
        zk = np.linalg.solve(D[sl, sl], r[sl])
        assert np.allclose(z[sl], zk, rtol=1e-10, atol=1e-10 * np.abs(zk).max())
    # a y slab height has no effect on a column one cell wide in y
    o.set_subdomains(8, 4)
    o.ilu0()
    assert np.array_equal(o.ilu_apply(r), z)


def test_block_jacobi_ilu0_boxes_in_y_and_z():
    """With cuts in y and z the subdomains are boxes: a residual on one box
    stays on it; with cuts in z alone a residual on one z slab stays on that
    slab; cutting in z and cutting in y give different preconditioners."""
    m = synth.small_model(4, 12, 10, wells="5spot", dz=3.0)
    o = oracle.Oracle(m)
    o.set_state(*synth.random_state(m, seed_member=8, frac_sat=0.5))
    o.begin_step()
    o.assemble(0.5 * synth.DAY)
    n = o.n
    c = np.arange(n)
    j, k = (c // 4) % 12, c // 48
    box = (j // 4) + 3 * (k // 4)               # 3 x 3 boxes (the last in z is 2 layers)
    o.set_subdomains(4, 4)
    o.ilu0()
    rng = np.random.default_rng(9)
    for b in (0, 4, 8):
        r = np.zeros((n, 3))
        r[box == b] = rng.standard_normal(((box == b).sum(), 3))
        z = o.ilu_apply(r.reshape(-1)).reshape(n, 3)
        assert np.all(z[box != b] == 0.0)
        assert np.abs(z[box == b]).max() > 0
    r = rng.standard_normal(3 * n)
    o.set_subdomains(0, 4)
    o.ilu0()
    zz = o.ilu_apply(r).reshape(n, 3)
    o.set_subdomains(4, 0)
    o.ilu0()
    zy = o.ilu_apply(r).reshape(n, 3)
    assert not np.allclose(zz, zy)
    # a residual on z slab 1 (layers 4..7) stays there when only z is cut
    rs = np.zeros((n, 3))
    rs[k // 4 == 1] = 1.0
    o.set_subdomains(0, 4)
    o.ilu0()
    z1 = o.ilu_apply(rs.reshape(-1)).reshape(n, 3)
    assert np.all(z1[k // 4 != 1] == 0.0)


# ---------------------------------------------------------------------------
# Equilibration (Section 2.1.3): RK4 zones against an independent integrator
# ---------------------------------------------------------------------------
def _equil_reference(F, e, z_cells):
    """Phase pressures at z_cells by scipy's adaptive RK45 at tight
    tolerances, anchored as the paper states: the datum's zone from the
    datum, the others from the contacts (equal phase pressures there)."""
    from scipy.integrate import solve_ivp
    datum_z, datum_p, woc, goc, rgo, swc = e

    def rho(zone, p):
        if zone == "water":
            return F["rho_s"][0] * F["bw_ref"] * math.exp(F["c_w"] * (p - F["p_ref"]))
        if zone == "gas":
            return F["rho_s"][2] * p / (F["p_sc"] * F["Z"])
        r = min(rgo, F["R_sb"] / F["p_b"] * p)
        bo = math.exp(F["c_o"] * (p - r * F["p_b"] / F["R_sb"])) / (1 + F["Bo_slope"] * r)
        return bo * (F["rho_s"][1] + r * F["rho_s"][2])

    def integ(zone, z0, p0, z1):
        if z1 == z0:
            return p0
        sol = solve_ivp(lambda z, p: [F["g"] * rho(zone, p[0])], (z0, z1), [p0],
                        method="RK45", rtol=1e-13, atol=1e-8)
        return float(sol.y[0, -1])

    def zone_of(z):
        return "gas" if z < goc else ("oil" if z < woc else "water")

    zd = zone_of(datum_z)
    anchor = {zd: (datum_z, datum_p)}
    if zd == "oil":
        anchor["gas"] = (goc, integ("oil", datum_z, datum_p, goc))
        anchor["water"] = (woc, integ("oil", datum_z, datum_p, woc))
    elif zd == "gas":
        anchor["oil"] = (goc, integ("gas", datum_z, datum_p, goc))
        anchor["water"] = (woc, integ("oil", goc, anchor["oil"][1], woc))
    else:
        anchor["oil"] = (woc, integ("water", datum_z, datum_p, woc))
        anchor["gas"] = (goc, integ("oil", woc, anchor["oil"][1], goc))
    return np.array([integ(zone_of(z), *anchor[zone_of(z)], z) for z in z_cells]), zone_of


@pytest.mark.parametrize("datum_z", [2650.0, 2540.0, 2760.0])   # oil, gas, water zone
def test_equilibration_matches_independent_integration(datum_z):
    m = make_model(1, 1, 60, 1e-13, 0.2, [], dz=5.0)
    o = oracle.Oracle(m)
    e = (datum_z, 25.0e6, 2720.0, 2580.0, 100.0, 0.15)
    o.init_equilibrium(*e)
    p, sw, x, flag, _ = o.get_state()
    z = o.static()["depth"]
    ref, zone_of = _equil_reference(m["fluid"], e, z)
    assert np.max(np.abs(p - ref) / ref) <= 1e-10
    F = m["fluid"]
    for c in range(len(z)):
        zone = zone_of(z[c])
        rs = F["R_sb"] / F["p_b"] * p[c]
        if zone == "gas":
            assert flag[c] == 0 and sw[c] == 0.15 and x[c] == pytest.approx(1 - 0.15 - F["s_org"])
        else:
            assert sw[c] == (1 - F["s_orw"] if zone == "water" else 0.15)
            assert (flag[c], x[c]) == ((1, 100.0) if 100.0 < rs else (0, 0.0))


def test_equilibration_gas_column_is_exponential():
    """All cells in the gas zone: dp/dz = (g rho_Sg / (p_sc Z)) p, so
    p(z) = p0 exp(g rho_Sg (z - z0) / (p_sc Z)) exactly."""
    m = make_model(1, 1, 40, 1e-13, 0.2, [], dz=10.0)
    o = oracle.Oracle(m)
    o.init_equilibrium(2600.0, 20.0e6, 5000.0, 4000.0, 100.0, 0.15)
    p = o.get_state()[0]
    z = o.static()["depth"]
    F = m["fluid"]
    k = F["g"] * F["rho_s"][2] / (F["p_sc"] * F["Z"])
    assert np.allclose(p, 20.0e6 * np.exp(k * (z - 2600.0)), rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# Wells (Section 2.2.1): inflow by hand, and a rate target met at convergence
# ---------------------------------------------------------------------------
def _props_at(m, p, sw, x, flag):
    return oracle.cell_props(m["fluid"], p, sw, x, flag)


@pytest.mark.parametrize("flag", [0, 1])
def test_producer_inflow_by_hand(flag):
    """One cell with one BHP producer, assembled at its own step-start state
    (no accumulation change, no faces): the residual is the producer's
    surface rates, q_a = WI b_a lambda_a (p - p_bhp), gas also carrying
    r_go times the oil term."""
    pb = 3000 * PSI
    m = make_model(1, 1, 1, 200 * MD, 0.2, [_well(0, 0, [0], "prod", "bhp", pb, pb)],
                   dx=30.0, dy=30.0, dz=6.0)
    o = oracle.Oracle(m)
    p, sw = 25.0e6, 0.3
    x = 0.1 if flag == 0 else 120.0
    o.set_state(np.array([p]), np.array([sw]), np.array([x]), np.array([flag], np.uint8),
                np.array([pb]))
    o.begin_step()
    o.assemble(synth.DAY)
    R = o.system()[3][0]
    wi = o.static()["wi"][0]
    cp = _props_at(m, p, sw, x, flag)
    b = [cp["b_w"][0], cp["b_o"][0], cp["b_g"][0]]
    lam = [cp["lam_w"][0], cp["lam_o"][0], cp["lam_g"][0]]
    rgo = cp["r_go"][0]
    dp = p - pb
    want = [wi * b[0] * lam[0] * dp, wi * b[1] * lam[1] * dp,
            wi * (b[2] * lam[2] + rgo * b[1] * lam[1]) * dp]
    assert np.allclose(R, want, rtol=1e-12, atol=0)
    # the production report gives the same surface rates
    q, bhp, ctl = o.well_rates()
    assert np.allclose(q[0], want, rtol=1e-12, atol=0) and bhp[0] == pb and ctl[0] == 1


def test_well_rates_sum_the_residual():
    """At the step-start state the accumulation term vanishes and the face
    fluxes cancel in the sum over cells, so the summed residual of each
    component is the sum of the wells' reported surface rates."""
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    o = oracle.Oracle(m)
    o.set_state(*synth.random_state(m, seed_member=6, frac_sat=0.5))
    o.begin_step()
    o.assemble(synth.DAY)
    R = o.system()[3]
    q, bhp, ctl = o.well_rates()
    assert q.shape == (len(m["wells"]), 3)
    scale = np.abs(q).sum(axis=0) + np.abs(R).sum(axis=0) * 1e-4
    assert np.all(np.abs(R.sum(axis=0) - q.sum(axis=0)) <= 1e-10 * scale)
    assert np.any(q > 0) and np.any(q < 0)      # producers and an injector


def test_producer_wellbore_head_over_two_layers():
    """A BHP producer perforating two stacked cells (Eq. wellinflow with the
    wellbore head of Section 2.2.1): the datum is the first connection, the
    head of the connection below it is g rho_well dz with rho_well the
    mobility-weighted density of the connected cells at the step start, and
    each connection produces q_a = WI b_a lambda_a (p_j - p_bhp - h_j).  The
    face flux between the cells cancels in the sum of their residuals, which
    must equal the summed connection rates."""
    pb, dz = 3000 * PSI, 6.0
    m = make_model(1, 1, 2, 200 * MD, 0.2, [_well(0, 0, [0, 1], "prod", "bhp", pb, pb)],
                   dx=30.0, dy=30.0, dz=dz)
    o = oracle.Oracle(m)
    p = np.array([25.0e6, 25.3e6])
    sw = np.array([0.3, 0.45])
    x = np.array([120.0, 120.0])
    fl = np.ones(2, np.uint8)
    o.set_state(p, sw, x, fl, np.array([pb]))
    o.begin_step()
    o.assemble(synth.DAY)
    R = o.system()[3]
    wi = o.static()["wi"]
    cps = [_props_at(m, p[j], sw[j], x[j], 1) for j in range(2)]
    num = sum(cp[f"lam_{a}"][0] * cp[f"rho_{a}"][0] for cp in cps for a in "wog")
    den = sum(cp[f"lam_{a}"][0] for cp in cps for a in "wog")
    h = [0.0, m["fluid"]["g"] * (num / den) * dz]
    want = np.zeros(3)
    for j, cp in enumerate(cps):
        dp = p[j] - pb - h[j]
        assert dp > 0
        qo = wi[j] * cp["b_o"][0] * cp["lam_o"][0] * dp
        want += [wi[j] * cp["b_w"][0] * cp["lam_w"][0] * dp, qo,
                 wi[j] * cp["b_g"][0] * cp["lam_g"][0] * dp + cp["r_go"][0] * qo]
    assert np.allclose(R.sum(axis=0), want, rtol=1e-11, atol=0), (R.sum(axis=0), want)
    # the match is far finer than the head's share of the oil rate, so a
    # missing or misplaced head would fail it
    assert abs(R.sum(axis=0)[1] - want[1]) < 1e-6 * abs(
        wi[1] * cps[1]["b_o"][0] * cps[1]["lam_o"][0] * h[1])


def test_rate_injector_meets_its_target():
    """A water injector under rate control in a single layer (no wellbore
    head): at convergence its surface rate, summed by hand over the
    connections as WI lambda_t b_w (p_bhp - p_j), equals the target."""
    target = 50 * synth.STB / synth.DAY
    wells = [_well(2, 2, [0], "inj", "rate", target, 10000 * PSI, phase="water"),
             _well(0, 0, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI),
             _well(4, 4, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI)]
    m = make_model(5, 5, 1, 200 * MD, 0.2, wells, dx=30.0, dy=30.0, dz=6.0)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    st, rep = o.step(2 * synth.DAY, tol_mb=1e-12, tol_cnv=1e-12, tol_well=1e-12, tol_lin=1e-12)
    assert st == 0
    p, sw, x, fl, bhp = o.get_state()
    c = 2 + 5 * 2
    cp = _props_at(m, p[c], sw[c], x[c], fl[c])
    lam_t = cp["lam_w"][0] + cp["lam_o"][0] + cp["lam_g"][0]
    q = o.static()["wi"][0] * lam_t * cp["b_w"][0] * (bhp[0] - p[c])
    assert q == pytest.approx(target, rel=1e-8)


def test_rate_injector_switches_to_its_bhp_limit():
    """A water injector asked for far more than its BHP limit allows: after
    the update that would push p_bhp over the limit it switches to BHP
    control (Section 2.2.1's control switch), ends the step exactly at the
    limit, and injects what Eq. wellinflow gives at the limit,
    WI lambda_t b_w (p_limit - p_j), by hand, less than the target.  (A well
    that kept the rate target, or took the rate target as its BHP after the
    switch, fails this.)"""
    target = 1e5 * synth.STB / synth.DAY
    limit = 5200 * PSI
    wells = [_well(2, 2, [0], "inj", "rate", target, limit, phase="water"),
             _well(0, 0, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI),
             _well(4, 4, [0], "prod", "bhp", 3000 * PSI, 3000 * PSI)]
    m = make_model(5, 5, 1, 200 * MD, 0.2, wells, dx=30.0, dy=30.0, dz=6.0)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    st, rep = o.step(0.5 * synth.DAY, tol_mb=1e-12, tol_cnv=1e-12, tol_well=1e-12, tol_lin=1e-12)
    assert st == 0
    p, sw, x, fl, bhp = o.get_state()
    q, bhp_r, ctl = o.well_rates()
    assert ctl[0] == 1 and bhp[0] == limit and bhp_r[0] == limit
    c = 2 + 5 * 2
    assert p[c] < limit
    cp = _props_at(m, p[c], sw[c], x[c], fl[c])
    lam_t = cp["lam_w"][0] + cp["lam_o"][0] + cp["lam_g"][0]
    hand = o.static()["wi"][0] * lam_t * cp["b_w"][0] * (limit - p[c])
    assert q[0][0] < 0 and -q[0][0] == pytest.approx(hand, rel=1e-8)
    assert hand < 0.5 * target


def test_failed_step_restores_the_state_and_cuts_the_substep():
    """Section 2.3's time-step control: a Newton solve that fails (here one
    Newton iteration allowed, no cut allowed) leaves every unknown -- cell
    pressures, saturations, r_go or s_g, phase states, well BHPs -- bit for
    bit as at the step start, and the next sub-step is the failed one times
    the cut factor; with cuts allowed the same step completes in more than
    one sub-step."""
    m = synth.small_model(6, 5, 4, wells="5spot", dz=4.0)
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    o.step(1.0 * synth.DAY)                 # a moving state (wells have flowed)
    assert o.well_rates()[2][0] == 0        # the injector's BHP is an unknown (rate control)
    before = [a.copy() for a in o.get_state()]
    o.dt_next = 10.0 * synth.DAY
    st, rep = o.step(30 * synth.DAY, max_newton=1, max_cuts=0)
    assert st != 0 and rep["cuts"] == 1 and rep["substeps"] == 0
    for a, b in zip(before, o.get_state()):
        assert np.array_equal(a, b)
    assert o.dt_next == 5.0 * synth.DAY
    # six Newton iterations are too few for the 5-day sub-step, enough for 2.5 days
    st, rep = o.step(30 * synth.DAY, max_newton=6, max_cuts=8)
    assert st == 0 and rep["cuts"] >= 1 and rep["substeps"] >= 2
