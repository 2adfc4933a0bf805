"""The paper's full standard well (four unknowns per well, cross-flow and
wellbore storage) coupled to the oracle's reservoir equations, in plain
NumPy with a dense Newton solve for small models.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` this is the slow,
readable CPU reference; only tests may import it.  Section 2.2.1 defines the
model: per well the weighted total rate Q_t, the weighted fractions F_w and
F_g and the bottom-hole pressure p_bhp (Eq. weighted_total_rate, with
weights g_w = g_o = 1 and g_g = 0.01, the small gas weight the section
recommends); connection inflow by Eq. (wellinflow); one conservation
equation per component with a storage term (Eq. conseq-swell); the BHP or
rate control equation.  Readings taken where the section is silent:

* Component surface rates of the well: Q_a = F_a Q_t / g_a, F_o = 1 - F_w - F_g;
  production positive, so an injector has Q_t < 0.
* A producing connection (p_j > p_bhp + h_j) carries each phase at the
  cell's mobility, q_a = WI b_a lambda_a dp, gas adding r_go times the oil
  term (as in the reduced well).  An injecting connection (of an injector,
  or in cross-flow of a producer) carries the total reservoir volume rate
  WI lambda_t dp split by
  the wellbore mixture: surface rate q_a = WI lambda_t dp Q_a / V, with
  V = Q_w / b_w + Q_o / b_o + (Q_g - r Q_o) / b_g the reservoir volume of the
  mixture at the cell's pressure (r the dissolved gas ratio the mixture can
  hold there, min(r_s(p), Q_g / Q_o)).  A pure injected phase gives the
  reduced well's injector exactly.
* An injector's wellbore holds its injected phase: F is fixed (1 for that
  phase), its two other component equations become F_w = F_w,inj and
  F_g = F_g,inj, and its connections only inject.  Without this, a well whose
  every connection injects leaves its composition undetermined (any mixture
  passes through), which the section's storage term otherwise resolves.
  Cross-flow is therefore a producer's: fluid produced through some
  connections re-enters the reservoir through others with the wellbore's
  composition.
* Heads h_j and the datum as in the reduced well: the first connection's
  depth, the mobility-weighted density of the connected cells for a
  producer and the injected phase's density for an injector, at the step
  start.
* Storage: A_a,w = V_w F_a / g_a with V_w = pi r_w^2 times the perforated
  thickness (0 turns it off).
* Jacobian: exact throughout -- the reservoir block from the C++ oracle's
  automatic differentiation, the well terms by forward-mode dual numbers
  over the connection cell's three unknowns and the well's four
  (``assemble``); ``assemble_fd`` takes central differences of the well
  terms instead and serves as the check of the exact one.  Newton stops on
  the MB and CNV measures of the reservoir residual with the well terms and
  on |R_w| relative to the well's rate scale.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

G_WEIGHTS = (1.0, 1.0, 0.01)
NV = 7   # dual slots: the connection cell's (p, s_w, x), the well's (Q_t, F_w, F_g, p_bhp)


class Dual:
    """Forward-mode dual number: value v and derivatives d[NV]."""
    __slots__ = ("v", "d")

    def __init__(self, v, d=None):
        self.v = float(v)
        self.d = np.zeros(NV) if d is None else np.asarray(d, float)

    @staticmethod
    def var(v, slot):
        d = np.zeros(NV)
        d[slot] = 1.0
        return Dual(v, d)

    @staticmethod
    def lift(x):
        return x if isinstance(x, Dual) else Dual(x)

    def __add__(self, o):
        o = Dual.lift(o)
        return Dual(self.v + o.v, self.d + o.d)

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual.lift(o)
        return Dual(self.v - o.v, self.d - o.d)

    def __rsub__(self, o):
        return Dual.lift(o) - self

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __mul__(self, o):
        o = Dual.lift(o)
        return Dual(self.v * o.v, self.d * o.v + self.v * o.d)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if not isinstance(o, Dual):
            return Dual(self.v / o, self.d / o)
        return Dual(self.v / o.v, (self.d * o.v - self.v * o.d) / (o.v * o.v))

    def __rtruediv__(self, o):
        return Dual.lift(o) / self


class StandardWellModel:
    """Reservoir (oracle) + full standard wells; one Newton solve per step."""

    def __init__(self, model: dict, storage: bool = True, g=G_WEIGHTS):
        self.model = model
        self.F = model["fluid"]
        self.g = np.asarray(g, float)
        res = dict(model)
        res["wells"] = []
        self.o = oracle.Oracle(res)                       # reservoir equations only
        full = oracle.Oracle(model)                       # for WI and depth
        st = full.static()
        self.depth = st["depth"]
        self.n, self.nx, self.ny = self.o.n, self.o.nx, self.o.ny
        self.wells = []
        off = 0
        for q, w in enumerate(model["wells"]):
            cells = list(full.well_cells[q])
            dz = np.asarray(model["dz"], float)
            thick = sum(dz[c // (self.nx * self.ny)] for c in cells)
            self.wells.append({
                "spec": w, "cells": cells, "wi": st["wi"][off:off + len(cells)],
                "inj": w["kind"] == "inj", "phase": 0 if w.get("phase", "gas") == "water" else 2,
                "control": 0 if w["control"] == "rate" else 1,
                "vw": math.pi * w["rw"] ** 2 * thick if storage else 0.0,
                "x": np.zeros(4), "A0": np.zeros(3), "z_datum": 0.0, "rho": 0.0,
            })
            off += len(cells)
        self.nw = len(self.wells)

    # -- state --------------------------------------------------------------
    def cells(self):
        p, sw, x, fl, _ = self.o.get_state()
        return p, sw, x, fl

    def props(self, c, p, sw, x, fl):
        return oracle.cell_props(self.F, p[c], sw[c], x[c], fl[c])

    def set_state(self, p, sw, x, flag, bhp):
        self.o.set_state(p, sw, x, flag, np.zeros(0))
        for w, b in zip(self.wells, bhp):
            w["x"] = np.array([0.0, 0.0, 0.0, float(b)])
            w["control"] = 0 if w["spec"]["control"] == "rate" else 1
            if w["control"] == 1:
                w["x"][3] = w["spec"]["target"]
            if w["inj"]:
                w["x"][1 + (0 if w["phase"] == 0 else 1)] = 1.0   # F of the injected phase
        self._begin_wells()
        for w in self.wells:                                    # Q_t, F from the current inflow
            if not w["inj"]:
                q = self._well_rates(w, *self.cells(), w["x"][3])
                Q = q.sum(axis=0)
                qt = float(self.g @ Q)
                if qt > 0:
                    w["x"][0] = qt
                    w["x"][1], w["x"][2] = self.g[0] * Q[0] / qt, self.g[2] * Q[2] / qt
            else:
                w["x"][0] = -w["spec"]["target"] * self.g[w["phase"]] if w["control"] == 0 else 0.0

    def _begin_wells(self):
        """Step start: controls from the specification (a switch to BHP control
        lasts for the rest of a step, as for the reduced well), the datum and
        the wellbore density, the storage at the step start."""
        p, sw, x, fl = self.cells()
        for w in self.wells:
            w["control"] = 0 if w["spec"]["control"] == "rate" else 1
            if w["control"] == 1:
                w["x"][3] = w["spec"]["target"]
            c0 = w["cells"][0]
            w["z_datum"] = self.depth[c0]
            if w["inj"]:
                w["rho"] = self.props(c0, p, sw, x, fl)["rho_" + "wog"[w["phase"]]][0]
            else:
                num = den = 0.0
                for c in w["cells"]:
                    cp = self.props(c, p, sw, x, fl)
                    for a in "wog":
                        num += cp["lam_" + a][0] * cp["rho_" + a][0]
                        den += cp["lam_" + a][0]
                w["rho"] = num / den if den > 0 else 0.0
            w["A0"] = self._storage(w, w["x"])

    def get_state(self):
        p, sw, x, fl = self.cells()
        return p, sw, x, fl, np.array([w["x"][3] for w in self.wells])

    @staticmethod
    def _bhp_target(w):
        """The BHP a BHP-controlled well holds: its target under BHP control by
        specification, its BHP limit after a switch from rate control."""
        return w["spec"]["target"] if w["spec"]["control"] == "bhp" else w["spec"]["bhp_limit"]

    def _opening_bhp(self, w, p):
        """The BHP at which the first connection starts to flow: the lowest
        p_j - h_j for an injector, the highest for a producer."""
        v = [p[c] - self.F["g"] * w["rho"] * (self.depth[c] - w["z_datum"]) for c in w["cells"]]
        return min(v) if w["inj"] else max(v)

    # -- well terms ---------------------------------------------------------
    def _Q(self, xw):
        qt, fw, fg = xw[0], xw[1], xw[2]
        return np.array([fw, 1.0 - fw - fg, fg]) * qt / self.g

    def _storage(self, w, xw):
        fw, fg = xw[1], xw[2]
        return w["vw"] * np.array([fw, 1.0 - fw - fg, fg]) / self.g

    def _well_rates(self, w, p, sw, x, fl, bhp, xw=None):
        """Surface rates [ncon, 3] flowing from each connection's cell into
        the well (production positive)."""
        F = self.F
        out = np.zeros((len(w["cells"]), 3))
        xw = w["x"] if xw is None else xw
        # the mixture's surface composition (any positive multiple of Q_a)
        Qw = np.array([xw[1], 1.0 - xw[1] - xw[2], xw[2]]) / self.g
        for j, c in enumerate(w["cells"]):
            cp = self.props(c, p, sw, x, fl)
            h = F["g"] * w["rho"] * (self.depth[c] - w["z_datum"])
            dp = p[c] - bhp - h
            wi = w["wi"][j]
            b = [cp["b_" + a][0] for a in "wog"]
            lam = [cp["lam_" + a][0] for a in "wog"]
            if dp > 0.0:
                if w["inj"]:
                    continue                                  # injectors only inject
                q = [wi * b[a] * lam[a] * dp for a in range(3)]
                q[2] += cp["r_go"][0] * q[1]
                out[j] = q
            elif dp < 0.0:
                qres = wi * (lam[0] + lam[1] + lam[2]) * dp      # reservoir volume rate, < 0
                rmix = 0.0
                if abs(Qw[1]) > 0:
                    rmix = min((F["R_sb"] / F["p_b"]) * p[c], max(Qw[2] / Qw[1], 0.0))
                V = Qw[0] / b[0] + Qw[1] / b[1] + (Qw[2] - rmix * Qw[1]) / b[2]
                if V != 0.0:
                    out[j] = qres * Qw / V
        return out

    def _conn_duals(self, w, j, c, p, sw, x, fl, xw):
        """Surface rates (3 duals) of connection j into the well: the same
        arithmetic as ``_well_rates`` carried on duals over the cell's and
        the well's unknowns."""
        F = self.F
        cp = self.props(c, p, sw, x, fl)

        def cell(name):
            a = cp[name]
            return Dual(a[0], [a[1], a[2], a[3], 0, 0, 0, 0])

        xv = [Dual.var(xw[k], 3 + k) for k in range(4)]
        pc = Dual.var(p[c], 0)
        h = F["g"] * w["rho"] * (self.depth[c] - w["z_datum"])
        dp = pc - xv[3] - h
        wi = w["wi"][j]
        b = [cell("b_" + a) for a in "wog"]
        lam = [cell("lam_" + a) for a in "wog"]
        zero = [Dual(0.0), Dual(0.0), Dual(0.0)]
        if dp.v > 0.0:
            if w["inj"]:
                return zero
            q = [wi * b[a] * lam[a] * dp for a in range(3)]
            q[2] = q[2] + cell("r_go") * q[1]
            return q
        if dp.v < 0.0:
            qres = wi * (lam[0] + lam[1] + lam[2]) * dp
            Qw = [xv[1] / self.g[0], (1.0 - xv[1] - xv[2]) / self.g[1], xv[2] / self.g[2]]
            rmix = Dual(0.0)
            if abs(Qw[1].v) > 0:
                rs = (F["R_sb"] / F["p_b"]) * pc
                ratio = Qw[2] / Qw[1] if Qw[2].v / Qw[1].v > 0.0 else Dual(0.0)
                rmix = rs if rs.v < ratio.v else ratio
            V = Qw[0] / b[0] + Qw[1] / b[1] + (Qw[2] - rmix * Qw[1]) / b[2]
            if V.v != 0.0:
                return [qres * Qw[a] / V for a in range(3)]
        return zero

    def well_blocks(self, k, dt, p=None, sw=None, x=None, fl=None):
        """Exact well terms of well k (Eq. wellequation's blocks): per
        connection the cell-row rates q [ncon, 3] and their derivatives in the
        cell's unknowns dq_dc [ncon, 3, 3] and in the well's dq_dw [ncon, 3, 4];
        the well residual Rw [4], its derivatives in each connection cell's
        unknowns C [ncon, 4, 3] and in the well's unknowns D [4, 4]."""
        if p is None:
            p, sw, x, fl = self.cells()
        w = self.wells[k]
        xw = w["x"]
        nc = len(w["cells"])
        q = np.zeros((nc, 3))
        dq_dc = np.zeros((nc, 3, 3))
        dq_dw = np.zeros((nc, 3, 4))
        for j, c in enumerate(w["cells"]):
            qd = self._conn_duals(w, j, c, p, sw, x, fl, xw)
            for a in range(3):
                q[j, a] = qd[a].v
                dq_dc[j, a] = qd[a].d[:3]
                dq_dw[j, a] = qd[a].d[3:]
        # wellbore balance R_a = (A_a - A0_a)/dt + Q_a - sum_j q_ja, A_a = V_w F_a / g_a
        Fv = [Dual.var(xw[1], 4), Dual.var(xw[2], 5)]
        qt = Dual.var(xw[0], 3)
        frac = [Fv[0], 1.0 - Fv[0] - Fv[1], Fv[1]]
        bal = [(w["vw"] * frac[a] / self.g[a] - w["A0"][a]) / dt + frac[a] * qt / self.g[a]
               for a in range(3)]
        Rw = np.zeros(4)
        D = np.zeros((4, 4))
        C = np.zeros((nc, 4, 3))
        for a in range(3):
            Rw[a] = bal[a].v - q[:, a].sum()
            D[a] = bal[a].d[3:] - dq_dw[:, a].sum(axis=0)
            C[:, a] = -dq_dc[:, a]
        if w["inj"]:
            a = w["phase"]
            Rw[0], D[0], C[:, 0] = Rw[a], D[a].copy(), C[:, a].copy()
            Rw[1] = xw[1] - (1.0 if a == 0 else 0.0)
            Rw[2] = xw[2] - (1.0 if a == 2 else 0.0)
            D[1] = [0, 1, 0, 0]
            D[2] = [0, 0, 1, 0]
            C[:, 1:3] = 0.0
        C[:, 3] = 0.0
        if w["control"] == 1:
            Rw[3] = xw[3] - self._bhp_target(w)
            D[3] = [0, 0, 0, 1]
        else:
            a = w["phase"] if w["inj"] else 1
            Qa = frac[a] * qt / self.g[a]
            ctl = (-Qa if w["inj"] else Qa) - w["spec"]["target"]
            Rw[3] = ctl.v
            D[3] = ctl.d[3:]
        return {"q": q, "dq_dc": dq_dc, "dq_dw": dq_dw, "Rw": Rw, "C": C, "D": D}

    def _well_residual(self, w, q, xw, dt):
        R = np.zeros(4)
        R[:3] = (self._storage(w, xw) - w["A0"]) / dt + self._Q(xw) - q.sum(axis=0)
        if w["inj"]:   # the injected phase's balance; the composition is fixed
            a = w["phase"]
            R[0] = R[a]
            R[1] = xw[1] - (1.0 if a == 0 else 0.0)
            R[2] = xw[2] - (1.0 if a == 2 else 0.0)
        if w["control"] == 1:
            R[3] = xw[3] - self._bhp_target(w)
        elif w["inj"]:
            R[3] = -self._Q(xw)[w["phase"]] - w["spec"]["target"]
        else:
            R[3] = self._Q(xw)[1] - w["spec"]["target"]
        return R

    # -- the coupled system --------------------------------------------------
    def residual(self, dt, p=None, sw=None, x=None, fl=None, xs=None):
        """Cell residual [n, 3] (reservoir + connection terms) and well residuals [nw, 4]."""
        if p is None:
            p, sw, x, fl = self.cells()
        xs = [w["x"] for w in self.wells] if xs is None else xs
        Rc = np.zeros((self.n, 3))
        Rw = np.zeros((self.nw, 4))
        for k, w in enumerate(self.wells):
            q = self._well_rates(w, p, sw, x, fl, xs[k][3], xs[k])
            for j, c in enumerate(w["cells"]):
                Rc[c] += q[j]
            Rw[k] = self._well_residual(w, q, xs[k], dt)
        return Rc, Rw

    def assemble(self, dt):
        """Dense Jacobian and residual of cells (3n) and wells (4 nw), the
        well terms differentiated exactly (``well_blocks``)."""
        n, nw = self.n, self.nw
        self.o.assemble(dt)
        rp, ci, vals, Rres = self.o.system()
        N = 3 * n + 4 * nw
        J = np.zeros((N, N))
        for c in range(n):
            for q in range(rp[c], rp[c + 1]):
                J[3 * c:3 * c + 3, 3 * ci[q]:3 * ci[q] + 3] = vals[q]
        Rc = np.asarray(Rres, float).reshape(-1).copy()
        Rw_all = np.zeros(4 * nw)
        for k, w in enumerate(self.wells):
            blk = self.well_blocks(k, dt)
            col = 3 * n + 4 * k
            for j, c in enumerate(w["cells"]):
                Rc[3 * c:3 * c + 3] += blk["q"][j]
                J[3 * c:3 * c + 3, 3 * c:3 * c + 3] += blk["dq_dc"][j]
                J[3 * c:3 * c + 3, col:col + 4] += blk["dq_dw"][j]
                J[col:col + 4, 3 * c:3 * c + 3] += blk["C"][j]
            J[col:col + 4, col:col + 4] = blk["D"]
            Rw_all[4 * k:4 * k + 4] = blk["Rw"]
        return J, np.concatenate([Rc, Rw_all])

    def assemble_fd(self, dt):
        """Dense Jacobian and residual with central differences of the well
        terms (the check of ``assemble``)."""
        n, nw = self.n, self.nw
        self.o.assemble(dt)
        rp, ci, vals, Rres = self.o.system()
        N = 3 * n + 4 * nw
        J = np.zeros((N, N))
        for c in range(n):
            for q in range(rp[c], rp[c + 1]):
                J[3 * c:3 * c + 3, 3 * ci[q]:3 * ci[q] + 3] = vals[q]
        p, sw, x, fl = self.cells()
        Rc, Rw = self.residual(dt, p, sw, x, fl)
        R = np.concatenate([(Rres + Rc).reshape(-1), Rw.reshape(-1)])
        # central differences of the well terms (their cell rows and the well
        # rows) in every variable they depend on: the connection cells' and
        # the wells' unknowns
        con = sorted({c for w in self.wells for c in w["cells"]})
        cols = [(c, None, v) for c in con for v in range(3)]
        cols += [(None, k, v) for k in range(nw) for v in range(4)]
        for c, k, v in cols:
            if c is None:
                xk = self.wells[k]["x"]
                hstep = 1e-6 * [abs(xk[0]) + 1e-6, 1.0, 1.0, xk[3]][v]
            else:
                hstep = 1e-6 * [p[c], 1.0, 1.0 if fl[c] == 0 else max(x[c], 1.0)][v]
            pair = []
            for sgn in (1.0, -1.0):
                pp, ss, xx = p.copy(), sw.copy(), x.copy()
                xs = [wl["x"].copy() for wl in self.wells]
                if c is None:
                    xs[k][v] += sgn * hstep
                else:
                    (pp, ss, xx)[v][c] += sgn * hstep
                pair.append(self.residual(dt, pp, ss, xx, fl, xs))
            dRc = (pair[0][0] - pair[1][0]) / (2 * hstep)
            dRw = (pair[0][1] - pair[1][1]) / (2 * hstep)
            col = 3 * c + v if c is not None else 3 * n + 4 * k + v
            for cc in con:
                J[3 * cc:3 * cc + 3, col] += dRc[cc]
            J[3 * n:, col] += dRw.reshape(-1)
        return J, R

    def norms(self, dt, R):
        """MB and CNV of the cell residual (reading of Section 2.3) and the
        largest well residual relative to its rate scale."""
        n = self.n
        p, sw, x, fl = self.cells()
        Rc = R[:3 * n].reshape(n, 3)
        binv = np.array([[1.0 / self.props(c, p, sw, x, fl)["b_" + a][0] for a in "wog"]
                         for c in range(n)])
        pv = self.o.static()["pv"]
        bavg = binv.mean(axis=0)
        mb = dt * bavg * np.abs(Rc.sum(axis=0)) / pv.sum()
        cnv = dt * bavg * np.max(np.abs(Rc) / pv[:, None], axis=0)
        wres = 0.0
        for k, w in enumerate(self.wells):
            Rw = R[3 * n + 4 * k:3 * n + 4 * k + 4]
            qs = max(abs(w["x"][0]), 1e-12)
            if w["inj"]:
                wres = max(wres, abs(Rw[0]) / qs, abs(Rw[1]), abs(Rw[2]))
            else:
                wres = max(wres, np.abs(Rw[:3]).max() / qs)
            scale = w["spec"]["target"] if w["control"] == 0 else max(self._bhp_target(w), 1.0)
            wres = max(wres, abs(Rw[3]) / scale)
        return mb, cnv, wres

    def step(self, dt, tol=1e-8, max_newton=30):
        """One Newton solve of a sub-step of length dt (no cuts); returns
        (converged, Newton iterations)."""
        self.o.begin_step()
        self._begin_wells()
        for it in range(max_newton + 1):
            J, R = self.assemble(dt)
            mb, cnv, wres = self.norms(dt, R)
            if max(mb.max(), cnv.max(), wres) <= tol:
                return True, it
            if it == max_newton:
                return False, it
            self.apply_update(np.linalg.solve(J, R))
        return False, max_newton

    def apply_update(self, dx):
        """Newton update y -= dx of cells (the oracle's chop and switching) and
        wells: the BHP step chopped to 30% of the BHP, a rate well's BHP at most
        halving its distance to the opening pressure, fractions clamped, the
        switch to BHP control past the limit."""
        n = self.n
        self.o.newton_update(dx[:3 * n])          # cells: dy = -dx with the chop
        p_new = self.cells()[0]
        for k, w in enumerate(self.wells):
            d = -dx[3 * n + 4 * k:3 * n + 4 * k + 4]
            dmax = 0.3 * w["x"][3]
            d[3] = max(-dmax, min(dmax, d[3]))
            old = w["x"][3]
            w["x"] += d
            if w["control"] == 0:
                # as for the reduced well: a rate-controlled well keeps
                # flowing, its BHP at most halves the distance to the
                # opening pressure (at the updated cell pressures)
                po = self._opening_bhp(w, p_new)
                if w["inj"]:
                    floor = po + 0.5 * (old - po) if old > po else po + 1e-3 * abs(po)
                    w["x"][3] = max(w["x"][3], floor)
                else:
                    ceil = po - 0.5 * (po - old) if old < po else po - 1e-3 * abs(po)
                    w["x"][3] = min(w["x"][3], ceil)
            w["x"][1] = min(max(w["x"][1], 0.0), 1.0)
            w["x"][2] = min(max(w["x"][2], 0.0), 1.0 - w["x"][1])
            if w["control"] == 0:
                lim = w["spec"]["bhp_limit"]
                if (w["inj"] and w["x"][3] > lim) or (not w["inj"] and w["x"][3] < lim):
                    w["control"] = 1
                    w["x"][3] = lim
