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
* Jacobian: exact for the reservoir block (the C++ oracle's automatic
  differentiation); central differences for every term that involves a
  well.  Newton stops on the MB and CNV measures of the reservoir residual
  with the well terms and on |R_w| relative to the well's rate scale.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

G_WEIGHTS = (1.0, 1.0, 0.01)


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
        p, sw, x, fl = self.cells()
        for w in self.wells:
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
                    rmix = min(F["R_sb"] * p[c] / F["p_b"], max(Qw[2] / Qw[1], 0.0))
                V = Qw[0] / b[0] + Qw[1] / b[1] + (Qw[2] - rmix * Qw[1]) / b[2]
                if V != 0.0:
                    out[j] = qres * Qw / V
        return out

    def _well_residual(self, w, q, xw, dt):
        R = np.zeros(4)
        R[:3] = (self._storage(w, xw) - w["A0"]) / dt + self._Q(xw) - q.sum(axis=0)
        if w["inj"]:   # the injected phase's balance; the composition is fixed
            a = w["phase"]
            R[0] = R[a]
            R[1] = xw[1] - (1.0 if a == 0 else 0.0)
            R[2] = xw[2] - (1.0 if a == 2 else 0.0)
        if w["control"] == 1:
            R[3] = xw[3] - w["spec"]["target"]
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
        """Dense Jacobian and residual of cells (3n) and wells (4 nw)."""
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
            scale = w["spec"]["target"] if w["control"] == 0 else max(w["spec"]["target"], 1.0)
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
            dx = np.linalg.solve(J, R)
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
        return False, max_newton
