// Cell quantities of the black-oil model with their derivatives (arXiv
// 1910.06059, Sections 2.1.2-2.1.6: PVT, rock compressibility, relative
// permeabilities by Eq. gwseg; Section 2.4 forward-mode AD), shared by the
// reservoir assembly and the well kernels.
#pragma once
#include "common.cuh"
#include "dual.cuh"

namespace bo {

enum { W_ = 0, O_ = 1, G_ = 2 };

struct CellD {
    D3 b[3], lam[3], rho[3], mphi, rgo, A[3];
};

// Cell quantities at (p_o, s_w, x, state) with derivatives with respect to
// the cell's primary variables (Section 2.1.2).
__device__ __forceinline__ void cell_eval(const DevFluid& F, double p_, double sw_, double x_,
                                          int flag, CellD& c) {
    D3 p = dvar(p_, 0), sw = dvar(sw_, 1), x = dvar(x_, 2);
    D3 sg, rgo;
    if (flag == 0) {            // SAT: gas present, oil saturated at r_s(p)
        sg = x;
        rgo = (F.R_sb / F.p_b) * p;
    } else {                    // USAT: no free gas, x is the dissolved ratio
        sg = dconst(0.0);
        rgo = x;
    }
    D3 so = 1.0 - sw - sg;
    c.rgo = rgo;
    c.b[W_] = F.bw_ref * dexp(F.c_w * (p - F.p_ref));
    D3 psat = (F.p_b / F.R_sb) * rgo;
    D3 bsat = 1.0 + F.Bo_slope * rgo;
    c.b[O_] = ddiv(dexp(F.c_o * (p - psat)), bsat);
    D3 mu_o = ddiv(dconst(F.mu_o0), 1.0 + F.mu_o_r * rgo) * dexp(F.c_mu * (p - psat));
    c.b[G_] = (1.0 / (F.p_sc * F.Z)) * p;
    D3 mu_g = F.mu_g0 * (1.0 + (1.0 / F.mu_g_p) * p);
    c.mphi = dexp(F.c_r * (p - F.p_ref));
    c.rho[W_] = F.rho_s[W_] * c.b[W_];
    c.rho[O_] = c.b[O_] * (F.rho_s[O_] + F.rho_s[G_] * rgo);
    c.rho[G_] = F.rho_s[G_] * c.b[G_];
    const double n = F.n_corey;
    D3 krw = dpow(dclamp01((1.0 / (1.0 - F.s_wco - F.s_orw)) * (sw - F.s_wco)), n);
    D3 krg = dpow(dclamp01((1.0 / (1.0 - F.s_wco - F.s_org)) * sg), n);
    D3 krow = dpow(dclamp01((1.0 / (1.0 - F.s_wco - F.s_orw)) * (so - F.s_orw)), n);
    D3 krog = dpow(dclamp01((1.0 / (1.0 - F.s_wco - F.s_org)) * (so - F.s_org)), n);
    D3 ww = sw - F.s_wco;
    if (ww.v < 0.0) ww = dconst(0.0);
    D3 den = ww + sg;
    // Eq. (gwseg): volume-weighted oil relperm of the two sub-systems.
    D3 kro = (den.v <= 1e-14) ? krow : ddiv(ww * krow + sg * krog, den);
    c.lam[W_] = (1.0 / F.mu_w) * krw;
    c.lam[O_] = ddiv(kro, mu_o);
    c.lam[G_] = ddiv(krg, mu_g);
    c.A[W_] = c.mphi * c.b[W_] * sw;
    c.A[O_] = c.mphi * c.b[O_] * so;
    c.A[G_] = c.mphi * (c.b[G_] * sg + rgo * c.b[O_] * so);
}

}  // namespace bo
