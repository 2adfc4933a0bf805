"""Seeded synthetic black-oil models shaped like the paper's workloads.

This module only draws random fields and lays out numbers: grid sizes, cell
sizes, permeability and porosity fields, well positions and controls, fluid
parameter VALUES, the time-step schedule and random trial states. It holds none
of the method's arithmetic (no PVT, relative permeability, transmissibility,
flux or solver code), so both the CPU oracle and the CUDA path can take their
inputs from it without sharing any of the computation.

Every array comes from ``numpy.random.Generator(PCG64(seed))`` with
``seed = 1910060590 + 100 * config + member``.

Units are SI throughout: Pa, m, s, m^2 (permeability), Pa.s, and surface m^3
for well rates.  Cell index ``c = i + nx * (j + ny * k)``, 0-based, with ``k``
counting layers downward from the top.
"""
from __future__ import annotations

import numpy as np

# Unit conversions (exact or standard definitions).
PSI = 6894.757293168
FT = 0.3048
MD = 9.869233e-16
CP = 1.0e-3
DAY = 86400.0
STB = 0.158987294928
MSCF = 28.316846592

SEED0 = 1910060590


def rng_for(config: int, member: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + 100 * config + member))


def fluid_params() -> dict:
    """Parameter values of the analytic fluid and rock model (SI units).

    The paper states the forms of the PVT and relative-permeability
    relations (Section 2.1.4-2.1.6) but not their values; these values are
    the build's stated reading, shared by both implementations.
    """
    return {
        "g": 9.80665,
        "rho_s": [1000.0, 800.0, 0.9],        # surface densities w, o, g (kg/m^3)
        "p_ref": 4000.0 * PSI,                # reference pressure for water and rock
        "bw_ref": 1.0 / 1.01,                 # water shrinkage factor at p_ref
        "c_w": 4.5e-10,                       # water compressibility (1/Pa)
        "mu_w": 0.5 * CP,                     # water viscosity
        "R_sb": 180.0,                        # dissolved gas ratio at bubble point
        "p_b": 4000.0 * PSI,                  # bubble-point pressure
        "Bo_slope": 0.0025,                   # B_o,sat(r) = 1 + Bo_slope * r
        "c_o": 2.0e-9,                        # undersaturated oil compressibility
        "mu_o0": 2.0 * CP,                    # dead-oil viscosity scale
        "mu_o_r": 0.004,                      # mu_o,sat = mu_o0 / (1 + mu_o_r * r)
        "c_mu": 1.0e-9,                       # undersaturated viscosity slope
        "p_sc": 101325.0,                     # standard pressure
        "Z": 1.2,                             # gas deviation factor
        "mu_g0": 0.01 * CP,                   # gas viscosity at p = 0
        "mu_g_p": 3.0e7,                      # gas viscosity pressure scale
        "c_r": 5.0e-10,                       # rock compressibility
        "s_wco": 0.1,                         # connate water
        "s_orw": 0.1,                         # residual oil to water
        "s_org": 0.1,                         # residual oil to gas
        "n_corey": 2.0,                       # Corey exponent
    }


def _well(i, j, ks, kind, control, target, bhp_limit, phase="gas", rw=0.1, skin=0.0):
    return {
        "i": int(i), "j": int(j), "ks": [int(k) for k in ks],
        "kind": kind,            # "inj" or "prod"
        "phase": phase,          # injected phase for injectors: "water" or "gas"
        "control": control,      # "rate" or "bhp"
        "target": float(target), # surface rate (m^3/s, > 0) or BHP (Pa)
        "bhp_limit": float(bhp_limit),
        "rw": float(rw), "skin": float(skin),
    }


def _grf2d(rng, nx, ny, corr):
    """Unit-variance 2-D Gaussian random field, Gaussian covariance of
    correlation length ``corr`` cells, by the FFT spectral method on a grid
    padded to twice the size."""
    px, py = 2 * nx, 2 * ny
    white = rng.standard_normal((py, px))
    kx = np.fft.fftfreq(px)
    ky = np.fft.fftfreq(py)
    k2 = kx[None, :] ** 2 + ky[:, None] ** 2
    amp = np.exp(-0.5 * (np.pi * corr) ** 2 * k2)
    f = np.real(np.fft.ifft2(np.fft.fft2(white) * amp))[:ny, :nx]
    f -= f.mean()
    s = f.std()
    return f / s if s > 0 else f


def _grf3d(rng, nx, ny, nz, corr):
    px, py, pz = 2 * nx, 2 * ny, 2 * nz
    white = rng.standard_normal((pz, py, px))
    kx = np.fft.fftfreq(px)
    ky = np.fft.fftfreq(py)
    kz = np.fft.fftfreq(pz)
    k2 = kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + kz[:, None, None] ** 2
    amp = np.exp(-0.5 * (np.pi * corr) ** 2 * k2)
    f = np.real(np.fft.ifftn(np.fft.fftn(white) * amp))[:nz, :ny, :nx]
    f -= f.mean()
    s = f.std()
    return f / s if s > 0 else f


def _poro_from_lnk(lnk, mean, sigma):
    return np.clip(0.2 + 0.05 * (lnk - mean) / sigma, 0.05, 0.35)


def _base(name, nx, ny, nz, dx, dy, dz, perm, poro, wells, n_steps, dt):
    return {
        "name": name,
        "nx": nx, "ny": ny, "nz": nz,
        "dx": np.full(nx, dx) if np.isscalar(dx) else np.asarray(dx, float),
        "dy": np.full(ny, dy) if np.isscalar(dy) else np.asarray(dy, float),
        "dz": np.full(nz, dz) if np.isscalar(dz) else np.asarray(dz, float),
        "top_depth": 2500.0,
        "perm": np.ascontiguousarray(perm.reshape(-1), dtype=np.float64),
        "poro": np.ascontiguousarray(poro.reshape(-1), dtype=np.float64),
        "fluid": fluid_params(),
        "wells": wells,
        "init": {"p_top": 4800.0 * PSI, "sw": 0.15, "rgo": 180.0},
        "n_steps": n_steps, "dt": dt,
    }


def anisotropic(model: dict, seed: int = 0, ky_kx=(0.3, 3.0), kz_kx=(0.01, 0.3)) -> dict:
    """The model with cell-wise anisotropic permeability [3][n] (kx, ky, kz):
    kx is the model's field, ky / kx and kz / kx are log-uniform per cell in
    the given ranges (kv/kh of layered sandstones lies in the lower range)."""
    m = dict(model)
    rng = np.random.default_rng(10_000 + seed)
    kx = np.asarray(model["perm"], dtype=np.float64).reshape(-1)
    n = kx.size
    ry = np.exp(rng.uniform(np.log(ky_kx[0]), np.log(ky_kx[1]), n))
    rz = np.exp(rng.uniform(np.log(kz_kx[0]), np.log(kz_kx[1]), n))
    m["perm"] = np.ascontiguousarray(np.concatenate([kx, kx * ry, kx * rz]))
    m["name"] = model["name"] + " anisotropic"
    return m


def config0() -> dict:
    """10x10x3 SPE1-shaped model: 1000x1000x50 ft cells, ln k ~ N(ln 200 mD, 1)
    i.i.d., porosity 0.3, gas injector at (1,1,1) under rate control
    (100 MMscf/d, BHP limit 9014 psia), BHP producer at (10,10,3) (1000 psia);
    10 steps of 30 days."""
    rng = rng_for(0)
    nx, ny, nz = 10, 10, 3
    lnk = np.log(200 * MD) + rng.standard_normal((nz, ny, nx))
    perm = np.exp(lnk)
    poro = np.full((nz, ny, nx), 0.3)
    wells = [
        _well(0, 0, [0], "inj", "rate", 100e3 * MSCF / DAY, 9014 * PSI, phase="gas"),
        _well(9, 9, [2], "prod", "bhp", 1000 * PSI, 1000 * PSI),
    ]
    return _base("spe1-shaped 10x10x3", nx, ny, nz, 1000 * FT, 1000 * FT, 50 * FT,
                 perm, poro, wells, 10, 30 * DAY)


def layered_model(nx, ny, nz, config=1, corr=8.0, sigma=2.0, name=None):
    """Layered log-permeability: per layer ln k = ln 200 mD + sigma*G_k; even
    layers smooth GRF, odd layers channelised (+3 in ln k inside sinusoidal
    bands |sin(2 pi (x cos t + y sin t)/lam + ph)| > 0.8, t in [20,60] deg,
    lam in [20,60] cells).  Porosity correlated with ln k in [0.05, 0.35].
    Five-spot: water injector at the centre column under rate control
    (5000 stb/d, BHP limit 10000 psi), four BHP producers at the corner
    columns (3000 psi); all wells perforate every layer.  20x10x2 ft cells."""
    rng = rng_for(config)
    mean = np.log(200 * MD)
    lnk = np.empty((nz, ny, nx))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for k in range(nz):
        g = _grf2d(rng, nx, ny, corr)
        lnk[k] = mean + sigma * g
        if k % 2 == 1:
            th = np.deg2rad(rng.uniform(20, 60))
            lam = rng.uniform(20, 60)
            ph = rng.uniform(0, 2 * np.pi)
            band = np.abs(np.sin(2 * np.pi * (xx * np.cos(th) + yy * np.sin(th)) / lam + ph)) > 0.8
            lnk[k] += 3.0 * band
    perm = np.exp(lnk)
    poro = _poro_from_lnk(lnk, mean, sigma)
    ks = list(range(nz))
    wells = [
        _well(nx // 2, ny // 2, ks, "inj", "rate", 5000 * STB / DAY, 10000 * PSI, phase="water"),
        _well(0, 0, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(nx - 1, 0, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(0, ny - 1, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(nx - 1, ny - 1, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
    ]
    return _base(name or f"layered {nx}x{ny}x{nz}", nx, ny, nz, 20 * FT, 10 * FT, 2 * FT,
                 perm, poro, wells, 20, 10 * DAY)


def config1() -> dict:
    """60x220x85 layered model (1,122,000 cells); 20 steps of 10 days."""
    return layered_model(60, 220, 85, config=1, name="layered 60x220x85")


def config2() -> dict:
    """100x100x50 model, 3-D GRF ln k (corr. length 10 cells, sigma 1.5),
    wells and PVT as config 1; 30 steps of 5 days."""
    rng = rng_for(2)
    nx, ny, nz = 100, 100, 50
    mean = np.log(200 * MD)
    lnk = mean + 1.5 * _grf3d(rng, nx, ny, nz, 10.0)
    ks = list(range(nz))
    wells = [
        _well(nx // 2, ny // 2, ks, "inj", "rate", 5000 * STB / DAY, 10000 * PSI, phase="water"),
        _well(0, 0, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(nx - 1, 0, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(0, ny - 1, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
        _well(nx - 1, ny - 1, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
    ]
    return _base("grf 100x100x50", nx, ny, nz, 20 * FT, 10 * FT, 2 * FT,
                 np.exp(lnk), _poro_from_lnk(lnk, mean, 1.5), wells, 30, 5 * DAY)


def small_model(nx, ny, nz, config=7, seed_member=0, wells="5spot", dx=20 * FT,
                dy=10 * FT, dz=2 * FT, sigma=1.0):
    """Small lognormal model for parity tests (several tiles, ragged sizes)."""
    rng = rng_for(config, seed_member)
    mean = np.log(200 * MD)
    lnk = mean + sigma * rng.standard_normal((nz, ny, nx))
    ks = list(range(nz))
    if wells == "5spot":
        w = [
            _well(nx // 2, ny // 2, ks, "inj", "rate", 200 * STB / DAY, 10000 * PSI, phase="water"),
            _well(0, 0, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
            _well(nx - 1, ny - 1, ks, "prod", "bhp", 3500 * PSI, 3500 * PSI),
        ]
    elif wells == "gas":
        w = [
            _well(0, 0, [0], "inj", "rate", 2e3 * MSCF / DAY, 9014 * PSI, phase="gas"),
            _well(nx - 1, ny - 1, [nz - 1], "prod", "bhp", 3000 * PSI, 3000 * PSI),
        ]
    else:
        w = []
    return _base(f"small {nx}x{ny}x{nz}", nx, ny, nz, dx, dy, dz,
                 np.exp(lnk), _poro_from_lnk(lnk, mean, sigma), w, 5, 1 * DAY)


def random_state(model: dict, seed_member: int = 0, frac_sat: float = 0.5):
    """Random trial state for Jacobian/assembly checks.

    SAT cells (flag 0): s_g ~ U[0.02, 0.3], x = s_g.
    USAT cells (flag 1): x = r_go ~ U[50, 170] with p >= 4000 psi, so that
    r_go stays below the dissolution limit of the configured gas-oil ratio.
    s_w ~ U[0.12, 0.6] with s_w + s_g <= 0.85.  Pressures in psi drawn
    U[2500, 6000] (SAT) or U[4100, 6000] (USAT).  Well BHPs are drawn around
    their targets.
    """
    rng = rng_for(9, seed_member)
    n = model["nx"] * model["ny"] * model["nz"]
    flag = (rng.uniform(size=n) >= frac_sat).astype(np.uint8)
    sw = rng.uniform(0.12, 0.6, n)
    sg = rng.uniform(0.02, 0.3, n)
    sg = np.minimum(sg, 0.85 - sw)
    p_sat = rng.uniform(2500, 6000, n) * PSI
    p_usat = rng.uniform(4100, 6000, n) * PSI
    rgo = rng.uniform(50, 170, n)
    p = np.where(flag == 1, p_usat, p_sat)
    x = np.where(flag == 1, rgo, sg)
    bhp = []
    for w in model["wells"]:
        if w["control"] == "bhp":
            bhp.append(w["target"])
        elif w["kind"] == "inj":
            bhp.append(rng.uniform(6500, 8000) * PSI)
        else:
            bhp.append(rng.uniform(1500, 2500) * PSI)
    return (np.ascontiguousarray(p), np.ascontiguousarray(sw), np.ascontiguousarray(x),
            np.ascontiguousarray(flag), np.asarray(bhp, dtype=np.float64))


def config3_member(member: int) -> dict:
    """Member `member` of the 256-member ensemble: nx, ny ~ U{20..64},
    nz ~ U{5..16}; ln k = ln 200 mD + sigma_m G with sigma_m ~ U[1, 2] and G a
    unit-variance 3-D Gaussian-covariance GRF (correlation length 8 cells);
    porosity as config 1; 20x10x2 ft cells.  Water injector at (1, 1, .) under
    rate control (0.2% of the pore volume per day at surface conditions, BHP
    limit 10000 psi) and a BHP producer (3000 psi) at (nx, ny, .), both
    perforating every layer; 20 steps of 15 days.  Draws from
    PCG64(1910060590 + 300 + member)."""
    rng = rng_for(3, member)
    nx, ny = (int(v) for v in rng.integers(20, 65, size=2))
    nz = int(rng.integers(5, 17))
    sigma = float(rng.uniform(1.0, 2.0))
    mean = np.log(200 * MD)
    lnk = mean + sigma * _grf3d(rng, nx, ny, nz, 8.0)
    poro = _poro_from_lnk(lnk, mean, sigma)
    pv = float(np.sum(poro) * (20 * FT) * (10 * FT) * (2 * FT))
    ks = list(range(nz))
    wells = [
        _well(0, 0, ks, "inj", "rate", 0.002 * pv / DAY, 10000 * PSI, phase="water"),
        _well(nx - 1, ny - 1, ks, "prod", "bhp", 3000 * PSI, 3000 * PSI),
    ]
    return _base(f"ensemble member {member} ({nx}x{ny}x{nz})", nx, ny, nz, 20 * FT, 10 * FT,
                 2 * FT, np.exp(lnk), poro, wells, 20, 15 * DAY)


def config3(members: int = 256) -> list:
    """The ensemble: members 0 .. members-1 of config3_member."""
    return [config3_member(q) for q in range(members)]


CONFIGS = {0: config0, 1: config1, 2: config2}


# ---------------------------------------------------------------------------
# Initial parameters of the learned preconditioner stage (an input to both
# the GPU library and the oracle): a 63 -> 128 -> 128 -> 9 MLP stored flat as
# W1[128,63], b1[128], W2[128,128], b2[128], W3[9,128], b3[9].
# ---------------------------------------------------------------------------
ML_SHAPES = [(128, 63), (128,), (128, 128), (128,), (9, 128), (9,)]


def learned_init(seed: int = 0) -> np.ndarray:
    """He-uniform hidden layers and a zero output layer (so the untrained
    stage adds nothing and training starts from plain ILU(0)), drawn from
    PCG64(seed); flat float64 vector of 25,865 parameters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for shape in ML_SHAPES:
        if len(shape) == 2 and shape[0] == 128:
            lim = np.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, shape).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts)
