"""The learned preconditioner stage on the GPU against the oracle
(oracle/learned.py), through the C ABI.

Tolerances:
  tensor-core network (BF16 weights, features and activations, FP32
  accumulation) and FP32 per-cell products vs the FP64 oracle: 3e-2 of the
  largest |delta| per unknown family.  BF16 keeps 8 significant bits (relative rounding 2^-9); each of
  the three layers rounds its inputs once, and the sums over 66 and 128
  terms average the independent roundings, so the outputs carry errors of a
  few 2^-9 relative to their scale; 3e-2 leaves a margin of ~5.
  FP32 training pass vs the FP64 oracle: loss 1e-4 relative, gradient 2e-3
  relative in the 2-norm of each parameter tensor (FP32 sums over all cells
  and the cancellation in e - A delta).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from oracle import learned as ML

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


def random_params(seed, out_scale=0.3):
    theta = synth.learned_init(seed).copy()
    p = ML.unflatten(theta)
    rng = np.random.default_rng(seed + 100)
    p["W3"][:] = out_scale * rng.standard_normal(p["W3"].shape) / np.sqrt(128)
    p["b3"][:] = out_scale * rng.standard_normal(ML.NOUT)
    p["b1"][:] = 0.1 * rng.standard_normal(128)
    p["b2"][:] = 0.1 * rng.standard_normal(128)
    return theta


MODELS = {
    "small_5spot": lambda: synth.small_model(6, 5, 4, wells="5spot", dz=4.0),
    "ragged_33x17x9": lambda: synth.small_model(33, 17, 9, wells="5spot", dz=3.0),
}


def _system(name, seed=4, dt_days=0.5):
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    st = synth.random_state(m, seed_member=seed, frac_sat=0.5)
    g.set_state(*st)
    o.set_state(*st)
    g.begin_step()
    o.begin_step()
    g.assemble(dt_days * synth.DAY)
    o.assemble(dt_days * synth.DAY)
    g.factor()
    o.ilu0()
    rp, ci, v, R = o.system()
    nb = ML.neighbours(m["nx"], m["ny"], m["nz"])
    A7 = ML.blocks7(rp, ci, v, m["nx"], m["ny"], m["nz"])
    return m, g, o, A7, nb, np.asarray(st[3]), R


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9"])
def test_tensor_core_inference_vs_oracle(name, engine):
    m, g, o, A7, nb, flag, R = _system(name)
    theta = random_params(7)
    g.learn_engine = engine
    assert g.learn_engine == engine
    g.learn_set_params(theta)
    p = ML.unflatten(theta)
    rng = np.random.default_rng(3)
    for r in (R, R * (1 + 0.5 * rng.standard_normal(R.shape))):
        dg = g.learn_delta(r.reshape(-1)).reshape(-1, 3)
        do = ML.stage_delta(p, A7, nb, flag, r)
        for v in range(3):
            scale = np.abs(do[:, v]).max()
            assert scale > 0
            err = np.abs(dg[:, v] - do[:, v]).max() / scale
            assert err <= 3e-2, (v, err)
    # linear in r: scaling by a power of two is exact, sums up to FP32 rounding
    d1 = g.learn_delta(R.reshape(-1))
    d2 = g.learn_delta(4.0 * R.reshape(-1))
    assert np.allclose(d2, 4.0 * d1, rtol=1e-12, atol=0)
    r2 = R * rng.standard_normal(R.shape)
    d3 = g.learn_delta((R + r2).reshape(-1))
    d4 = g.learn_delta(r2.reshape(-1))
    for v in range(3):
        scale = np.abs(d3[v::3]).max()
        assert np.abs(d3[v::3] - d1[v::3] - d4[v::3]).max() <= 1e-5 * scale


@pytest.mark.parametrize("name", ["ragged_33x17x9"])
def test_tcgen05_and_mma_sync_networks_agree(name):
    """The two tensor-core kernels compute the same BF16 network with FP32
    accumulation; they differ only in the order of the FP32 sums (and where
    that moves a hidden activation across a BF16 rounding boundary), so the
    per-cell corrections agree far inside the BF16 bar against the oracle."""
    m, g, o, A7, nb, flag, R = _system(name)
    g.learn_set_params(random_params(11))
    out = {}
    for engine in ("mma_sync", "tcgen05"):
        g.learn_engine = engine
        out[engine] = g.learn_delta(R.reshape(-1)).reshape(-1, 3)
    for v in range(3):
        a, b = out["tcgen05"][:, v], out["mma_sync"][:, v]
        assert np.abs(a - b).max() <= 1e-2 * np.abs(b).max(), v


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9"])
def test_fp32_training_pass_vs_oracle(name):
    m, g, o, A7, nb, flag, R = _system(name, seed=6)
    theta = random_params(11)
    g.learn_set_params(theta)
    theta32 = theta.astype(np.float32).astype(np.float64)   # what the device holds
    p = ML.unflatten(theta32)
    r = R * (1 + 0.2 * np.random.default_rng(5).standard_normal(R.shape))
    z0 = o.ilu_apply(r.reshape(-1)).reshape(-1, 3)
    L_o, g_o = ML.loss_and_grad(p, A7, nb, flag, r, z0)
    L_g, grad_g = g.learn_loss_grad(r.reshape(-1))
    assert L_g == pytest.approx(L_o, rel=1e-4)
    gg = ML.unflatten(grad_g)
    for k, _ in ML.PARAM_SHAPES:
        ref = np.linalg.norm(g_o[k])
        assert ref > 0, k
        err = np.linalg.norm(gg[k] - g_o[k]) / ref
        assert err <= 2e-3, (k, err)
    # the pass leaves the parameters unchanged
    assert np.array_equal(g.learn_get_params(), theta32)


def test_untrained_stage_equals_plain_ilu0():
    """Zero output layer: delta = 0 exactly, so the solve with the stage on
    takes the same iterations to the same solution bit for bit."""
    m, g, o, A7, nb, flag, R = _system("ragged_33x17x9", seed=7, dt_days=0.1)
    st0, its0, sol0 = g.solve(1e-3, 1000)
    assert st0 == 0
    g.learn_set_params(synth.learned_init(0))
    g.learn_enable(True)
    st1, its1, sol1 = g.solve(1e-3, 1000)
    assert st1 == 0
    assert its0 == its1
    assert np.array_equal(sol0, sol1)
    assert g.learn_report()["fallbacks"] == 0


def test_online_training_reduces_the_loss():
    m, g, o, A7, nb, flag, R = _system("ragged_33x17x9", seed=7, dt_days=0.1)
    g.learn_set_params(synth.learned_init(1))
    g.learn_online(samples=8, epochs=40, lr=3e-3)
    st, its, sol = g.solve(1e-3, 1000)
    rep = g.learn_report()
    assert st == 0 and rep["systems"] == 1
    assert rep["steps"] % 40 == 0 and 0 < rep["steps"] <= 40 * 8
    assert 0 < rep["last_loss"] < rep["first_loss"], rep
    th = g.learn_get_params()
    assert np.all(np.isfinite(th))
    assert not np.array_equal(th, synth.learned_init(1).astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("name", ["small_5spot", "ragged_33x17x9"])
def test_newton_with_learned_stage_matches_oracle(name):
    """The stage changes the preconditioner only: Newton steps at tight
    tolerances reach the oracle's states (same bar as the FP64 path)."""
    m = MODELS[name]()
    g, o = Sim(m), oracle.Oracle(m)
    g.learn_set_params(random_params(13, out_scale=0.05))
    g.learn_enable(True)
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
        sat = fo == 0
        assert np.max(np.abs(xg[sat] - xo[sat]), initial=0.0) <= 1e-6
        assert np.max(np.abs(xg[~sat] - xo[~sat]) / xo[~sat].clip(1e-300), initial=0.0) <= 1e-6


def test_trained_stage_against_plain_ilu0():
    """What the trained stage gains or loses against the method without it.

    The stage is trained online on the solver's own residuals over one
    report step of a model of the layered generator, then the next Newton
    system is solved with plain ILU(0) and with the trained stage (BiCGStab
    to 1e-3 both times).  The iterations and times are printed, win or loss;
    both solves must reach the tolerance (the stage falls back to plain
    ILU(0) on divergence).  A guard window then solves the next systems both
    ways and keeps the stage only if it needed fewer iterations."""
    import time
    m = synth.layered_model(20, 30, 20, config=1, name="layered 20x30x20")
    g = Sim(m)
    g.init_hydrostatic()
    g.learn_set_params(synth.learned_init(0))
    g.learn_online(samples=8, epochs=1, lr=1e-3)
    st, _ = g.step(5 * synth.DAY)
    assert st == 0
    g.learn_online(on=False)
    trained = g.learn_report()
    assert trained["systems"] > 0 and trained["steps"] > 0
    dt = 5 * synth.DAY
    g.begin_step()
    g.assemble(dt)
    g.factor()
    g.learn_enable(False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st0, its0, x0 = g.solve(tol=1e-3, maxit=500)
    t_plain = time.perf_counter() - t0
    g.learn_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st1, its1, x1, info = g.solve(tol=1e-3, maxit=500, report=True)
    t_stage = time.perf_counter() - t0
    verdict = "gain" if its1 < its0 else "loss"
    print(f"trained stage ({trained['systems']} systems, {trained['steps']} Adam steps): "
          f"{its1} BiCGStab its in {1e3 * t_stage:.1f} ms (fallback mask {info['fallback']}) "
          f"vs plain ILU(0): {its0} its in {1e3 * t_plain:.1f} ms -> {verdict}")
    assert st0 == 0 and st1 == 0
    g.learn_guard(3)
    st, _ = g.step(dt)
    assert st == 0
    r = g.learn_report()
    print(f"guard: stage {r['guard_stage_its']} its vs plain {r['guard_plain_its']} its over 3 "
          f"systems -> {'kept' if r['guard_state'] == 2 else 'turned off'}")
    assert r["guard_state"] in (2, 3)
    assert (r["guard_state"] == 2) == (r["guard_stage_its"] < r["guard_plain_its"])
    g.close()


def test_offline_set_from_earlier_steps():
    """The offline training set: the simulator's own systems and BiCGStab
    residuals from a report step (the reading of 'Jacobian/residual pairs
    from earlier steps' at this model's scale), several passes of Adam over
    all of them, then the trained stage against plain ILU(0) on the next
    system, printed win or loss."""
    import time
    m = synth.layered_model(20, 30, 20, config=1, name="layered 20x30x20")
    g = Sim(m)
    g.init_hydrostatic()
    g.learn_set_params(synth.learned_init(0))
    g.learn_collect(100, samples=16)
    st, rep = g.step(5 * synth.DAY)
    assert st == 0
    g.learn_collect(0)
    systems, residuals = g.learn_set_info()
    assert 0 < systems <= 100 and systems <= residuals <= 16 * systems
    first, last = g.learn_train_offline(epochs=3, lr=1e-3)
    print(f"offline set: {systems} systems, {residuals} residuals; mean loss {first:.4f} "
          f"in the first pass, {last:.4f} in the last")
    assert np.isfinite(first) and np.isfinite(last) and last < first
    dt = 5 * synth.DAY
    g.begin_step()
    g.assemble(dt)
    g.factor()
    g.learn_enable(False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st0, its0, _ = g.solve(tol=1e-3, maxit=500)
    t_plain = time.perf_counter() - t0
    g.learn_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st1, its1, _, info = g.solve(tol=1e-3, maxit=500, report=True)
    t_stage = time.perf_counter() - t0
    print(f"offline-trained stage: {its1} BiCGStab its in {1e3 * t_stage:.1f} ms "
          f"(fallback mask {info['fallback']}) vs plain ILU(0): {its0} its in "
          f"{1e3 * t_plain:.1f} ms -> {'gain' if its1 < its0 else 'loss'}")
    assert st0 == 0 and st1 == 0
    g.close()
