"""Pins of the learned-stage oracle (oracle/learned.py) against facts that do
not depend on it: a dense Jacobian and its transpose, the normalisation
identities of the features, homogeneity of the stage, a least-squares closed
form for the output bias, and central finite differences of the loss."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from oracle import learned as ML
from tests.helpers import bcsr_to_dense


@pytest.fixture(scope="module")
def system():
    m = synth.small_model(5, 4, 3, wells="5spot", dz=3.0)
    o = oracle.Oracle(m)
    st = synth.random_state(m, seed_member=4, frac_sat=0.5)
    o.set_state(*st)
    o.begin_step()
    o.assemble(0.5 * synth.DAY)
    rp, ci, v, R = o.system()
    nb = ML.neighbours(m["nx"], m["ny"], m["nz"])
    A7 = ML.blocks7(rp, ci, v, m["nx"], m["ny"], m["nz"])
    o.ilu0()
    return dict(o=o, m=m, rp=rp, ci=ci, v=v, R=R, nb=nb, A7=A7, flag=np.asarray(st[3]),
                dense=bcsr_to_dense(rp, ci, v, o.n))


def random_params(seed, out_scale=0.1):
    p = ML.unflatten(synth.learned_init(seed).copy())
    rng = np.random.default_rng(seed + 100)
    p["W3"] = out_scale * rng.standard_normal(p["W3"].shape)
    p["b3"] = out_scale * rng.standard_normal(ML.NOUT)
    p["b1"] = 0.1 * rng.standard_normal(128)
    p["b2"] = 0.1 * rng.standard_normal(128)
    return p


def test_seven_block_operator_and_transpose(system):
    n = system["o"].n
    x = np.random.default_rng(1).standard_normal((n, 3))
    D = system["dense"]
    y = ML.apply_A(system["A7"], system["nb"], x).reshape(-1)
    yt = ML.apply_AT(system["A7"], system["nb"], x).reshape(-1)
    assert np.allclose(y, D @ x.reshape(-1), rtol=1e-13, atol=1e-13 * np.abs(D).max() * np.abs(x).max())
    assert np.allclose(yt, D.T @ x.reshape(-1), rtol=1e-13, atol=1e-13 * np.abs(D).max() * np.abs(x).max())


def test_feature_normalisation(system):
    A7, nb, flag = system["A7"], system["nb"], system["flag"]
    F = ML.block_features(A7, nb, flag).reshape(-1, 7, 3, 3)
    # each row of the scaled diagonal block has largest magnitude exactly 1
    assert np.allclose(np.abs(F[:, 0]).max(axis=2), 1.0, rtol=0, atol=1e-15)
    # one entry by hand: cell 7, neighbour +y (block 4), equation 2, unknown 1
    c, b, e, v = 7, 4, 2, 1
    j = nb[c, b]
    sig_c = [1e6, 0.05, 0.05 if flag[c] == 0 else 5.0]
    sig_j = [1e6, 0.05, 0.05 if flag[j] == 0 else 5.0]
    rho = max(abs(A7[c, 0, e, w]) * sig_c[w] for w in range(3))
    assert F[c, b, e, v] == pytest.approx(A7[c, b, e, v] * sig_j[v] / rho, rel=1e-14)
    # a missing neighbour (cell 0 has no -x, -y, -z) gives zero blocks
    assert np.all(F[0, [1, 3, 5]] == 0.0)


def test_stage_is_linear_in_the_residual(system):
    p = random_params(3)
    rng = np.random.default_rng(2)
    r1 = rng.standard_normal((system["o"].n, 3)) * [1e-3, 1e-2, 1.0]
    r2 = rng.standard_normal((system["o"].n, 3)) * [1e-3, 1e-2, 1.0]
    args = (system["A7"], system["nb"], system["flag"])
    d = ML.stage_delta(p, *args, 3.7 * r1 - 1.5 * r2)
    assert np.allclose(d, 3.7 * ML.stage_delta(p, *args, r1) - 1.5 * ML.stage_delta(p, *args, r2),
                       rtol=1e-12, atol=1e-12 * np.abs(d).max())
    assert np.all(ML.stage_delta(p, *args, 0 * r1) == 0)
    # one cell by hand: delta_c[v] = sigma_v sum_e N(f_c)[3 v + e] r_c[e] / rho_c[e]
    c = 11
    F = ML.block_features(*args)
    h1 = np.maximum(p["W1"] @ F[c] + p["b1"], 0)
    h2 = np.maximum(p["W2"] @ h1 + p["b2"], 0)
    out = p["W3"] @ h2 + p["b3"]
    sg, rho = ML.scales(system["A7"], system["flag"])
    want = [sg[c, v] * sum(out[3 * v + e] * r1[c, e] / rho[c, e] for e in range(3)) for v in range(3)]
    assert np.allclose(ML.stage_delta(p, *args, r1)[c], want, rtol=1e-12, atol=0)


def test_untrained_stage_is_plain_ilu0(system):
    o, A7, nb, flag = system["o"], system["A7"], system["nb"], system["flag"]
    p = ML.unflatten(synth.learned_init(0).copy())
    r = system["R"].copy()
    z0 = o.ilu_apply(r.reshape(-1)).reshape(-1, 3)
    assert np.all(ML.stage_delta(p, A7, nb, flag, r) == 0)
    L, g = ML.loss_and_grad(p, A7, nb, flag, r, z0)
    e = r.reshape(-1) - system["dense"] @ z0.reshape(-1)
    assert L == pytest.approx(e @ e / np.sum(r * r), rel=1e-12)
    # with a zero output layer only the output layer receives gradient
    for k in ("W1", "b1", "W2", "b2"):
        assert np.all(g[k] == 0)
    assert np.abs(g["W3"]).max() > 0


def test_output_bias_least_squares(system):
    """W1 = W2 = 0 and zero hidden biases: every cell gets the same matrix
    W = b3 (3x3), so delta = sigma (W rhat) is linear in the nine entries of
    b3 and L(b3) is a linear least-squares problem; its minimiser (numpy's
    lstsq on the dense Jacobian) zeroes the gradient."""
    o, A7, nb, flag = system["o"], system["A7"], system["nb"], system["flag"]
    D = system["dense"]
    p = ML.unflatten(np.zeros(ML.NPARAM))
    r = system["R"].copy()
    z0 = o.ilu_apply(r.reshape(-1)).reshape(-1, 3)
    sg, rho = ML.scales(A7, flag)
    rhat = r / rho
    G = np.zeros((3 * o.n, 9))
    for v in range(3):
        for e in range(3):
            x = np.zeros((o.n, 3))
            x[:, v] = sg[:, v] * rhat[:, e]
            G[:, 3 * v + e] = D @ x.reshape(-1)
    e = r.reshape(-1) - D @ z0.reshape(-1)
    b3, *_ = np.linalg.lstsq(G, e, rcond=None)
    p["b3"] = b3
    L, grads = ML.loss_and_grad(p, A7, nb, flag, r, z0)
    res = e - G @ b3
    assert L == pytest.approx(res @ res / np.sum(r * r), rel=1e-10)
    scale = np.abs(G).max() * np.abs(e).max() / np.sum(r * r)
    assert np.abs(grads["b3"]).max() <= 1e-9 * scale


def test_gradient_matches_central_differences(system):
    o, A7, nb, flag = system["o"], system["A7"], system["nb"], system["flag"]
    p = random_params(5, out_scale=0.3)
    rng = np.random.default_rng(9)
    r = system["R"] * (1 + 0.1 * rng.standard_normal(system["R"].shape))
    z0 = o.ilu_apply(r.reshape(-1)).reshape(-1, 3)
    L0, grads = ML.loss_and_grad(p, A7, nb, flag, r, z0)
    theta = ML.flatten(p)
    gflat = ML.flatten(grads)
    idx = rng.choice(ML.NPARAM, 40, replace=False)
    # make sure every tensor is sampled
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in ML.PARAM_SHAPES])
    idx = np.concatenate([idx, offs[:-1] + 1])
    gnorm = np.abs(gflat).max()
    for q in idx:
        h = 1e-6 * max(1.0, abs(theta[q]))
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        Lp, _ = ML.loss_and_grad(ML.unflatten(tp), A7, nb, flag, r, z0)
        Lm, _ = ML.loss_and_grad(ML.unflatten(tm), A7, nb, flag, r, z0)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gflat[q]) <= 1e-6 * gnorm + 1e-5 * abs(gflat[q]), (q, fd, gflat[q])
