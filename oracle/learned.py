"""CPU FP64 oracle of the learned preconditioner stage (NumPy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the plain reference
that the GPU kernels of the learned stage are checked against.  It shares no
code with the CUDA path.

The stage corrects the ILU(0) preconditioner of the linear solver (Section
2.3.1 of arXiv 1910.06059: BiCGStab preconditioned by ILU(0)) with a small
per-cell network that reads the cell's row of the Jacobian and returns a
3x3 matrix acting on the cell's residual:

    z = M^-1 r + delta(r),   delta_c = sigma_c * (W_c rhat_c),   W_c = N(f_c)

N is a two-hidden-layer MLP (63 -> 128 -> 128 -> 9, ReLU), f_c the 63
normalised entries of the cell's Jacobian row (diagonal block and six
neighbour blocks), rhat_c the row-scaled residual.  The correction is linear
in r, so for a given Jacobian the whole preconditioner is one fixed linear
map, as BiCGStab requires.  Definitions (the GPU kernels implement the same):

* unknown scales sigma_c = (1e6 Pa, 0.05, 0.05) for a saturated cell (x = s_g)
  and (1e6 Pa, 0.05, 5) for an undersaturated one (x = r_go);
* equation scales rho_{c,e} = max_v |A_cc[e][v]| sigma_{c,v};
* block features F_{c,b}[e][v] = A_{c,b}[e][v] sigma_{nb,v} / rho_{c,e} for the
  diagonal (b = 0, nb = c) and the six neighbours -x, +x, -y, +y, -z, +z
  (zero where the neighbour is missing);
* rhat_c[e] = r_c[e] / rho_{c,e}; W_c[v][e] = N(f_c)[3 v + e].

Training minimises, per sample (A, r), the squared residual of the corrected
preconditioner against the reservoir Jacobian A:

    L = || e - A delta ||^2 / ||r||^2,   e = r - A M^-1 r

and its gradient is back-propagated through delta by A^T.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 128
NFEAT = 63
NOUT = 9
SIGMA_P, SIGMA_S, SIGMA_SG, SIGMA_RGO = 1e6, 0.05, 0.05, 5.0

# parameter tensors in the order of the flat parameter vector
PARAM_SHAPES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
                ("b2", (HIDDEN,)), ("W3", (NOUT, HIDDEN)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


def unflatten(theta):
    """Flat parameter vector -> dict of views."""
    out, off = {}, 0
    for name, shape in PARAM_SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + k]).reshape(shape)
        off += k
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).reshape(-1)
                           for name, _ in PARAM_SHAPES])


# ---------------------------------------------------------------------------
# Jacobian in the seven-block layout (diagonal, -x, +x, -y, +y, -z, +z)
# ---------------------------------------------------------------------------
def neighbours(nx, ny, nz):
    """(n, 7) neighbour index per direction, -1 where missing."""
    n = nx * ny * nz
    c = np.arange(n)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    nb = np.full((n, 7), -1, dtype=np.int64)
    nb[:, 0] = c
    nb[i > 0, 1] = c[i > 0] - 1
    nb[i < nx - 1, 2] = c[i < nx - 1] + 1
    nb[j > 0, 3] = c[j > 0] - nx
    nb[j < ny - 1, 4] = c[j < ny - 1] + nx
    nb[k > 0, 5] = c[k > 0] - nx * ny
    nb[k < nz - 1, 6] = c[k < nz - 1] + nx * ny
    return nb


def blocks7(rowptr, colind, vals, nx, ny, nz):
    """BCSR (rowptr, colind, vals[nnzb,3,3]) -> A7[n, 7, 3, 3]."""
    nb = neighbours(nx, ny, nz)
    n = nb.shape[0]
    A7 = np.zeros((n, 7, 3, 3))
    for c in range(n):
        for q in range(rowptr[c], rowptr[c + 1]):
            b = int(np.nonzero(nb[c] == colind[q])[0][0])
            A7[c, b] = vals[q]
    return A7


def apply_A(A7, nb, x):
    """y = A x for x[n, 3]."""
    y = np.zeros_like(x)
    for b in range(7):
        ok = nb[:, b] >= 0
        y[ok] += np.einsum("cij,cj->ci", A7[ok, b], x[nb[ok, b]])
    return y


def apply_AT(A7, nb, x):
    """y = A^T x for x[n, 3]: the transpose of block (c, nb) scatters to nb."""
    y = np.zeros_like(x)
    for b in range(7):
        ok = np.nonzero(nb[:, b] >= 0)[0]
        np.add.at(y, nb[ok, b], np.einsum("cji,cj->ci", A7[ok, b], x[ok]))
    return y


# ---------------------------------------------------------------------------
# Features and the network
# ---------------------------------------------------------------------------
def sigma(flag):
    """Unknown scales per cell; flag 0 = saturated (x = s_g), 1 = undersaturated."""
    s = np.empty((len(flag), 3))
    s[:, 0] = SIGMA_P
    s[:, 1] = SIGMA_S
    s[:, 2] = np.where(np.asarray(flag) == 0, SIGMA_SG, SIGMA_RGO)
    return s


def scales(A7, flag):
    """(sigma[n,3], rho[n,3]) as defined in the module docstring."""
    sg = sigma(flag)
    rho = np.max(np.abs(A7[:, 0]) * sg[:, None, :], axis=2)
    return sg, rho


def block_features(A7, nb, flag):
    """[n, 63]: the seven normalised blocks, row-major, diagonal first."""
    sg, rho = scales(A7, flag)
    n = A7.shape[0]
    F = np.zeros((n, 7, 3, 3))
    for b in range(7):
        ok = nb[:, b] >= 0
        F[ok, b] = A7[ok, b] * sg[nb[ok, b]][:, None, :] / rho[ok][:, :, None]
    return F.reshape(n, 63)


def mlp_forward(params, F):
    """o[n, 9] and the activations needed by the backward pass."""
    a1 = F @ params["W1"].T + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ params["W3"].T + params["b3"]
    return o, (F, a1, h1, a2, h2)


def mlp_backward(params, cache, do):
    """Parameter gradients for the upstream gradient do[n, 9]."""
    F, a1, h1, a2, h2 = cache
    grads = {"W3": do.T @ h2, "b3": do.sum(0)}
    dh2 = (do @ params["W3"]) * (a2 > 0)
    grads["W2"] = dh2.T @ h1
    grads["b2"] = dh2.sum(0)
    dh1 = (dh2 @ params["W2"]) * (a1 > 0)
    grads["W1"] = dh1.T @ F
    grads["b1"] = dh1.sum(0)
    return grads


def cell_matrices(params, A7, nb, flag):
    """W[n, 3, 3] = N(f) per cell."""
    o, _ = mlp_forward(params, block_features(A7, nb, flag))
    return o.reshape(-1, 3, 3)


def stage_delta(params, A7, nb, flag, r):
    """delta[n, 3] = sigma * (W rhat)."""
    sg, rho = scales(A7, flag)
    W = cell_matrices(params, A7, nb, flag)
    return sg * np.einsum("cve,ce->cv", W, r / rho)


def loss_and_grad(params, A7, nb, flag, r, z0):
    """(L, grads) for one sample: residual r[n,3], ILU(0) result z0 = M^-1 r."""
    sg, rho = scales(A7, flag)
    o, cache = mlp_forward(params, block_features(A7, nb, flag))
    W = o.reshape(-1, 3, 3)
    rhat = r / rho
    delta = sg * np.einsum("cve,ce->cv", W, rhat)
    e = r - apply_A(A7, nb, z0)
    u = e - apply_A(A7, nb, delta)
    rr = float(np.sum(r * r))
    L = float(np.sum(u * u)) / rr
    ddelta = -2.0 * apply_AT(A7, nb, u) / rr
    dW = np.einsum("cv,ce->cve", sg * ddelta, rhat)
    return L, mlp_backward(params, cache, dW.reshape(-1, 9))
