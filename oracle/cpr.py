"""CPR (constrained pressure residual) two-stage preconditioner with an
aggregation AMG for its pressure stage, in plain NumPy / SciPy.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` this is the slow,
readable CPU reference; only tests may import it.  Section 2.3.1 names CPR
(Wallis's two-stage method, with the decoupling of Scheichl, Masson and
Wendebourg) with algebraic multigrid for the pressure as the option beyond
ILU(0) for large cases, and leaves the details to the solver library.  The
readings taken here:

* Decoupling: the alternate block factorisation scales each cell's equations
  by the inverse of its diagonal block; only its pressure row is needed, so
  the pressure weights of cell c are w_c = D_c^-T e_p (quasi-IMPES):
  w_c^T A_cc = e_p^T, the weighted equation has no diagonal dependence on
  s_w or x.
* Pressure matrix: A_p[c, j] = w_c^T A_cj e_p on the pattern of A (unit
  diagonal), the restriction of the residual r_p[c] = w_c^T r_c.
* Pressure solve: one V-cycle of plain-aggregation AMG on A_p: strength
  |a_ij| >= theta max_k |a_ik| (k != i, theta = 0.25, symmetrised), greedy
  aggregation (seeds whose strong neighbours are all free, then attachment
  to a neighbouring aggregate, then singletons), the piecewise-constant
  prolongator P, restriction P^T, Galerkin coarse operators P^T A P, two
  damped-Jacobi sweeps (omega 2/3) before and after the coarse correction,
  an exact solve on the coarsest level (at most 200 unknowns).  A_p is a
  row-scaled, far from symmetric matrix (its rows carry the inverse diagonal
  blocks); plain aggregation keeps the coarse operators' positive diagonals
  and row diagonal dominance, which a Jacobi-smoothed prolongator lost on
  these systems (negative coarse diagonals, a divergent V-cycle).
* Two stages: x1 = E_p A_p^-1 r_p, then x = x1 + M_ILU^-1 (r - S x1), with
  S the operator the Krylov method solves (the well-reduced system) and
  M_ILU the block ILU(0) of the reservoir matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# Decoupling and the pressure system
# ---------------------------------------------------------------------------
def quasi_impes_weights(diag_blocks: np.ndarray) -> np.ndarray:
    """w[n, 3] with w_c^T D_c = e_p^T for the diagonal blocks D[n, 3, 3]
    (rows: equations, columns: unknowns, pressure first)."""
    n = diag_blocks.shape[0]
    e_p = np.zeros((n, 3, 1))
    e_p[:, 0, 0] = 1.0
    return np.linalg.solve(np.transpose(diag_blocks, (0, 2, 1)), e_p)[:, :, 0]


def pressure_matrix(rowptr, colind, vals, w) -> sp.csr_matrix:
    """A_p[c, j] = w_c^T A_cj[:, 0] for every block A_cj of the BCSR matrix."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    data = np.einsum("qe,qe->q", w[rows], vals[:, :, 0])
    return sp.csr_matrix((data, (rows, np.asarray(colind))), shape=(n, n))


def diagonal_blocks(rowptr, colind, vals) -> np.ndarray:
    n = len(rowptr) - 1
    out = np.zeros((n, 3, 3))
    for c in range(n):
        for q in range(rowptr[c], rowptr[c + 1]):
            if colind[q] == c:
                out[c] = vals[q]
    return out


# ---------------------------------------------------------------------------
# Plain-aggregation AMG
# ---------------------------------------------------------------------------
def strength(A: sp.csr_matrix, theta: float) -> sp.csr_matrix:
    """Boolean strong-connection graph: |a_ij| >= theta max_{k != i} |a_ik|."""
    A = A.tocsr()
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    off = rows != A.indices
    mag = np.abs(A.data) * off
    rowmax = np.zeros(n)
    np.maximum.at(rowmax, rows, mag)
    keep = off & (mag >= theta * rowmax[rows]) & (mag > 0)
    S = sp.csr_matrix((np.ones(keep.sum()), (rows[keep], A.indices[keep])), shape=(n, n))
    return ((S + S.T) > 0).astype(np.float64).tocsr()   # symmetrised


def aggregate(S: sp.csr_matrix) -> np.ndarray:
    """Aggregate index of every node (three greedy passes over the strong graph)."""
    n = S.shape[0]
    agg = -np.ones(n, dtype=np.int64)
    nagg = 0
    nbrs = [S.indices[S.indptr[i]:S.indptr[i + 1]] for i in range(n)]
    for i in range(n):                       # pass 1: free node with all-free strong neighbours
        if agg[i] < 0 and np.all(agg[nbrs[i]] < 0):
            agg[i] = nagg
            agg[nbrs[i]] = nagg
            nagg += 1
    for i in range(n):                       # pass 2: join a neighbouring aggregate
        if agg[i] < 0:
            joined = nbrs[i][agg[nbrs[i]] >= 0]
            if len(joined):
                agg[i] = agg[joined[0]]
    for i in range(n):                       # pass 3: what is left stands alone
        if agg[i] < 0:
            agg[i] = nagg
            nagg += 1
    return agg


def transmissibility_laplacian(Tx, Ty, Tz, nx, ny, nz) -> sp.csr_matrix:
    """The graph Laplacian of the face transmissibilities (T of the +x, +y,
    +z face of each cell, natural order), with a tiny diagonal shift."""
    n = nx * ny * nz
    c = np.arange(n)
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    rows, cols, vals = [], [], []
    for T, off, inside in ((Tx, 1, i < nx - 1), (Ty, nx, j < ny - 1), (Tz, nx * ny, k < nz - 1)):
        cc = c[inside]
        rows += [cc, cc + off]
        cols += [cc + off, cc]
        vals += [-np.asarray(T)[cc], -np.asarray(T)[cc]]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    d = -np.asarray(A.sum(axis=1)).ravel()
    return (A + sp.diags(d * (1.0 + 1e-12) + 1e-300)).tocsr()


class AMG:
    """Plain-aggregation hierarchy of A and its V-cycle.  With ``prolongators``
    the aggregation is not recomputed: the given piecewise-constant maps (for
    example the hierarchy of the transmissibility Laplacian, built once per
    model) carry A's Galerkin coarse operators."""

    def __init__(self, A, theta=0.25, coarse_size=200, max_levels=12, nu=2, omega=2.0 / 3.0,
                 prolongators=None):
        self.nu, self.omega = nu, omega
        self.A, self.P, self.dinv = [], [], []
        A = sp.csr_matrix(A)
        if prolongators is not None:
            for P in prolongators:
                self.A.append(A)
                self.dinv.append(1.0 / A.diagonal())
                self.P.append(P)
                A = (P.T @ A @ P).tocsr()
            self.A.append(A)
            self.dinv.append(1.0 / A.diagonal())
            self.coarse = np.linalg.inv(A.toarray())
            return
        while True:
            self.A.append(A)
            self.dinv.append(1.0 / A.diagonal())
            if A.shape[0] <= coarse_size or len(self.A) == max_levels:
                break
            agg = aggregate(strength(A, theta))
            nc = int(agg.max()) + 1
            if nc >= A.shape[0]:
                break
            P = sp.csr_matrix((np.ones(A.shape[0]), (np.arange(A.shape[0]), agg)),
                              shape=(A.shape[0], nc))
            self.P.append(P)
            A = (P.T @ A @ P).tocsr()
        self.coarse = np.linalg.inv(self.A[-1].toarray())

    def _jacobi(self, lvl, x, b):
        A, dinv = self.A[lvl], self.dinv[lvl]
        for _ in range(self.nu):
            x = x + self.omega * dinv * (b - A @ x)
        return x

    def vcycle(self, b, lvl=0):
        if lvl == len(self.A) - 1:
            return self.coarse @ b
        x = self._jacobi(lvl, np.zeros_like(b), b)
        r = b - self.A[lvl] @ x
        x = x + self.P[lvl] @ self.vcycle(self.P[lvl].T @ r, lvl + 1)
        return self._jacobi(lvl, x, b)


# ---------------------------------------------------------------------------
# The two-stage preconditioner and a right-preconditioned BiCGStab
# ---------------------------------------------------------------------------
class CPR:
    """z = x1 + M2^-1 (r - S x1), x1 = E_p P1^-1 (W^T r) on cell-major 3-vectors."""

    def __init__(self, rowptr, colind, vals, op, second_stage, pressure_solve=None):
        self.w = quasi_impes_weights(diagonal_blocks(rowptr, colind, vals))
        self.Ap = pressure_matrix(rowptr, colind, vals, self.w)
        self.op = op
        self.second = second_stage
        self.psolve = pressure_solve if pressure_solve is not None else AMG(self.Ap).vcycle

    def first_stage(self, r):
        rp = np.einsum("ce,ce->c", self.w, r.reshape(-1, 3))
        x1 = np.zeros((len(rp), 3))
        x1[:, 0] = self.psolve(rp)
        return x1.reshape(-1)

    def __call__(self, r):
        x1 = self.first_stage(r)
        return x1 + self.second(r - self.op(x1))


def bicgstab(op, b, precond, tol=1e-3, maxit=1000):
    """Right-preconditioned BiCGStab (van der Vorst): returns (x, iterations,
    converged); stops when ||b - op x|| <= tol ||b|| (recurrence residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    rhat = r.copy()
    nb = np.linalg.norm(b)
    rho = alpha = omega = 1.0
    v = p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        ph = precond(p)
        v = op(ph)
        alpha = rho / (rhat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * nb:
            return x + alpha * ph, it, True
        sh = precond(s)
        t = op(sh)
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        if np.linalg.norm(r) <= tol * nb:
            return x, it, True
    return x, maxit, False
