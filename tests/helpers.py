"""Shared helpers for the test suite: model construction and comparison metrics."""
from __future__ import annotations

import numpy as np

import synth
from synth.models import _base, _well  # noqa: F401  (model layout helpers)


def make_model(nx, ny, nz, perm, poro, wells, fluid=None, dx=10.0, dy=10.0, dz=2.0,
               init=None, dt=synth.DAY):
    m = _base("test", nx, ny, nz, dx, dy, dz, np.asarray(perm, float) * np.ones(nx * ny * nz),
              np.asarray(poro, float) * np.ones(nx * ny * nz), wells, 1, dt)
    if fluid:
        m["fluid"].update(fluid)
    if init:
        m["init"].update(init)
    return m


def bcsr_to_dense(rowptr, colind, vals, n):
    A = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for q in range(rowptr[i], rowptr[i + 1]):
            j = colind[q]
            A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = vals[q]
    return A


def entrywise_rel_ok(a, b, rel, floor_rows=None):
    """|a - b| <= rel * max(|b|, 1e-3 * row_inf_norm(b)) entry by entry.

    Entries that cancel to near zero are judged against the size of their
    block row instead of their own size.
    """
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if floor_rows is None:
        floor_rows = np.max(np.abs(b), axis=-1, keepdims=True)
    scale = np.maximum(np.abs(b), 1e-3 * floor_rows)
    scale = np.where(scale == 0, 1.0, scale)
    err = np.abs(a - b) / scale
    return err.max() <= rel, float(err.max())


def family_close(a, b, rowptr, per_equation=True):
    """Max relative error of Jacobian-like blocks (nnzb, 3, 3).  Each entry
    J[r][s] is judged against max(|oracle|, 1e-3 * the largest |J[r][s]| over
    the blocks of its block row), i.e. against entries of the same equation
    and the same unknown family (pressure columns are per Pa, the others are
    dimensionless).  per_equation=False floors over all three equations."""
    a = np.asarray(a)
    b = np.asarray(b)
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    absb = np.abs(b)
    fam = np.zeros((n, 3, 3))
    np.maximum.at(fam, rows, absb)
    if not per_equation:
        fam = np.broadcast_to(fam.max(axis=1, keepdims=True), fam.shape)
    scale = np.maximum(absb, 1e-3 * fam[rows])
    scale = np.where(scale == 0, 1.0, scale)
    return float((np.abs(a - b) / scale).max())


def vec_close(a, b):
    """max |a - b| relative to max |b|."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
