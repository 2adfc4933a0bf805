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
