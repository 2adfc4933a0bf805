"""The allocation-free convergence measures (bo_residual_norms_noalloc) agree
with bo_norms.

This entry point is for callers that cannot allocate device memory: it takes
the residual, pore volumes and shrinkage factors in the caller's own device
buffers and keeps its partial sums in a fixed array inside the library.  The
test calls it twice in a row through the C ABI (the second call reuses the
array the first one left behind) and compares both results with bo_norms at
the tolerance of the assembly parity tests.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1910_06059_gb300.build import build
    build()


def _close(got, ref, R, pv):
    # CNV: a maximum, compared entry by entry
    assert np.allclose(got[3:], ref[3:], rtol=1e-12, atol=0)
    # MB: a cancelling sum, bounded as in the assembly parity test
    factor = ref[3:6] / (np.abs(R) / pv[:, None]).max(axis=0) / pv.sum()
    assert np.all(np.abs(got[:3] - ref[:3]) <= 1e-12 * factor * np.abs(R).sum(axis=0) + 1e-15 * ref[:3])


def test_noalloc_norms_match_bo_norms_twice():
    from paper_1910_06059_gb300 import Sim, _lib
    m = synth.small_model(33, 17, 9, wells="5spot", dz=3.0)   # 5049 cells: three blocks
    g = Sim(m)
    st = synth.random_state(m, seed_member=3)
    g.set_state(*st)
    g.begin_step()
    g.set_state(st[0] * 1.003, st[1] + 0.004, *st[2:])
    dt = 3 * synth.DAY
    g.assemble(dt)
    ref = g.norms(dt)
    _, _, _, R = g.system()                  # [n, 3] cell-major
    pv = g.get_static()["pv"]
    f = m["fluid"]
    p, sw, x, fl, _ = g.get_state()
    b = np.empty((3, g.n))
    for c in range(g.n):
        cp = oracle.cell_props(f, p[c], sw[c], x[c], fl[c])
        b[0, c], b[1, c], b[2, c] = cp["b_w"][0], cp["b_o"][0], cp["b_g"][0]
    dev = torch.device("cuda", 0)
    R_d = torch.from_numpy(np.ascontiguousarray(R.T)).to(dev)
    pv_d = torch.from_numpy(pv).to(dev)
    b_d = torch.from_numpy(b).to(dev)
    out = torch.zeros(6, dtype=torch.float64, device=dev)
    lib = _lib.load()
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        st_ = lib.bo_residual_norms_noalloc(_lib.ptr(R_d), _lib.ptr(pv_d), _lib.ptr(b_d), g.n,
                                            ctypes.c_double(dt), _lib.ptr(out), None)
        assert st_ == 0, lib.bo_last_error().decode()
        torch.cuda.synchronize()
        _close(out.cpu().numpy(), ref[:6], R, pv)


def test_noalloc_norms_reject_oversize():
    from paper_1910_06059_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(6, dtype=torch.float64, device=dev)
    st_ = lib.bo_residual_norms_noalloc(_lib.ptr(buf), _lib.ptr(buf), _lib.ptr(buf), 8_388_609,
                                        ctypes.c_double(1.0), _lib.ptr(buf), None)
    assert st_ == 1  # BO_ERR_INVALID_ARG, nothing launched
    assert b"exceeds the maximum" in lib.bo_last_error()
