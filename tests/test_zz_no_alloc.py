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


def _norms_ref(R, pv, b, dt):
    """MB and CNV in float64 NumPy, the definition of bo_norms (Section 2.3
    convergence measures) written out: independent of both GPU paths."""
    n = pv.size
    bavg = (1.0 / b).sum(axis=1) / n
    mb = dt * bavg * np.abs(R.sum(axis=1)) / pv.sum()
    cnv = dt * bavg * (np.abs(R) / pv[None, :]).max(axis=1)
    return np.concatenate([mb, cnv])


def _call(lib, _lib, R_d, pv_d, b_d, n, dt, out, stream=None):
    st_ = lib.bo_residual_norms_noalloc(_lib.ptr(R_d), _lib.ptr(pv_d), _lib.ptr(b_d), n,
                                        ctypes.c_double(dt), _lib.ptr(out), stream)
    assert st_ == 0, lib.bo_last_error().decode()


def test_noalloc_sizes_stream_memory_and_nan():
    """A call with fewer blocks after one with more ignores the leftover
    partials; a call on a non-null stream agrees; free device memory is the
    same before and after warm calls; a NaN residual entry gives NaN."""
    from paper_1910_06059_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(21)
    dt = 2.5 * synth.DAY
    cases = []
    for n in (40_000, 3_000):   # 20 blocks, then 2 blocks
        R = rng.standard_normal((3, n)) * np.array([[1e-3], [2e-3], [5e-1]])
        pv = rng.uniform(5.0, 50.0, n)
        b = rng.uniform(0.8, 1.2, (3, n)) * np.array([[1.0], [1.1], [90.0]])
        cases.append((n, R, pv, b))
    dev_bufs = [(n, torch.from_numpy(R).to(dev), torch.from_numpy(pv).to(dev),
                 torch.from_numpy(b).to(dev), R, pv, b) for n, R, pv, b in cases]
    outs = [torch.full((6,), -1.0, dtype=torch.float64, device=dev) for _ in cases]
    side = torch.cuda.Stream()
    n0, R0_d, pv0_d, b0_d, *_ = dev_bufs[0]
    warm = torch.zeros(6, dtype=torch.float64, device=dev)
    _call(lib, _lib, R0_d, pv0_d, b0_d, n0, dt, warm)   # the first call loads the module
    torch.cuda.synchronize()
    # only library calls between the two readings (torch's own kernels load lazily too)
    free0, _ = torch.cuda.mem_get_info()
    for k, (n, R_d, pv_d, b_d, *_rest) in enumerate(dev_bufs):
        if k == 1:
            _call(lib, _lib, R_d, pv_d, b_d, n, dt, outs[k], ctypes.c_void_p(side.cuda_stream))
            side.synchronize()
        else:
            _call(lib, _lib, R_d, pv_d, b_d, n, dt, outs[k])
            torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for k, (n, R_d, pv_d, b_d, R, pv, b) in enumerate(dev_bufs):
        ref = _norms_ref(R, pv, b, dt)
        got = outs[k].cpu().numpy()
        assert np.allclose(got[3:], ref[3:], rtol=1e-12, atol=0), (k, got, ref)
        # MB: a cancelling sum, rounding bounded by the sum of magnitudes
        bound = 1e-12 * dt * (1.0 / b).mean(axis=1) * np.abs(R).sum(axis=1) / pv.sum()
        assert np.all(np.abs(got[:3] - ref[:3]) <= bound + 1e-15 * ref[:3]), (k, got, ref)
    # NaN in one residual entry: MB and CNV of its component are NaN
    n, R_d, pv_d, b_d, *_ = dev_bufs[1]
    R_nan = R_d.clone()
    R_nan[1, n // 2] = float("nan")
    out = torch.zeros(6, dtype=torch.float64, device=dev)
    _call(lib, _lib, R_nan, pv_d, b_d, n, dt, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isnan(got[1]) and np.isnan(got[4]), got
    assert np.all(np.isfinite(got[[0, 2, 3, 5]])), got


def test_noalloc_norms_reject_oversize():
    from paper_1910_06059_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(6, dtype=torch.float64, device=dev)
    st_ = lib.bo_residual_norms_noalloc(_lib.ptr(buf), _lib.ptr(buf), _lib.ptr(buf), 8_388_609,
                                        ctypes.c_double(1.0), _lib.ptr(buf), None)
    assert st_ == 1  # BO_ERR_INVALID_ARG, nothing launched
    assert b"exceeds the maximum" in lib.bo_last_error()
