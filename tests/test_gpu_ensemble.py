"""Batched ensembles on the GPU (bo_ensemble_*, through the C ABI).

Members stepped together must reach exactly the states they reach when
stepped alone (same kernels, same decisions per member; the concurrency only
interleaves independent work), one member is checked against the oracle,
and the autotuner must leave every member's state as it found it.
"""
from __future__ import annotations

import time

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


def small_members(k=6, pool=40):
    """The k smallest of the first `pool` ensemble members (uneven sizes)."""
    ms = [synth.config3_member(q) for q in range(pool)]
    ms.sort(key=lambda m: m["nx"] * m["ny"] * m["nz"])
    return ms[:k]


def test_ensemble_equals_members_stepped_alone():
    from paper_1910_06059_gb300 import Ensemble, Sim
    models = small_members(6)
    ens = Ensemble(models, streams=3)
    ens.init_hydrostatic()
    alone = [Sim(m) for m in models]
    for s in alone:
        s.init_hydrostatic()
    for days in (1.0, 3.0):
        t0 = time.perf_counter()
        sts, reps = ens.step(days * synth.DAY)
        host_ms = 1e3 * (time.perf_counter() - t0)
        assert all(st == 0 for st in sts)
        # the step's device time (events bracketing every worker stream) is
        # measured and lies within the host's view of the same call
        ms = ens.last_step_ms()
        assert 0.0 < ms <= host_ms
        for q, s in enumerate(alone):
            st, rep = s.step(days * synth.DAY)
            assert st == 0
            assert (rep["newton_its"], rep["lin_its"], rep["substeps"]) == \
                (reps[q]["newton_its"], reps[q]["lin_its"], reps[q]["substeps"])
            for a, b in zip(ens.members[q].get_state(), s.get_state()):
                assert np.array_equal(a, b)
    ens.close()


def test_ensemble_with_member_timers():
    """Members timed while the workers step them concurrently: each member
    keeps its own open intervals, and every member's timers are filled."""
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(6)
    ens = Ensemble(models, streams=3)
    ens.init_hydrostatic()
    for sm in ens.members:
        sm.set_timing(True)
    sts, reps = ens.step(1.0 * synth.DAY)
    assert all(st == 0 for st in sts)
    for sm, rep in zip(ens.members, reps):
        t = sm.timing()
        assert t["ilu_fwd_sweep"][1] >= rep["lin_its"] > 0
        assert all(np.isfinite(v[0]) and v[0] >= 0 for v in t.values())
        sm.set_timing(False)
    ens.close()


def test_ensemble_member_vs_oracle():
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(3)
    ens = Ensemble(models, streams=3)
    ens.init_hydrostatic()
    o = oracle.Oracle(models[0])
    o.init_hydrostatic()
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10)
    for days in (0.5, 1.0):
        sts, reps = ens.step(days * synth.DAY, **tight)
        st_o, rep_o = o.step(days * synth.DAY, **tight)
        assert sts[0] == 0 and st_o == 0
        assert reps[0]["substeps"] == rep_o["substeps"]
        pg, swg, xg, fg, bg = ens.members[0].get_state()
        po, swo, xo, fo, bo = o.get_state()
        assert np.array_equal(fg, fo)
        assert np.max(np.abs(pg - po) / po) <= 1e-6
        assert np.max(np.abs(swg - swo)) <= 1e-6
    ens.close()


def test_autotune_restores_every_member():
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(5)
    ens = Ensemble(models, streams=1)
    ens.init_hydrostatic()
    ens.step(0.5 * synth.DAY)
    before = [s.get_state() for s in ens.members]
    dt_before = [s.dt_next for s in ens.members]
    res = ens.autotune(0.2 * synth.DAY, candidates=(1, 2, 5))
    assert res["chosen"]["streams"] in (1, 2, 5)
    assert all(t > 0 for t in res["largest_first"].values())
    for s, b, d in zip(ens.members, before, dt_before):
        for x, y in zip(s.get_state(), b):
            assert np.array_equal(x, y)
        assert s.dt_next == d
    ens.close()


def test_autotune_precond_per_size_class():
    """The preconditioner choice per size class probes all four combinations,
    puts every member back as it was after each probe, sets the chosen
    preconditioner on each member by its class, and the ensemble then steps
    (a member under CPR still matches the oracle's state)."""
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(6)
    ens = Ensemble(models, streams=3)
    ens.init_hydrostatic()
    ens.step(0.5 * synth.DAY)
    before = [s.get_state() for s in ens.members]
    dt_before = [s.dt_next for s in ens.members]
    res = ens.autotune_precond(0.2 * synth.DAY)
    assert len(res["probe_s"]) == 4 and all(t > 0 for t in res["probe_s"].values())
    sizes = sorted(s.n for s in ens.members)
    median = sizes[(len(sizes) - 1) // 2]
    for s, b, d in zip(ens.members, before, dt_before):
        for x, y in zip(s.get_state(), b):
            assert np.array_equal(x, y)
        assert s.dt_next == d
        want = res["chosen"]["small"] if s.n <= median else res["chosen"]["large"]
        assert s.preconditioner == want
    # every member through CPR for one report step against the oracle
    for s in ens.members:
        s.preconditioner = "cpr"
    orc = [oracle.Oracle(m) for m in models]
    for o, s in zip(orc, ens.members):
        o.set_state(*s.get_state())
        o.dt_next = s.dt_next
    tight = dict(tol_mb=1e-10, tol_cnv=1e-10, tol_well=1e-10, tol_lin=1e-10)
    sts, _ = ens.step(1.0 * synth.DAY, **tight)
    assert all(st == 0 for st in sts)
    for o, s in zip(orc, ens.members):
        st, _ = o.step(1.0 * synth.DAY, **tight)
        assert st == 0
        pg, pgo = s.get_state()[0], o.get_state()[0]
        assert np.max(np.abs(pg - pgo) / pgo) <= 1e-6
    ens.close()


def test_failing_members_are_reported_and_restored():
    """A Newton budget of zero with no cuts fails every member: the step
    reports each failure and leaves each member at the start of the step."""
    from paper_1910_06059_gb300 import Ensemble
    models = small_members(4)
    ens = Ensemble(models, streams=2)
    ens.init_hydrostatic()
    before = [s.get_state() for s in ens.members]
    sts, reps = ens.step(1.0 * synth.DAY, raise_on_fail=False, max_newton=0, max_cuts=0)
    assert all(st == 4 for st in sts)      # BO_ERR_NOT_CONVERGED
    for s, b in zip(ens.members, before):
        for x, y in zip(s.get_state(), b):
            assert np.array_equal(x, y)
    ens.close()
