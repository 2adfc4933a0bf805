"""The oracle's host threads change its speed, not its results.

The CPU baseline times the oracle on one thread and on all host cores.  The
loops that run on several threads have independent iterations and every
floating-point sum keeps its sequential order, so the system, the norms, the
linear solve and the states after two report steps must be bit for bit the
same on 1 and 4 threads.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth


def _run(m, threads):
    oracle.set_threads(threads)
    try:
        o = oracle.Oracle(m)
        o.init_hydrostatic()
        o.begin_step()
        o.assemble(m["dt"])
        out = list(o.system()) + [o.norms(m["dt"])]
        st, its, sol = o.solve(tol=1e-8, maxit=200)
        out += [np.asarray([st, its]), sol]
        for _ in range(2):
            o.step(m["dt"])
        out += [np.asarray(a) for a in o.get_state()]
        return out
    finally:
        oracle.set_threads(1)


def test_threads_do_not_change_results():
    m = synth.layered_model(12, 16, 9, config=1, name="layered 12x16x9")
    one = _run(m, 1)
    four = _run(m, 4)
    assert len(one) == len(four)
    for a, b in zip(one, four):
        assert np.array_equal(a, b)
