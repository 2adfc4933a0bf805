"""Record the oracle's operation counts per report step (assemblies, ILU(0)
factorisations, BiCGStab iterations) on a benchmark model, for converting
timed oracle samples to cell-steps/s.  Calls only the oracle.

    python oracle/calibrate.py --config 1 --steps 3
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    a = ap.parse_args()
    m = synth.config1() if a.config == 1 else synth.config0()
    o = oracle.Oracle(m)
    o.init_hydrostatic()
    tot = {"assemblies": 0, "solves": 0, "lin_its": 0}
    per = []
    for s in range(a.steps):
        t0 = time.perf_counter()
        st, rep = o.step(m["dt"])
        el = time.perf_counter() - t0
        if st != 0:
            raise SystemExit(f"oracle step {s} failed: {rep}")
        asm = rep["newton_its"] + rep["substeps"] + rep["cuts"]
        tot["assemblies"] += asm
        tot["solves"] += rep["newton_its"]
        tot["lin_its"] += rep["lin_its"]
        per.append({**rep, "assemblies": asm, "seconds": round(el, 2)})
        print(s, per[-1], flush=True)
        _write(a, tot, per, s + 1)



def _write(a, tot, per, done):
    out_path = os.path.join(HERE, "op_counts.json")
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    # per report step; bench.py averages the steps it times
    data[str(a.config)] = {k: v / done for k, v in tot.items()}
    data[str(a.config)]["steps_measured"] = done
    data[str(a.config)]["per_step"] = per
    json.dump(data, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main()
