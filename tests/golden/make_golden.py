"""Write the oracle's reference curves used by the GPU parity tests.

Every number in this directory's JSON files comes from oracle/ only (never
from the CUDA path).  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

names: bar1d (1D bar, all 200 steps), sen_plate_prefix (200 x 200 notched
plate, first 30 load steps, ~30 CPU minutes).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lgdm_inputs as li          # noqa: E402
from oracle import newton as nw   # noqa: E402


def curve(problem, n_steps):
    t0 = time.time()
    out = nw.run(problem, n_steps=n_steps, energy=True)
    return {"load": out["load"].tolist(), "reaction": out["reaction"].tolist(),
            "newton_iters": out["newton_iters"].tolist(), "psi": out["psi"].tolist(),
            "dissipated": out["dissipated"].tolist(), "oracle_seconds": time.time() - t0}


CASES = {
    "bar1d": lambda: ("bar_problem()", li.bar_problem(), 200),
    "sen_plate_prefix": lambda: ("sen_plate_problem()", li.sen_plate_problem(), 30),
}


def main(names):
    for name in names or list(CASES):
        desc, p, n = CASES[name]()
        rec = {"problem": f"lgdm_inputs.{desc}", "steps": n,
               "source": "oracle/newton.run (numpy element integration, scipy SuperLU), tests/golden/make_golden.py"}
        rec.update(curve(p, n))
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(name, "done", rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
