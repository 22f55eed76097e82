"""Write the oracle's reference curves used by the GPU parity tests.

Every number in this directory's JSON files comes from oracle/ only (never
from the CUDA path).  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

names: bar1d (1D bar, all 200 steps), sen_plate_prefix (200 x 200 notched
plate, first 30 load steps, ~30 CPU minutes), batch_plate8_step1 (plate 8
of the 256-plate batch, 200 x 200, first load step: its Newton iterations
pass through tangents that defeat the Jacobi-preconditioned Krylov solvers,
~1 CPU minute), and, only when named, tpb_beam_40x8x8_90 (the notched beam
at 40 x 8 x 8 hexahedra, first 90 of its 300 load steps, a few CPU hours),
trace_plate_r14_30 and trace_beam_r7_40 (requests 14 and 7 of the seeded
serving trace: a 56 x 56 notched plate, first 30 load steps, and a 42 x 8 x 8
notched beam, first 40 load steps; the served results are compared with
them).  paper_bar_l3_500_1000 (the paper's bar, quadratic u, 500 elements,
all 1000 steps, ~1 CPU minute) and paper_sen_plate_q9_10_80 (the paper's 2D
notched specimen with 9-node u, 10 x 10 elements, all 80 steps, ~15 CPU
seconds) are part of the default set, as is paper_sen_slab_h8_10x10x2_80
(the paper's 3D notched specimen at 10 x 10 x 2 hexahedra, all 80 steps,
~2 CPU minutes).
The 200 x 200 plate has no displacement-controlled solution at step 32 (the
oracle's Newton diverges there through all halvings), so its stored run
ends at step 30.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np                # noqa: E402

import lgdm_inputs as li          # noqa: E402
from oracle import constitutive as cm  # noqa: E402
from oracle import newton as nw   # noqa: E402


def curve(problem, n_steps):
    t0 = time.time()
    out = nw.run(problem, n_steps=n_steps, energy=True)
    mat = problem.material
    D, _ = cm.damage(out["state"].kappa_hist, mat.kappa0, mat.alpha, mat.beta)
    nz = np.flatnonzero(D > 0.0)
    # damage at the committed final state, per Gauss point (element-major), stored sparsely:
    # every Gauss point not listed has D = 0 exactly
    return {"load": out["load"].tolist(), "reaction": out["reaction"].tolist(),
            "newton_iters": out["newton_iters"].tolist(), "psi": out["psi"].tolist(),
            "dissipated": out["dissipated"].tolist(), "oracle_seconds": time.time() - t0,
            "damage_final": {"n_gp": int(D.size), "idx": nz.tolist(), "val": D[nz].tolist()}}


CASES = {
    "bar1d": lambda: ("bar_problem()", li.bar_problem(), 200),
    "sen_plate_prefix": lambda: ("sen_plate_problem()", li.sen_plate_problem(), 30),
    "tpb_beam_40x8x8_90": lambda: ("tpb_beam_problem(40, 8, 8)", li.tpb_beam_problem(40, 8, 8), 90),
    "batch_plate8_step1": lambda: ("batch_plate_problems()[8]", li.batch_plate_problems()[8], 1),
    "trace_plate_r14_30": lambda: ("serving_trace()[14].problem", li.serving_trace()[14].problem, 30),
    "trace_beam_r7_40": lambda: ("serving_trace()[7].problem", li.serving_trace()[7].problem, 40),
    "paper_bar_l3_500_1000": lambda: ("paper_bar_problem(500, 1000)", li.paper_bar_problem(500, 1000), 1000),
    "paper_sen_plate_q9_10_80": lambda: ("paper_sen_plate_problem(10, 80)", li.paper_sen_plate_problem(10, 80), 80),
    "paper_sen_slab_h8_10x10x2_80": lambda: ("paper_sen_slab_problem(10, 2)", li.paper_sen_slab_problem(10, 2), 80),
}
ONLY_WHEN_NAMED = ("tpb_beam_40x8x8_90", "trace_plate_r14_30", "trace_beam_r7_40")


def main(names):
    for name in names or [n for n in CASES if n not in ONLY_WHEN_NAMED]:
        desc, p, n = CASES[name]()
        rec = {"problem": f"lgdm_inputs.{desc}", "steps": n,
               "source": "oracle/newton.run (numpy element integration, scipy SuperLU), tests/golden/make_golden.py"}
        rec.update(curve(p, n))
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(rec, f, indent=1)
        print(name, "done", rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
