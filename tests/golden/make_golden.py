"""Write the oracle trajectories that the GPU parity tests compare against.

Calls only `oracle/` (and the seeded input generator).  Run from the repo root:
    python tests/golden/make_golden.py
Each output records, per IPM iteration, mu, the objective, E_0, every
inertia-correction attempt (dw, dc, inertia of the 4x4 matrix) and the step.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth                                  # noqa: E402
from oracle import ipm                         # noqa: E402
from oracle.model import SynthModel            # noqa: E402

CASES = {
    # benchmark family member 0: n_d=32, n_s=2000, m_E=1000, m_I=1, full 4x4 solves
    "mds0_full": dict(kind="config", k=0, linsolve="full"),
    # nonconvex variant of the same shape (Q shifted by -20 I): exercises inertia correction
    "mds0_nonconvex_full": dict(kind="inst", n_d=32, m_E=1000, m_I=1, sigma_a=0.1, seed=0,
                                q_shift=-20.0, linsolve="full"),
}


def instance_for(case):
    if case["kind"] == "config":
        return synth.make_config(case["k"])
    return synth.make_instance(case["n_d"], case["m_E"], case["m_I"], case["sigma_a"],
                               seed=case["seed"], q_shift=case["q_shift"])


def run(name):
    case = CASES[name]
    inst = instance_for(case)
    r = ipm.solve(SynthModel(inst), opt=ipm.Options(linsolve=case["linsolve"]))
    out = dict(case=case, status=r["status_str"], iters=r["iters"], f=r["f"], E0=r["E0"],
               x_sum=float(r["point"].x.sum()), x_norm=float((r["point"].x ** 2).sum() ** 0.5),
               log=[{k: v for k, v in rec.items()} for rec in r["log"]])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(name, out["status"], out["iters"], out["f"], out["E0"])


if __name__ == "__main__":
    for name in (sys.argv[1:] or CASES):
        run(name)
