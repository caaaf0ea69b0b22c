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
    # the member-0 shape with four inequalities that also carry a sparse x_s part
    # (J_sh != 0, six terms each), nonconvex (Q shifted by -20 I) so that all four
    # inequalities are active and inertia correction runs: path P1's general
    # sparse condensation
    "mds0_jsh_full": dict(kind="inst", n_d=32, m_E=1000, m_I=4, sigma_a=0.1, seed=0,
                          q_shift=-20.0, jsh_per_row=6, linsolve="full"),
    # benchmark family member 1: n_d=2000, n_s=200000, m_E=100000, m_I=50; the 4x4 matrix
    # (302050^2) does not fit, so the two-stage condensed solve (itself pinned against the full
    # 4x4 solve on small inputs) gives each direction
    "mds1_p2": dict(kind="config", k=1, linsolve="p2"),
    # member 2 (n_d=4000, n_s=400000, m_E=200000, m_I=50), condensed as above: the final objective
    # the mixed-precision solves are compared against
    "mds2_p2": dict(kind="config", k=2, linsolve="p2"),
}


def instance_for(case):
    if case["kind"] == "config":
        return synth.make_config(case["k"])
    return synth.make_instance(case["n_d"], case["m_E"], case["m_I"], case["sigma_a"],
                               seed=case["seed"], q_shift=case["q_shift"],
                               jsh_per_row=case.get("jsh_per_row", 0))


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
    # the large members take minutes of CPU time each: name them on the command line
    default = [k for k in CASES if not k.startswith(("mds1", "mds2"))]
    for name in (sys.argv[1:] or default):
        run(name)
