"""Writes tests/golden/oracle_small.json: oracle values on small seeded cases.

The paper prints no worked example, so these fixtures are regression anchors
written by the oracle alone (this script imports only ``oracle`` and the
seeded input generator).  Each entry names the paper passage it evaluates.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lagrangian as L  # noqa: E402
from oracle.objective import Problem, gradient, hessvec, objective  # noqa: E402
from paper_1703_04446_gb300 import synth  # noqa: E402


def _case(model, K, d):
    ig = L.Grid((12, 10, 8)[:d])
    vg = L.Grid((6, 5, 4)[:d])
    gs = synth.GridSpec(ig.m, tuple(ig.lo), tuple(ig.hi))
    T = synth.gaussian_blobs(synth.centres(gs), [(1.0, 0.2, (0.45, 0.5, 0.5)[:d]),
                                                 (0.6, 0.1, (0.6, 0.4, 0.55)[:d])])
    R = synth.gaussian_blobs(synth.centres(gs), [(1.0, 0.2, (0.5, 0.47, 0.52)[:d]),
                                                 (0.6, 0.1, (0.62, 0.45, 0.5)[:d])])
    vs = synth.GridSpec(vg.m, tuple(vg.lo), tuple(vg.hi))
    v = synth.random_velocity(vs, K, 0.12, 21)
    p = synth.random_velocity(vs, K, 0.05, 22)
    prob = Problem(ig, vg, K=K, N=4, model=model, reg="diffusion", alpha=1e-2, gamma=1e-3)
    return prob, T.astype(np.float32).astype(np.float64), R.astype(np.float32).astype(np.float64), \
        v.astype(np.float32).astype(np.float64), p.astype(np.float32).astype(np.float64)


def main():
    out = {"_about": "oracle-written regression values; inputs from synth (float32-rounded), "
                     "Eq. 9-10 objective, Sec. 3.2 gradient and Gauss-Newton Hessian"}
    for model, K, d in [("transport", 1, 2), ("transport", 3, 2), ("continuity", 2, 2),
                        ("transport", 1, 3), ("continuity", 2, 3)]:
        prob, T, R, v, p = _case(model, K, d)
        J, D, S, u1 = objective(prob, v, T, R)
        g = gradient(prob, v, T, R)
        Hp = hessvec(prob, v, T, p)
        out[f"{model}_K{K}_d{d}"] = {
            "cite": "Eq. 6/7 final state, Eq. 10 SSD, Sec. 3.2 gradient and Hessian",
            "J": J, "D": D, "S": S,
            "u1_sum": float(u1.sum()), "u1_sq": float(np.sum(u1 * u1)),
            "g_norm": float(np.linalg.norm(g)), "g_dot_p": float(np.sum(g * p)),
            "pHp": float(np.sum(p * Hp)),
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("wrote", path)


if __name__ == "__main__":
    main()
