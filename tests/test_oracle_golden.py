"""The oracle still reproduces its stored small-case values (tests/golden/
oracle_small.json, written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np
import pytest

from tests.golden.make_golden import _case
from oracle.objective import gradient, hessvec, objective

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")))


@pytest.mark.parametrize("key", [k for k in GOLD if not k.startswith("_")])
def test_oracle_matches_golden(key):
    model, K, d = key.split("_")
    prob, T, R, v, p = _case(model, int(K[1:]), int(d[1:]))
    ref = GOLD[key]
    J, D, S, u1 = objective(prob, v, T, R)
    g = gradient(prob, v, T, R)
    Hp = hessvec(prob, v, T, p)
    got = {"J": J, "D": D, "S": S, "u1_sum": u1.sum(), "u1_sq": np.sum(u1 * u1),
           "g_norm": np.linalg.norm(g), "g_dot_p": np.sum(g * p), "pHp": np.sum(p * Hp)}
    for k, val in got.items():
        assert abs(val - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
