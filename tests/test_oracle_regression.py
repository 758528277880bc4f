"""Regression guard for the oracle: its values on two tiny seeded cases (Zel'dovich and
2LPT initial conditions, 4 steps) must not move unless its arithmetic is changed on
purpose (then tests/golden/make_oracle_regression.py rewrites the fixture and the commit
names the passage of the paper that justifies the change)."""
import json
import os

import numpy as np
import pytest

import golden.make_oracle_regression as gen

FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


@pytest.mark.parametrize("name", sorted(gen.CASES))
def test_oracle_values_unchanged(name):
    with open(FIXTURE) as f:
        stored = json.load(f)
    assert stored["cases"][name] == gen.CASES[name]
    want = stored["values"][name]
    got = gen.evaluate(gen.CASES[name])
    for key, ref in want.items():
        assert np.allclose(got[key], ref, rtol=1e-10, atol=1e-14 * np.max(np.abs(ref))), key
