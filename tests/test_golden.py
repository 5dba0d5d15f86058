"""Regression fixtures of the oracle (tests/golden/*.json, written by
tests/golden/make_golden.py from oracle/ only): the oracle's outputs on small
seeded cases must not change silently.  Not a GPU test."""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)

import make_golden  # noqa: E402

CASES = {"bulk_forces": make_golden.bulk_case, "bulk_daughters": make_golden.daughter_case,
         "confined_daughters": make_golden.confined_case, "cv_forward": make_golden.cv_case}


def _flat(v):
    if isinstance(v, (list, float, int)):
        return np.asarray(v, dtype=np.float64).ravel()
    return None


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_matches_its_golden_fixture(name):
    with open(os.path.join(HERE, name + ".json")) as f:
        stored = json.load(f)
    fresh = CASES[name]()
    assert stored["cite"] == fresh["cite"]
    for k, v in stored.items():
        a = _flat(v)
        if a is None:
            continue
        b = _flat(fresh[k])
        assert a.shape == b.shape, k
        assert np.allclose(b, a, rtol=1e-10, atol=1e-12 * max(1.0, np.abs(a).max())), k
