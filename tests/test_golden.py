"""The oracle still reproduces the regression fixtures of tests/golden (written
by tests/golden/make_golden.py from the oracle alone; the paper prints no
worked example, so they freeze the oracle's own results on tiny seeded cases
of the depth prior, NCC and TSDF rows)."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def _flat(d, prefix=""):
    for k, v in d.items():
        if isinstance(v, dict):
            yield from _flat(v, prefix + k + ".")
        elif isinstance(v, list):
            for i, x in enumerate(v):
                yield f"{prefix}{k}[{i}]", x
        else:
            yield prefix + k, v


def test_oracle_reproduces_the_fixtures():
    with open(os.path.join(HERE, "golden", "oracle_rows.json")) as f:
        stored = dict(_flat(json.load(f)["values"]))
    now = dict(_flat(make_golden.compute()))
    assert stored.keys() == now.keys()
    for k in stored:
        assert now[k] == pytest.approx(stored[k], rel=1e-9, abs=1e-12), k
