"""The oracle against its own stored snapshots (tests/golden/oracle_snapshots.json,
written by tests/golden/make_golden.py from the oracle alone): a change to the oracle's
arithmetic shows up here and has to be justified by the passage it follows. The values
agree to round-off across hosts (the oracle is built without FMA contraction)."""
import json
import math
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden  # noqa: E402

with open(make_golden.OUT) as fh:
    STORED = json.load(fh)


def close(a, b, rtol=1e-12):
    if isinstance(a, list):
        return len(a) == len(b) and all(close(x, y, rtol) for x, y in zip(a, b))
    if isinstance(a, int) and isinstance(b, int):
        return a == b
    return math.isclose(a, b, rel_tol=rtol, abs_tol=1e-300) or abs(a - b) <= rtol * 1e-3


@pytest.mark.parametrize("case", [c for c in make_golden.cases()], ids=lambda c: c[0])
def test_oracle_matches_its_snapshot(case):
    name, w, steps, order = case
    got = make_golden.snapshot(w, steps, order)
    want = STORED[name]
    assert set(got) == set(want)
    bad = {k: (got[k], want[k]) for k in want if not close(got[k], want[k])}
    assert not bad, bad
