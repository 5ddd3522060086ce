"""Regression of the CPU oracle against its own stored results
(tests/golden/oracle_regression.txt, written by
tests/golden/make_oracle_regression.py): the GHZ-4 pulse circuit at 2x2 in
the exact regime and seeded truncated runs at 4x4 (chi = 16) and 3x3 with
padding (chi = 9).  The stored values are not pins -- the oracle's pins are
the closed forms and invariants in the other test_oracle_* files -- they
catch an unintended change of the oracle's arithmetic.  Tolerance 1e-9:
LAPACK and BLAS rounding differs between machines, and the truncated runs
move by ~1e-14 under such rounding (QR dependence threshold 1e-10).
"""
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_oracle_regression as gen  # noqa: E402

TOL = 1e-9


def _stored():
    out = {}
    for line in open(os.path.join(HERE, "golden", "oracle_regression.txt")):
        if line.startswith("#") or not line.strip():
            continue
        case, key, val = line.split()
        out.setdefault(case, {})[key] = float(val)
    return out


def test_oracle_reproduces_its_stored_results():
    stored = _stored()
    seen = set()
    for name, o, o0 in gen.cases():
        seen.add(name)
        got = gen.values(o, o0)
        assert set(got) == set(stored[name]), name
        for k, v in got.items():
            ref = stored[name][k]
            assert abs(v - ref) <= TOL * max(1.0, abs(ref)), (name, k, v, ref)
    assert seen == set(stored)
