"""The FP64 oracle against its frozen regression fixtures (tests/golden/oracle_fixtures.txt,
written by tests/golden/make_golden.py from the oracle itself; the paper prints no worked
numerical example to store instead). A change of the oracle's arithmetic fails here until the
fixtures are rewritten, with the passage that justifies the change named in that commit."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden                                   # noqa: E402

RTOL = 1e-13     # the oracle is compiled without FMA contraction; libm may differ in the last bit


def _stored():
    d = {}
    with open(make_golden.OUT) as f:
        for ln in f:
            if ln.startswith("#") or " : " not in ln:
                continue
            k, v = ln.rstrip("\n").split(" : ")
            d[k] = v.split()
    return d


@pytest.fixture(scope="module")
def fresh():
    d = {}
    for ln in make_golden.lines():
        k, v = ln.split(" : ")
        d[k] = v.split()
    return d


def test_philox_words_are_unchanged(fresh):
    stored = _stored()
    keys = [k for k in stored if k.startswith("philox")]
    assert len(keys) == len(make_golden.PHILOX_CASES)
    for k in keys:
        assert fresh[k] == stored[k], k


def test_normals_and_one_step_are_unchanged(fresh):
    stored = _stored()
    assert set(fresh) == set(stored)
    for k in stored:
        if k.startswith("philox"):
            continue
        if k in ("step elem", "step lost", "walls elem", "walls lost", "walls mirrorings"):
            assert fresh[k] == stored[k], k
            continue
        a = np.array([float(v) for v in fresh[k]])
        b = np.array([float(v) for v in stored[k]])
        scale = max(float(np.max(np.abs(b))), 1e-300)
        assert a.shape == b.shape, k
        assert np.all(np.abs(a - b) <= RTOL * np.maximum(np.abs(b), scale * 1e-3)), k
