"""Host logic of bench.py that needs no GPU: the steps per batch graph launch
and the split of the timed steps into launches."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(steps, span=0):
    return argparse.Namespace(steps=steps, span=span)


def test_span_covers_the_timed_steps_in_the_fewest_launches():
    for steps in range(1, 120):
        s = bench.span_of(_args(steps))
        assert 1 <= s <= 16
        launches = steps // s + steps % s
        best = min(steps // k + steps % k for k in range(1, 17))
        assert launches == best, (steps, s)
    assert bench.span_of(_args(20)) == 10
    assert bench.span_of(_args(7)) == 7
    assert bench.span_of(_args(20, span=4)) == 4  # an explicit span is kept
