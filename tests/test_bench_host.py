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


def test_collision_traffic_is_its_algorithmic_bytes():
    """The roofline's algorithmic bytes per site of the BF16 collision (two
    passes over 19 BF16 populations, the reference density read and
    written, psi / phi / q read, the node kind) and the DRAM bytes per site
    that ncu measured for that kernel agree within 1 %: the kernel reads and
    writes each byte once, so the site-scaled traffic stands for the full
    lattice."""
    assert bench.bytes_per_site_collide() == 2 * 19 * 2 + 2 * 4 + 3 * 4 + 1 == 97
    assert abs(bench.COLLIDE_DRAM_BYTES_PER_SITE / 97.0 - 1.0) < 0.01


def test_peak_is_the_measured_copy_bandwidth():
    import json
    peak, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            assert kind == "measured" and peak == float(json.load(fh)["hbm_gbs"])
    else:
        assert kind == "fallback" and peak == 6800.0
