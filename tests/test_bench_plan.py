"""The split of a timed run into graph replays and plain steps (bench.py):
exactly the requested steps, graphs of even length, and enough plain steps
at the end to time the stream-collide launches (no GPU needed)."""
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))

import bench  # noqa: E402


def test_every_step_count_is_covered_exactly():
    for steps in range(1, 400):
        G, nrep, rest = bench.plan_timed_steps(steps, 16)
        assert nrep * G + rest == steps, steps
        assert G % 2 == 0 and 0 <= G <= 16
        assert nrep >= 0 and rest >= min(8, steps)
        if steps >= 64:
            assert G == 16 and 8 <= rest < 24


def test_the_default_and_short_runs():
    assert bench.plan_timed_steps(10000, 16) == (16, 624, 16)
    G, nrep, rest = bench.plan_timed_steps(20, 16)
    assert (nrep, rest) == (1, 8) and G == 12
    assert bench.plan_timed_steps(3, 16) == (0, 0, 3)
