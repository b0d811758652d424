"""The autotuner's choice among timed candidates (host logic, no GPU)."""
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
from paper_1404_2891_gb300.autotune import bucket, choose_single  # noqa: E402


def test_fastest_candidate_wins_outside_the_tie_band():
    times = {(192, 256): 40.0, (256, 256): 41.0, (-1, 256): 60.0}
    assert choose_single(times, 4096) == ((192, 256), 40.0)


def test_default_outer_block_wins_ties():
    times = {(192, 256): 46.78, (256, 512): 46.82, (256, 256): 46.93, (-1, -1): 70.0}
    assert choose_single(times, 4096) == ((256, 512), 46.82)


def test_small_orders_default_to_the_one_level_lu():
    times = {(128, 256): 5.00, (-1, 1024): 5.04}
    assert choose_single(times, 800) == ((-1, 1024), 5.04)
    assert choose_single(times, 800, tie=0.0) == ((128, 256), 5.00)


def test_order_buckets_are_the_next_power_of_two():
    assert [bucket(v) for v in (1, 64, 65, 1100, 2048, 4096, 4097)] == [1, 64, 128, 2048, 2048, 4096, 8192]
