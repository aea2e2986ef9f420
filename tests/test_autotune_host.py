"""Host logic of the autotuner: buckets, workload keys, candidate sets."""
import pytest

pytest.importorskip("torch")

from paper_2202_12567_gb300 import autotune


def test_bucket_is_the_largest_power_of_two_below():
    assert [autotune.bucket(x) for x in (0, 1, 2, 3, 4, 1023, 1024, 1437.5)] == [1, 1, 2, 2, 4, 512, 1024, 1024]


def test_workload_key():
    k = autotune.workload_key("room256_vpl16k_2box", 16, [1000, 1024, 1500], [600, 640, 700])
    assert k == "room256_vpl16k_2box|r16|m1024|n512"


def test_candidates_are_valid_tuning_values():
    for name, (cands, stage) in autotune.CANDIDATES.items():
        assert stage in ("pass1", "pass2", "eval", "complete", "render")
        assert cands == sorted(set(cands))
        if name.endswith("ctas_per_sm"):
            assert all(1 <= c <= 64 for c in cands)
        elif name in ("als_form", "p1_form"):
            assert cands == [0, 1]
        else:
            assert all(16 <= c <= 1024 for c in cands)


def test_each_form_is_tuned_before_the_shapes_that_act_under_it():
    names = list(autotune.CANDIDATES)
    assert names.index("p1_form") < names.index("ray_ctas_per_sm")
    assert names.index("als_form") < names.index("als_lane_entries")
