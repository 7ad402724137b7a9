"""The tile tuner's decision rule and table format (no GPU)."""
from paper_2107_01391_gb300 import tune


def test_crossover_is_the_last_n_of_the_leading_narrow_run():
    t = {1 << 13: (60.0, 50.0), 1 << 15: (61.0, 52.0), 1 << 17: (62.0, 55.0),
         1 << 19: (70.0, 70.0), 1 << 21: (90.0, 95.0), 1 << 23: (300.0, 290.0)}
    # narrow wins or ties up to 2^19; the later win at 2^23 is past a loss
    assert tune.crossover(t) == 1 << 19


def test_crossover_zero_when_wide_wins_first():
    assert tune.crossover({1 << 13: (50.0, 51.0), 1 << 15: (60.0, 40.0)}) == 0


def test_table_takes_the_smaller_crossover_of_the_two_shapes():
    m = {"device_name": "GPU X",
         "times_us": {"pairs": {1 << 13: (2.0, 1.0), 1 << 15: (2.0, 1.0), 1 << 17: (1.0, 2.0)},
                      "keys": {1 << 13: (2.0, 1.0), 1 << 15: (1.0, 2.0), 1 << 17: (1.0, 2.0)}}}
    t = tune.table(m)
    assert t["device_name"] == "GPU X"
    assert t["narrow_max_n"] == 1 << 13
    assert t["measured"]["pairs"][str(1 << 15)] == {"wide_us": 2.0, "narrow_us": 1.0}
