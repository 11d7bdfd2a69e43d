"""Seed counts against the reductions the paper prints (tests/golden)."""
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "reductions.txt")


def _rows():
    rows, abc = [], None
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        if parts[0] == "abc":
            abc = parts[1:]
        else:
            rows.append((int(parts[0]), int(parts[1])))
    return rows, abc


def test_reduction_ratio_matches_stride():
    rows, _ = _rows()
    n = 24                       # divisible by every stride in the table
    g = oracle.Grid.make((n, n, n), (0, 0, 0), (1.0 / n,) * 3)
    for X, s in rows:
        assert oracle.num_seeds(g, s) * X == n ** 3


def test_abc_seed_count_and_printed_termination_fraction():
    _, abc = _rows()
    cells, ranks, s, total = int(abc[0]), int(abc[1]), int(abc[2]), int(abc[3])
    per_axis = round(ranks ** (1 / 3))            # 4 x 4 x 4 blocks
    nb = cells // per_axis
    g = oracle.Grid.make((nb, nb, nb), (0, 0, 0), (1.0 / cells,) * 3)
    assert oracle.num_seeds(g, s) * ranks == total
    # "over 1.7M ... approximately 10% of all seeds"
    assert abs(float(abc[4]) / total - float(abc[5])) < 0.005
