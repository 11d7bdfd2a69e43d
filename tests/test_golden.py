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


ACCURACY = os.path.join(os.path.dirname(__file__), "golden", "abc_accuracy_table.txt")


def _accuracy_rows():
    rows = []
    for line in open(ACCURACY):
        line = line.split("#")[0].strip()
        if line:
            L, X, l2, acc = line.split()
            rows.append((int(L), int(X), float(l2), float(acc)))
    return rows


def _c_range(l2, acc):
    # cell sides C for which (C - L)/C * 100 rounds to the printed value
    lo_frac, hi_frac = 1.0 - (acc - 0.05) / 100.0, 1.0 - (acc + 0.05) / 100.0
    return l2 / lo_frac, l2 / hi_frac


def test_printed_accuracy_table_fits_one_cell_side_and_the_oracle_formula():
    # Sec. 4.3 / Sec. 5.2: the nine rows of the ABC table (reductions 1:1,
    # 1:8, 1:27) admit one common cell side C, so C does not grow with the
    # seed spacing (the reading C = h); and the oracle's accuracy formula,
    # evaluated at that C, reproduces every printed percentage.
    rows = _accuracy_rows()
    assert len(rows) == 9
    ranges = [_c_range(l2, acc) for _, _, l2, acc in rows]
    lo, hi = max(r[0] for r in ranges), min(r[1] for r in ranges)
    assert lo < hi, (lo, hi)
    C = 0.5 * (lo + hi)
    for _, _, l2, acc in rows:
        assert round(oracle.accuracy_percent(l2, C), 1) == acc
    # C scaled by the seed spacing (1:X -> stride X^(1/3)) fits no single value
    scaled = [(a / round(X ** (1 / 3)), b / round(X ** (1 / 3))) for (a, b), (_, X, _, _) in zip(ranges, rows)]
    assert max(r[0] for r in scaled) > min(r[1] for r in scaled)
