"""The benchmark's metric arithmetic (host logic, no GPU): particle-steps,
live counts, terminations per cycle and algorithmic bytes, on a case worked
by hand."""
import numpy as np

import bench


def test_particle_steps_live_and_terminations_by_hand():
    # 5 particles, L = 4 cycles: two survive (exit -1), one terminates in
    # cycle 0, one in cycle 2, one in the last cycle (3)
    L = 4
    e = np.array([-1, 0, 2, -1, 3], dtype=np.int32)
    # steps attempted: 4 + 1 + 3 + 4 + 4
    assert bench.count_particle_steps(e, L) == 16
    # live at the start of cycles 0..3: 5, 4, 4, 3
    assert list(bench.live_per_cycle(e, L)) == [5, 4, 4, 3]
    # terminated in cycles 0..3: 1, 0, 1, 1 (the last cycle counts too)
    assert list(bench.terminated_per_cycle(e, L)) == [1, 0, 1, 1]
    nodes = np.array([100, 90, 90, 80])
    want = [12 * 100 + 24 * 5 + 17, 12 * 90 + 24 * 4, 12 * 90 + 24 * 4 + 17, 12 * 80 + 24 * 3 + 17]
    assert list(bench.algorithmic_bytes(e, nodes, L)) == want
    # every attempted step is a live particle at a cycle start
    assert bench.live_per_cycle(e, L).sum() == bench.count_particle_steps(e, L)


def test_no_particle_and_none_terminated():
    L = 3
    assert bench.count_particle_steps(np.array([], dtype=np.int32), L) == 0
    assert list(bench.terminated_per_cycle(np.array([-1, -1], dtype=np.int32), L)) == [0, 0, 0]
    assert list(bench.algorithmic_bytes(np.array([-1, -1], dtype=np.int32), np.zeros(L), L)) == [48, 48, 48]
