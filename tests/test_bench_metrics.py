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


def test_reference_arm_line():
    """The reference arm (the FP64 oracle on the host cores, a bounded sample
    per step) prints one JSON line with the contract's keys, the GPU arm's
    metric, unit and direction, and the GPU arm's workload keys in its
    config."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                       timeout=600)
    assert r.returncode == 0, r.stderr.decode(errors="replace")[-2000:]
    lines = [ln for ln in r.stdout.decode().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    for k in ("metric", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling", "vs_baseline", "dtype",
              "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["unit"] == "particle-steps/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    h = 1.0 / bench.GLOBAL_CELLS
    want = bench.workload_config(bench.STRIDE, 8 * (bench.BLOCK_CELLS // bench.STRIDE) ** 3, 8, bench.INTERVAL,
                                 0.25 * h, "f3", 8 * (bench.BLOCK_CELLS + 1) ** 3 * 12)
    assert d["config"] == want
