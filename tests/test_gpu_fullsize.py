"""Full-size parity: the benchmark's workload (256^3 cells as 2x2x2 blocks of
128^3, stride 2, 2,097,152 particles, 100 cycles) in the benchmark's launch
configuration, against the FP64 oracle on sampled particles, plus the Eq. (hx)
invariant on every particle.

The fields are synthesised on the host (the seeded generator module, in
float64, rounded to float32) and copied to the device, so both sides read
identical inputs.
"""
import numpy as np
import pytest

import bench
import oracle
from paper_2004_02003_gb300 import bto, inputs

from gpu_helpers import compare

pytestmark = pytest.mark.gpu

SAMPLES_PER_BLOCK = 2048


def test_turb256_full_size_sampled_parity(cuda_device):
    import torch
    from paper_2004_02003_gb300 import build
    build.build()
    modes = inputs.fourier_modes(bench.SEED, m=bench.NMODES, kmin=1.0, kmax=16.0, drift_max=0.05)
    blocks, ext, org, spc = bench.block_layout(0, 1)
    nb, L = len(blocks), bench.INTERVAL
    h = 1.0 / bench.GLOBAL_CELLS
    dt = 0.25 * h
    n = bench.BLOCK_CELLS
    G = bench.GLOBAL_CELLS

    rng = np.random.default_rng(bench.SEED + 1)
    grids = [oracle.Grid.make(ext[b], org[b], spc[b]) for b in range(nb)]
    P_b = oracle.num_seeds(grids[0], bench.STRIDE)
    ids = [np.sort(rng.choice(P_b, size=SAMPLES_PER_BLOCK, replace=False)) for _ in range(nb)]
    states = [oracle.State(oracle.seeds(grids[b], bench.STRIDE, ids[b])) for b in range(nb)]

    dev_fields = []
    vmax = 0.0
    for c in range(L):
        gf = inputs.fourier_field_torch(modes, (G, G, G), (0, 0, 0), (h, h, h), c, "cpu").numpy()
        vmax = max(vmax, float(np.sqrt((gf * gf).sum(-1).max())))
        row = []
        for b, (bx, by, bz) in enumerate(blocks):
            f = np.ascontiguousarray(gf[bz * n: bz * n + n + 1, by * n: by * n + n + 1, bx * n: bx * n + n + 1])
            oracle.cycle(grids[b], f, dt, c, states[b])
            row.append(torch.from_numpy(f).to(cuda_device))
        dev_fields.append(row)
        del gf

    ctx = bto.Context.batch(ext, org, spc, [bench.STRIDE] * nb, L)    # default = bench's launch
    ptrs = [torch.tensor([t.data_ptr() for t in row], dtype=torch.int64, device=cuda_device)
            for row in dev_fields]
    for c in range(L):
        ctx.advect_batch(ptrs[c], dt)
    out = ctx.end_interval()
    ctx.check()
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    off = ctx.offsets()
    ctx.close()

    for b in range(nb):
        sub = {k: v[off[b]:off[b + 1]] for k, v in gpu.items()}
        compare(sub, states[b], spc[b], ids=ids[b])

    # Eq. (hx): a seed farther from every face than the largest displacement
    # of the interval cannot reach the boundary, so it must be valid.
    reach = L * dt * vmax
    for b in range(nb):
        seeds = gpu["seeds"][off[b]:off[b + 1]].astype(np.float64)
        lo = np.asarray(org[b])
        hi = lo + n * h
        d = np.min(np.minimum(seeds - lo, hi - seeds), axis=1)
        far = d > reach + 1e-9
        assert far.sum() > 0
        assert np.all(gpu["valid"][off[b]:off[b + 1]][far] == 1)
    assert 0.01 < 1.0 - gpu["valid"].mean() < 0.5
