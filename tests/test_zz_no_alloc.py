"""The allocation-free interval entry point, through the C ABI.

bto_interval_noalloc exists for callers that cannot let a library allocate
device memory (for example an in situ simulation whose own pool allocator owns
all device memory while it runs). It keeps the particle state in a static
device array instead of allocating it. This test checks that:

* two calls in a row (the second reusing the array the first left behind)
  give bit for bit the basis flows of the allocating context calls
  (bto_create / bto_advect_cycle / bto_end_interval) on the same inputs: both
  run the same per-particle arithmetic, only the order of the seeds in the
  list differs, so any difference would be an indexing or layout error;
* the outputs agree with the FP64 oracle under the parity rule;
* a call without the exit-cycle output writes the same seeds, ends and flags;
* a call after the first one on the device changes the free device memory by
  nothing (the first call loads the array; later calls allocate nothing);
* a block beyond the array's capacity is refused.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import bto, inputs

from gpu_helpers import compare

pytestmark = pytest.mark.gpu


def _context_run(n, origin, h, stride, fields, dt):
    import torch
    ctx = bto.Context(n, origin, h, stride, len(fields))
    for f in fields:
        ctx.advect(f, dt)
    out = ctx.end_interval()
    ctx.check()
    torch.cuda.synchronize()
    ctx.close()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _noalloc_outputs(P):
    import torch
    return {"seeds": torch.full((P, 3), float("nan"), device="cuda"),
            "ends": torch.full((P, 3), float("nan"), device="cuda"),
            "valid": torch.full((P,), 7, dtype=torch.uint8, device="cuda"),
            "exit_cycle": torch.full((P,), -99, dtype=torch.int32, device="cuda")}


def _noalloc_call(n, origin, h, stride, table, L, dt, out, with_exit=True):
    bto.bto_interval_noalloc(n, origin, h, stride, L, table, dt, out["seeds"], out["ends"], out["valid"],
                             out["exit_cycle"] if with_exit else None)


def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _same(a, b, keys=("seeds", "ends", "valid", "exit_cycle")):
    for k in keys:
        assert np.array_equal(a[k], b[k]), k


def test_noalloc_interval_matches_context_calls_twice(cuda_device):
    import torch
    from paper_2004_02003_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    cases = [
        ((40, 36, 30), (0.1, -0.2, 0.3), (0.02, 0.025, 0.03), 1, 16, 7),   # 41,400 seeds
        ((33, 21, 50), (-0.5, 0.0, 0.25), (0.03, 0.02, 0.02), 2, 24, 8),   # 8,775 seeds
    ]
    for n, origin, h, stride, L, seed in cases:
        modes = inputs.fourier_modes(seed, m=16, kmax=6.0)
        host = [inputs.fourier_field(modes, n, origin, h, c) for c in range(L)]
        fields = [torch.from_numpy(f).cuda() for f in host]
        table = torch.tensor([f.data_ptr() for f in fields], dtype=torch.int64, device="cuda")
        dt = 0.3 * min(h)
        P = int(np.prod([(n[a] + stride - 1) // stride for a in range(3)]))
        ref = _context_run(n, origin, h, stride, fields, dt)
        out = _noalloc_outputs(P)
        _noalloc_call(n, origin, h, stride, table, L, dt, out)
        torch.cuda.synchronize()
        _same(_np(out), ref)
        assert 0 < ref["valid"].sum() < ref["valid"].size
        # a second call on the array the first left behind: same outputs,
        # and no change in the device's free memory
        out2 = _noalloc_outputs(P)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _noalloc_call(n, origin, h, stride, table, L, dt, out2)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        _same(_np(out2), ref)
        # without the exit-cycle output
        out3 = _noalloc_outputs(P)
        _noalloc_call(n, origin, h, stride, table, L, dt, out3, with_exit=False)
        torch.cuda.synchronize()
        got3 = _np(out3)
        _same(got3, ref, keys=("seeds", "ends", "valid"))
        assert np.all(got3["exit_cycle"] == -99)
        # and against the FP64 oracle
        oref = oracle.run_interval(oracle.Grid.make(n, origin, h), stride, L, dt, lambda c: host[c])
        compare(_np(out2), oref, h)


def test_noalloc_refuses_blocks_beyond_its_capacity(cuda_device):
    import torch
    from paper_2004_02003_gb300 import build
    build.build()
    cap = bto.load().bto_interval_noalloc  # noqa: F841 (symbol must exist)
    n = (64, 64, 17)                       # 64*64*17 = 69,632 > 65,536 seeds
    f = torch.zeros((18, 65, 65, 3), dtype=torch.float32, device="cuda")
    table = torch.tensor([f.data_ptr()], dtype=torch.int64, device="cuda")
    out = torch.empty((69632, 3), dtype=torch.float32, device="cuda")
    valid = torch.empty((69632,), dtype=torch.uint8, device="cuda")
    with pytest.raises(bto.BtoError) as e:
        bto.bto_interval_noalloc(n, (0, 0, 0), (1, 1, 1), 1, 1, table, 0.1, out, out, valid)
    assert e.value.status == bto.BTO_ERR_UNSUPPORTED
