"""Device allocator hook (bto_set_device_allocator) through the C ABI, and
allocation-failure injection: every device allocation that bto_create,
bto_batch_create, bto_set_tiling and bto_tape_create make is made to fail in
turn; each call must return BTO_ERR_OOM and give back, through the hook,
everything it had taken. Nothing faults: the failing allocation is a NULL
returned by the test's own allocator.
"""
import numpy as np
import pytest

from paper_2004_02003_gb300 import adjoint, bto, inputs

pytestmark = pytest.mark.gpu


class Pool:
    """Test allocator over torch's caching allocator, with a failure switch."""

    def __init__(self):
        self.live = {}
        self.calls = 0
        self.fail_at = None
        self.errors = []

    def alloc(self, n):
        import torch
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(n)
        self.live[p] = n
        return p

    def free(self, p):
        import torch
        if p not in self.live:
            self.errors.append(p)
            return
        del self.live[p]
        torch.cuda.caching_allocator_delete(p)


@pytest.fixture()
def pool(cuda_device):
    from paper_2004_02003_gb300 import build
    build.build()
    bto.load()
    p = Pool()
    bto.bto_set_device_allocator(p.alloc, p.free)
    yield p
    bto.bto_set_device_allocator(None, None)


def _inject(pool, make):
    """Run make() once to count its allocations, then once per allocation
    with that one failing; each failing run must raise BTO_ERR_OOM and leave
    nothing allocated."""
    pool.calls, pool.fail_at = 0, None
    obj = make()
    n = pool.calls
    assert n > 0 and pool.live
    obj.close()
    assert not pool.live and not pool.errors
    for k in range(1, n + 1):
        pool.calls, pool.fail_at = 0, k
        with pytest.raises(bto.BtoError) as e:
            make()
        assert e.value.status == bto.BTO_ERR_OOM, k
        assert not pool.live, f"allocation {k} failing leaked {len(pool.live)} buffers"
    pool.fail_at = None
    assert not pool.errors
    return n


def test_create_oom_at_every_allocation(pool):
    n = _inject(pool, lambda: bto.Context((20, 18, 16), (0, 0, 0), (0.05, 0.05, 0.05), 2, 4))
    assert n >= 8


def test_batch_create_and_tiling_oom(pool):
    ext = [(16, 12, 10), (9, 20, 7)]

    def make_tiled():
        ctx = bto.Context.batch(ext, [(0, 0, 0), (1, 0, 0)], [(0.1, 0.1, 0.1)] * 2, [1, 2], 3)
        try:
            ctx.set_tiling((8, 8, 8), 256)
        except bto.BtoError:
            ctx.close()
            raise
        return ctx

    _inject(pool, make_tiled)


def test_tape_create_oom(pool):
    _inject(pool, lambda: adjoint.Tape((16, 16, 16), (0, 0, 0), (1, 1, 1), 100, 8, 4))


def test_context_on_hook_runs_and_frees_through_it_after_uninstall(pool):
    import torch
    n, h, L = (16, 16, 16), (1.0 / 16,) * 3, 6
    fields = [torch.from_numpy(inputs.abc_field(n, (0, 0, 0), h, 0.01 * c)).cuda() for c in range(L)]
    ctx = bto.Context(n, (0, 0, 0), h, 2, L)
    assert pool.live
    bto.bto_set_device_allocator(None, None)      # later allocations: cudaMalloc
    ref = bto.Context(n, (0, 0, 0), h, 2, L)
    outs = []
    for c in (ctx, ref):
        for f in fields:
            c.advect(f, 0.01)
        o = c.end_interval()
        c.check()
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    ref.close()
    ctx.close()                                     # frees through the hook it was created with
    assert not pool.live and not pool.errors
