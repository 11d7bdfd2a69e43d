"""Tiled advection kernel (shared-memory staged tiles, per-step rebinning)
through the C ABI.

The tiled cycle computes every particle with the same arithmetic on the same
node values as the untiled one (a cell outside the staged box is gathered
from global memory), so its outputs must equal the untiled outputs bit for
bit, whatever the tile shape, the thread count or the bucket overflow. The
untiled path is itself held to the FP64 oracle in test_gpu_parity.py; the
cases here also check the oracle or a closed form directly.
"""
import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import bto, inputs

from gpu_helpers import compare, run_gpu_interval, to_f4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    from paper_2004_02003_gb300 import build
    build.build()
    bto.load()
    import torch
    torch.cuda.set_device(0)
    yield


def _dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def _run(n, origin, h, s, L, devf, dt, tile=None, threads=256, layout=bto.BTO_FIELD_F3_AOS, exits=False):
    import torch
    ctx = bto.Context(n, origin, h, s, L)
    ctx.set_layout(layout)
    if tile is not None:
        ctx.set_tiling(tile, threads)
        t = ctx.tiling()
        assert t["tile_cells"] == tuple(tile) and t["threads_per_cta"] == threads and t["grid"] >= 1
    for f in devf:
        ctx.advect(f, dt)
    out = ctx.end_interval(exits=exits)
    ctx.check()
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    return res


# ABC on the unit box: ~1.5 cells per step, so stage points leave the staged
# box (one cell of halo) and the global fallback is exercised every cycle.
N1, H1, S1, L1, DT1 = (32, 32, 32), (1.0 / 32,) * 3, 2, 50, 0.01


@pytest.fixture(scope="module")
def abc_case():
    fields = [inputs.abc_field(N1, (0, 0, 0), H1, c * DT1) for c in range(L1)]
    ref = oracle.run_interval(oracle.Grid.make(N1, (0, 0, 0), H1), S1, L1, DT1, lambda c: fields[c])
    return fields, ref


@pytest.mark.parametrize("tile,threads", [((16, 16, 8), 256), ((8, 8, 8), 128), ((4, 8, 2), 256),
                                          ((32, 8, 4), 128)])
@pytest.mark.parametrize("layout", [bto.BTO_FIELD_F3_AOS, bto.BTO_FIELD_F4_AOS])
def test_tiled_equals_untiled_abc(abc_case, tile, threads, layout):
    fields, ref = abc_case
    devf = _dev(fields if layout == bto.BTO_FIELD_F3_AOS else [to_f4(f) for f in fields])
    base = _run(N1, (0, 0, 0), H1, S1, L1, devf, DT1, layout=layout)
    tiled = _run(N1, (0, 0, 0), H1, S1, L1, devf, DT1, tile=tile, threads=threads, layout=layout)
    _same(base, tiled)
    compare(tiled, ref, H1)


def test_tiled_ragged_turbulence_matches_oracle_and_untiled():
    # Slow turbulence (<= 0.3 cells per step): every sample comes from the
    # staged box; odd extents give ragged tiles at the upper faces.
    n, origin, h, s, L = (45, 37, 29), (-0.3, 0.7, 1.1), (0.02, 0.025, 0.03), 2, 40
    modes = inputs.fourier_modes(7, m=16, kmax=6.0)
    fields = [inputs.fourier_field(modes, n, origin, h, c) for c in range(L)]
    dt = 0.3 * min(h)
    ref = oracle.run_interval(oracle.Grid.make(n, origin, h), s, L, dt, lambda c: fields[c])
    devf = _dev(fields)
    base = _run(n, origin, h, s, L, devf, dt)
    for tile in ((16, 16, 16), (8, 16, 4)):
        tiled = _run(n, origin, h, s, L, devf, dt, tile=tile)
        _same(base, tiled)
        rep = compare(tiled, ref, h)
        assert 0 < rep["valid"] < rep["n"]


def test_tiled_exit_locations_equal_untiled(abc_case):
    fields, _ = abc_case
    devf = _dev(fields)
    base = _run(N1, (0, 0, 0), H1, S1, L1, devf, DT1, exits=True)
    tiled = _run(N1, (0, 0, 0), H1, S1, L1, devf, DT1, tile=(8, 8, 8), exits=True)
    assert "exit_pos" in tiled and "exit_time" in tiled
    _same(base, tiled)


def test_tiled_overflow_contraction_closed_form():
    # u = -k (x - c) contracts every particle towards c = (12, 12, 12), the
    # centre of tile [8, 16)^3: that tile's bucket (640 slots) overflows by
    # tens of thousands of particles, and the outer particles move up to 1.5
    # cells per step. RK4 of a linear field is the matrix polynomial R.
    n, h, s, L, dt, k = (32, 32, 32), (1.0, 1.0, 1.0), 1, 20, 0.1, 0.7
    c = np.array([12.0, 12.0, 12.0])
    A = -k * np.eye(3)
    field = inputs.affine_field(n, (0, 0, 0), h, A, -A @ c)
    devf = _dev([field] * L)
    base = _run(n, (0, 0, 0), h, s, L, devf, dt)
    tiled = _run(n, (0, 0, 0), h, s, L, devf, dt, tile=(8, 8, 8))
    _same(base, tiled)
    Z = dt * A
    R = np.eye(3) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    x0 = tiled["seeds"].astype(np.float64)
    want = c + (x0 - c) @ np.linalg.matrix_power(R, L).T
    assert np.all(tiled["valid"] == 1)
    assert np.max(np.abs(tiled["ends"] - want)) < 1e-4
    inside = np.all((tiled["ends"] >= 8) & (tiled["ends"] < 16), axis=1)
    assert inside.sum() > 20000                     # far beyond the bucket capacity


def test_tiled_live_list_holds_every_particle_once():
    import torch
    n, h, s, L, dt, k = (32, 32, 32), (1.0, 1.0, 1.0), 1, 20, 0.1, 0.7
    c = np.array([12.0, 12.0, 12.0])
    A = -k * np.eye(3)
    f = _dev([inputs.affine_field(n, (0, 0, 0), h, A, -A @ c)])[0]
    ctx = bto.Context(n, (0, 0, 0), h, s, L)
    ctx.set_tiling((8, 8, 8))
    act = torch.empty((ctx.P, 4), dtype=torch.float32, device="cuda")
    for cyc in range(L):
        ctx.advect(f, dt)
        if cyc in (0, 9, 19):
            live = ctx.copy_active(act)
            assert live == [ctx.P]
            ids = act[:, 3].contiguous().view(torch.int32).cpu().numpy()
            assert np.array_equal(np.sort(ids), np.arange(ctx.P))
    ctx.end_interval()
    ctx.check()
    ctx.close()


def test_tiled_batched_uneven_blocks_and_graph():
    import torch
    ext = [(16, 24, 20), (33, 17, 9), (8, 8, 40), (27, 27, 27), (5, 3, 2)]
    strides = [1, 2, 4, 3, 1]
    origins = [(0.1 * b, -0.2 * b, 0.05 * b) for b in range(len(ext))]
    spac = [(0.02, 0.03, 0.025), (0.04, 0.02, 0.05), (0.03, 0.03, 0.01), (0.02, 0.02, 0.02), (0.1, 0.1, 0.1)]
    L, dt = 16, 0.006
    nb = len(ext)
    modes = inputs.fourier_modes(5, m=16, kmax=5.0)
    fields = [[inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(nb)] for c in range(L)]
    devf = [_dev(fc) for fc in fields]
    table = torch.tensor([t.data_ptr() for fc in devf for t in fc], dtype=torch.int64, device="cuda")

    def run(tile, graph):
        ctx = bto.Context.batch(ext, origins, spac, strides, L)
        if tile:
            ctx.set_tiling(tile, 256)
        outs = []
        for rep in range(2):
            if graph:
                ctx.interval_graph(table, dt)
            else:
                for cyc in range(L):
                    ctx.advect_batch(table[cyc * nb:(cyc + 1) * nb], dt)
            outs.append({k: v.cpu().numpy() for k, v in ctx.end_interval().items()})
        ctx.check()
        ctx.close()
        return outs

    base = run(None, False)
    for tile, graph in (((8, 8, 8), False), ((16, 16, 16), True), ((4, 2, 16), True)):
        got = run(tile, graph)
        for a, b in zip(base, got):
            _same(a, b)
    off = np.concatenate([[0], np.cumsum([int(np.prod([-(-e // s) for e in ext[b]])) for b, s in
                                          zip(range(nb), strides)])])
    for b in range(nb):
        ref = oracle.run_interval(oracle.Grid.make(ext[b], origins[b], spac[b]), strides[b], L, dt,
                                  lambda c: fields[c][b])
        part = {k: v[off[b]:off[b + 1]] for k, v in base[0].items()}
        compare(part, ref, spac[b])


def test_tiled_nan_and_zero_dt():
    n, h, L = (6, 6, 6), (1.0, 1.0, 1.0), 2
    f = np.ones((7, 7, 7, 3), dtype=np.float32) * 0.5
    f[3, 3, 3] = np.nan
    devf = _dev([f, f])
    _same(_run(n, (0, 0, 0), h, 1, L, devf, 0.1), _run(n, (0, 0, 0), h, 1, L, devf, 0.1, tile=(2, 4, 2)))
    z = _run(n, (0, 0, 0), h, 1, L, _dev([np.ones_like(f)] * 2), 0.0, tile=(4, 4, 4))
    assert np.all(z["valid"] == 1) and np.array_equal(z["ends"], z["seeds"])


def test_tiling_contract():
    import torch
    n, h = (16, 16, 16), (1.0 / 16,) * 3
    ctx = bto.Context(n, (0, 0, 0), h, 1, 2)
    for bad in ((1, 8, 8), (8, 8, 256), (8, 12, 8)):
        with pytest.raises(bto.BtoError) as e:
            ctx.set_tiling(bad)
        assert e.value.status == bto.BTO_ERR_INVALID_ARG
    with pytest.raises(bto.BtoError) as e:
        ctx.set_tiling((8, 8, 8), 384)
    assert e.value.status == bto.BTO_ERR_INVALID_ARG
    with pytest.raises(bto.BtoError) as e:
        ctx.set_tiling((128, 128, 128))            # staging buffers beyond shared memory
    assert e.value.status == bto.BTO_ERR_UNSUPPORTED
    assert ctx.tiling()["tiles"] == 0
    ctx.set_tiling((8, 8, 8))
    assert ctx.tiling()["tiles"] == 8
    f = torch.zeros((17, 17, 17, 3), dtype=torch.float32, device="cuda")
    table = torch.tensor([f.data_ptr()] * 2, dtype=torch.int64, device="cuda")
    with pytest.raises(bto.BtoError) as e:
        ctx.autotune(table, 1, 0.01)
    assert e.value.status == bto.BTO_ERR_STATE
    with pytest.raises(bto.BtoError) as e:
        ctx.set_ingest(1)
    assert e.value.status == bto.BTO_ERR_STATE
    ctx.advect(f, 0.01)
    with pytest.raises(bto.BtoError) as e:
        ctx.set_tiling((4, 4, 4))
    assert e.value.status == bto.BTO_ERR_STATE
    ctx.advect(f, 0.01)
    ctx.end_interval()
    ctx.set_tiling(None)                           # back to the untiled kernel
    assert ctx.tiling()["tiles"] == 0
    ctx.advect(f, 0.01)
    ctx.advect(f, 0.01)
    out = ctx.end_interval()
    assert bool((out["valid"] == 1).all())
    ctx.check()
    ctx.close()


def test_bounded_wait_timeout_is_reported_and_context_stays_usable():
    # The test hook makes CTA 0's first staging barrier of one cycle expect
    # 16 bytes that never arrive: its bounded wait gives up (about two
    # seconds), the error word is raised, its tiles are left empty. The
    # status reaches the host as BTO_ERR_TIMEOUT, and the next interval of
    # the same context equals the untiled kernel's again.
    import time
    import torch
    n, origin, h, s, L = (45, 37, 29), (-0.3, 0.7, 1.1), (0.02, 0.025, 0.03), 2, 8
    modes = inputs.fourier_modes(7, m=16, kmax=6.0)
    fields = [inputs.fourier_field(modes, n, origin, h, c) for c in range(L)]
    dt = 0.3 * min(h)
    devf = _dev(fields)
    base = _run(n, origin, h, s, L, devf, dt)
    ctx = bto.Context(n, origin, h, s, L)
    ctx.set_tiling((8, 8, 8), 128)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_test_wait_timeout(ctx.handle, -1)
    assert e.value.status == bto.BTO_ERR_INVALID_ARG
    bto.bto_test_wait_timeout(ctx.handle, 1)
    t0 = time.perf_counter()
    for f in devf:
        ctx.advect(f, dt)
    ctx.end_interval()
    with pytest.raises(bto.BtoError) as e:
        ctx.check()
    assert e.value.status == bto.BTO_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    for f in devf:
        ctx.advect(f, dt)
    out = ctx.end_interval()
    ctx.check()
    torch.cuda.synchronize()
    _same(base, {k: v.cpu().numpy() for k, v in out.items()})
    ctx.close()


def test_every_particle_leaves_in_the_first_cycle_then_empty_lists():
    # u = (+40, 0, 0) cells per unit time with dt = 1 on a 16^3 block: every
    # stage point p2 lies 20 cells further in x, outside, so every particle
    # terminates in cycle 0 at its seed; the remaining cycles run on empty
    # lists (untiled and tiled).
    n, h, L, dt = (16, 16, 16), (1.0, 1.0, 1.0), 5, 1.0
    f = inputs.uniform_field(n, (40.0, 0.0, 0.0))
    devf = _dev([f] * L)
    for tile in (None, (4, 4, 4)):
        g = _run(n, (0, 0, 0), h, 2, L, devf, dt, tile=tile, exits=True)
        assert np.all(g["valid"] == 0) and np.all(g["exit_cycle"] == 0)
        assert np.array_equal(g["ends"], g["seeds"])
        # the clipped exit point lies on the +x face, at time 1/2 * t
        assert np.allclose(g["exit_pos"][:, 0], 16.0) and np.all(g["exit_time"] <= 0.5)
