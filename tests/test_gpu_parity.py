"""GPU path (through the C ABI) against the FP64 oracle and closed forms."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import bto, inputs

from gpu_helpers import block_views, compare, run_gpu_interval, to_f4

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


# ----------------------------------------------------------------------------
# ABC block: 32^3 cells over [0,1]^3, stride 2 (4096 seeds), 50 cycles, dt 0.01
# ----------------------------------------------------------------------------
N1, H1, S1, L1, DT1 = (32, 32, 32), (1.0 / 32,) * 3, 2, 50, 0.01


@pytest.fixture(scope="module")
def abc_case():
    fields = [inputs.abc_field(N1, (0, 0, 0), H1, c * DT1) for c in range(L1)]
    ref = oracle.run_interval(oracle.Grid.make(N1, (0, 0, 0), H1), S1, L1, DT1, lambda c: fields[c])
    return fields, ref


def test_abc_block_parity_f3(abc_case):
    # With |u| up to ~4.8 on the unit box and dt = 0.01 (about 1.5 cells per
    # step), every particle leaves the block within the interval: the case
    # checks exit cycles and last in-block positions against the oracle.
    fields, ref = abc_case
    ctx = bto.Context(N1, (0, 0, 0), H1, S1, L1)
    gpu = run_gpu_interval(ctx, _dev(fields), DT1)
    rep = compare(gpu, ref, H1)
    assert rep["n"] == 4096
    assert np.all(ref.exit_cycle >= 0) and ref.exit_cycle.max() >= 5
    assert np.array_equal(gpu["exit_cycle"], ref.exit_cycle)
    ctx.close()


def test_abc_block_f4_layout_is_bitwise_f3(abc_case):
    fields, _ = abc_case
    a = bto.Context(N1, (0, 0, 0), H1, S1, L1)
    ga = run_gpu_interval(a, _dev(fields), DT1)
    b = bto.Context(N1, (0, 0, 0), H1, S1, L1)
    b.set_layout(bto.BTO_FIELD_F4_AOS)
    gb = run_gpu_interval(b, _dev([to_f4(f) for f in fields]), DT1)   # NaN pad must be ignored
    for k in ga:
        assert np.array_equal(ga[k], gb[k], equal_nan=True), k
    a.close(); b.close()


@pytest.mark.parametrize("layout", [bto.BTO_FIELD_F3_AOS, bto.BTO_FIELD_F4_AOS])
def test_launch_shapes_give_identical_results(abc_case, layout):
    fields, _ = abc_case
    devf = _dev(fields if layout == bto.BTO_FIELD_F3_AOS else [to_f4(f) for f in fields])
    results = []
    for nt in (128, 256):
        for ppt in (1, 2, 4):
            for cps, cap in ((0, 0), (1, 0), (0, 1)):
                ctx = bto.Context(N1, (0, 0, 0), H1, S1, L1)
                ctx.set_layout(layout)
                ctx.set_launch(nt, ppt, cps, cap)
                results.append(run_gpu_interval(ctx, devf, DT1))
                ctx.close()
    for r in results[1:]:
        for k in r:
            assert np.array_equal(r[k], results[0][k]), k


# ----------------------------------------------------------------------------
# Ragged block: odd extents, stride 2 with ceil, offset origin, anisotropic h
# ----------------------------------------------------------------------------
def test_ragged_block_turbulence_parity():
    n, origin, h, s, L = (45, 37, 29), (-0.3, 0.7, 1.1), (0.02, 0.025, 0.03), 2, 40
    modes = inputs.fourier_modes(7, m=16, kmax=6.0)
    fields = [inputs.fourier_field(modes, n, origin, h, c) for c in range(L)]
    dt = 0.3 * min(h)                          # <= 0.3 cells per step (|u| <= ~1)
    g = oracle.Grid.make(n, origin, h)
    ref = oracle.run_interval(g, s, L, dt, lambda c: fields[c])
    ctx = bto.Context(n, origin, h, s, L)
    assert ctx.P == 23 * 19 * 15
    gpu = run_gpu_interval(ctx, _dev(fields), dt)
    rep = compare(gpu, ref, h)
    assert 0 < rep["valid"] < rep["n"]         # some terminate, some survive
    ctx.close()


def test_two_intervals_reseed_and_continue():
    n, h, s, L = (24, 20, 16), (0.05, 0.05, 0.05), 1, 12
    modes = inputs.fourier_modes(11, m=12, kmax=4.0)
    fields = [inputs.fourier_field(modes, n, (0, 0, 0), h, c) for c in range(2 * L)]
    dt = 0.4 * 0.05
    g = oracle.Grid.make(n, (0, 0, 0), h)
    ctx = bto.Context(n, (0, 0, 0), h, s, L)
    devf = _dev(fields)
    for k in range(2):
        gpu = run_gpu_interval(ctx, devf[k * L:(k + 1) * L], dt)
        ref = oracle.run_interval(g, s, L, dt, lambda c: fields[c], c0=k * L)
        compare(gpu, ref, h)
    ctx.close()


# ----------------------------------------------------------------------------
# Closed forms on the GPU path
# ----------------------------------------------------------------------------
def test_uniform_translation_gpu():
    n, h, s, L, dt = (16, 16, 16), (1.0 / 16,) * 3, 4, 20, 0.5
    c = np.array([0.0078125, -0.00390625, 0.001953125])
    ctx = bto.Context(n, (0, 0, 0), h, s, L)
    gpu = run_gpu_interval(ctx, _dev([inputs.uniform_field(n, c)] * L), dt)
    x0 = gpu["seeds"].astype(np.float64)
    want = x0 + L * dt * c
    inside = np.all((want >= 0) & (want <= 1), axis=1)
    assert np.array_equal(gpu["valid"] == 1, inside)
    assert np.max(np.abs(gpu["ends"][inside] - want[inside]) * 16) < 1e-4
    ctx.close()


def test_affine_field_gpu_matches_rk4_closed_form():
    A = np.array([[-0.75, 1.5, 0.25], [-1.25, 0.5, -0.5], [0.375, -0.25, -1.0]])
    b = np.array([0.5, -0.25, 0.125])
    n, h, origin, s, L, dt = (64, 64, 64), (0.25,) * 3, (-8.0,) * 3, 8, 12, 0.0625
    ctx = bto.Context(n, origin, h, s, L)
    gpu = run_gpu_interval(ctx, _dev([inputs.affine_field(n, origin, h, A, b)] * L), dt)
    Z = dt * A
    M = np.eye(3) + Z / 2 + Z @ Z / 6 + Z @ Z @ Z / 24
    x = gpu["seeds"].astype(np.float64)
    far = np.ones(x.shape[0], dtype=bool)          # whole path well inside the box
    for _ in range(L):
        x = x + dt * (x @ A.T + b) @ M.T
        far &= np.all(np.abs(x) < 6.0, axis=1)
    ok = gpu["valid"] == 1
    assert far.sum() > 50
    assert np.all(ok[far])
    assert np.max(np.abs(gpu["ends"][far] - x[far]) / 0.25) < 1e-4
    ctx.close()


def test_straight_line_exit_cycles_gpu_brute_force():
    n, h, s, L, dt = (20, 20, 20), (0.05,) * 3, 1, 30, 0.0099
    vel = (1.0, -0.5, 0.25)
    ctx = bto.Context(n, (0, 0, 0), h, s, L)
    gpu = run_gpu_interval(ctx, _dev([inputs.uniform_field(n, vel)] * L), dt)
    seeds = oracle.seeds(oracle.Grid.make(n, (0, 0, 0), h), s)
    step = [Fraction(v) * Fraction(dt) for v in vel]
    for p in range(seeds.shape[0]):
        x = [Fraction(v) for v in seeds[p]]
        want = -1
        for c in range(L):
            nxt = [x[a] + step[a] for a in range(3)]
            if any(not (0 <= v <= 1) for v in nxt):
                want = c
                break
            x = nxt
        assert gpu["exit_cycle"][p] == want, p
    ctx.close()


# ----------------------------------------------------------------------------
# Degenerate cases and contract
# ----------------------------------------------------------------------------
def test_zero_dt_is_a_no_op():
    n, h = (8, 8, 8), (0.125,) * 3
    ctx = bto.Context(n, (0, 0, 0), h, 1, 3)
    f = inputs.abc_field(n, (0, 0, 0), h, 0.0)
    gpu = run_gpu_interval(ctx, _dev([f] * 3), 0.0)
    assert np.all(gpu["valid"] == 1)
    assert np.array_equal(gpu["ends"], gpu["seeds"])
    ctx.close()


def test_single_cell_single_seed_and_backward_dt():
    f = np.zeros((2, 2, 2, 3), dtype=np.float32)
    f[..., 0] = -1.0
    ctx = bto.Context((1, 1, 1), (0, 0, 0), (1, 1, 1), 5, 2)
    assert ctx.P == 1
    gpu = run_gpu_interval(ctx, _dev([f, f]), -0.25)     # backward: moves +x
    assert gpu["valid"][0] == 1
    assert np.allclose(gpu["ends"][0], [0.5, 0.0, 0.0])
    ctx.close()


def test_nan_field_terminates_and_matches_oracle():
    n, h, L, dt = (6, 6, 6), (1.0, 1.0, 1.0), 2, 0.1
    f = np.ones((7, 7, 7, 3), dtype=np.float32) * 0.5
    f[3, 3, 3] = np.nan
    ctx = bto.Context(n, (0, 0, 0), h, 1, L)
    gpu = run_gpu_interval(ctx, _dev([f, f]), dt)
    ref = oracle.run_interval(oracle.Grid.make(n, (0, 0, 0), h), 1, L, dt, lambda c: f)
    assert np.array_equal(gpu["valid"], ref.valid)
    assert (gpu["valid"] == 0).sum() > 0
    ctx.close()


def test_call_order_and_argument_errors():
    import torch
    n, h = (4, 4, 4), (0.25,) * 3
    ctx = bto.Context(n, (0, 0, 0), h, 1, 2)
    f = torch.zeros((5, 5, 5, 3), dtype=torch.float32, device="cuda")
    out = ctx.alloc_outputs()
    with pytest.raises(bto.BtoError) as e:
        ctx.end_interval(out)
    assert e.value.status == bto.BTO_ERR_STATE
    ctx.advect(f, 0.1)
    with pytest.raises(bto.BtoError) as e:
        ctx.set_layout(bto.BTO_FIELD_F4_AOS)
    assert e.value.status == bto.BTO_ERR_STATE
    ctx.advect(f, 0.1)
    with pytest.raises(bto.BtoError) as e:
        ctx.advect(f, 0.1)
    assert e.value.status == bto.BTO_ERR_STATE
    with pytest.raises(bto.BtoError) as e:
        ctx.advect(f, float("nan"))
    assert e.value.status == bto.BTO_ERR_INVALID_ARG
    ctx.end_interval(out)
    ctx.set_layout(bto.BTO_FIELD_F4_AOS)
    g = torch.zeros(5 * 5 * 5 * 4 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(bto.BtoError) as e:
        ctx.advect(g[1:].data_ptr(), 0.1)               # not 16-byte aligned
    assert e.value.status == bto.BTO_ERR_INVALID_ARG
    assert ctx.launch()["grid"] >= 1
    ctx.check()
    ctx.close()


def test_every_output_entry_written_once():
    import torch
    n, h, L, dt = (30, 30, 30), (1.0 / 30,) * 3, 20, 0.02
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    ctx = bto.Context(n, (0, 0, 0), h, 2, L)
    out = ctx.alloc_outputs()
    out["seeds"].fill_(float("nan")); out["ends"].fill_(float("nan"))
    out["valid"].fill_(7); out["exit_cycle"].fill_(-99)
    for f in _dev(fields):
        ctx.advect(f, dt)
    ctx.end_interval(out)
    torch.cuda.synchronize()
    v = out["valid"].cpu().numpy()
    e = out["exit_cycle"].cpu().numpy()
    assert set(np.unique(v)) <= {0, 1}
    assert np.all((e == -1) == (v == 1)) and np.all(e[v == 0] >= 0) and np.all(e < L)
    assert torch.isfinite(out["ends"]).all() and torch.isfinite(out["seeds"]).all()
    ctx.close()


# ----------------------------------------------------------------------------
# Batched blocks, interval graph, global map
# ----------------------------------------------------------------------------
def _uneven_blocks():
    ext = [(16, 24, 20), (33, 17, 9), (8, 8, 40), (27, 27, 27), (5, 3, 2)]
    strides = [1, 2, 4, 3, 1]
    origins = [(0.1 * b, -0.2 * b, 0.05 * b) for b in range(len(ext))]
    spac = [(0.02, 0.03, 0.025), (0.04, 0.02, 0.05), (0.03, 0.03, 0.01), (0.02, 0.02, 0.02),
            (0.1, 0.1, 0.1)]
    return ext, origins, spac, strides


def test_batched_equals_single_blocks_and_oracle():
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt = 16, 0.006
    modes = inputs.fourier_modes(5, m=16, kmax=5.0)
    fields = [[inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(len(ext))]
              for c in range(L)]
    devf = [_dev(fc) for fc in fields]
    ptrs = [torch.tensor([t.data_ptr() for t in fc], dtype=torch.int64, device="cuda") for fc in devf]
    bctx = bto.Context.batch(ext, origins, spac, strides, L)
    off = bctx.offsets()
    for c in range(L):
        bctx.advect_batch(ptrs[c], dt)
    out = bctx.end_interval()
    bctx.check()
    torch.cuda.synchronize()
    bout = {k: v.cpu().numpy() for k, v in out.items()}
    for b in range(len(ext)):
        ctx = bto.Context(ext[b], origins[b], spac[b], strides[b], L)
        single = run_gpu_interval(ctx, [devf[c][b] for c in range(L)], dt)
        ctx.close()
        for k in single:
            assert np.array_equal(single[k], bout[k][off[b]:off[b + 1]]), (b, k)
        ref = oracle.run_interval(oracle.Grid.make(ext[b], origins[b], spac[b]), strides[b], L, dt,
                                  lambda c: fields[c][b])
        compare(single, ref, spac[b])
    bctx.close()


def test_interval_graph_equals_per_cycle_calls():
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt = 8, 0.006
    modes = inputs.fourier_modes(6, m=8, kmax=5.0)
    devf = [_dev([inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(len(ext))])
            for c in range(L)]
    table = torch.tensor([t.data_ptr() for fc in devf for t in fc], dtype=torch.int64, device="cuda")
    nb = len(ext)
    a = bto.Context.batch(ext, origins, spac, strides, L)
    for c in range(L):
        a.advect_batch(table[c * nb:(c + 1) * nb], dt)
    ra = {k: v.cpu().numpy() for k, v in a.end_interval().items()}
    b = bto.Context.batch(ext, origins, spac, strides, L)
    for rep in range(2):                               # capture, then relaunch
        b.interval_graph(table, dt)
        rb = {k: v.cpu().numpy() for k, v in b.end_interval().items()}
        for k in ra:
            assert np.array_equal(ra[k], rb[k]), (rep, k)
    a.check(); b.check()
    a.close(); b.close()


def test_bto_valid_ends_equal_global_map():
    # BTO blocks vs one block over the whole domain (particles cross blocks):
    # a particle that stays in its block follows the same cells and node
    # values. The global map (the no-termination-at-interior-faces run of
    # Sec. 3.1) is itself held to the FP64 oracle run on the whole 48^3 grid,
    # under the parity rule (end positions within 1e-3 cells; flags equal
    # away from the domain faces), and the BTO-valid particles satisfy the
    # Eq. (hx) reading: they stay valid in the global map with the same ends.
    import torch
    nbx, n, L = 2, 24, 30
    G = nbx * n
    h = (1.0 / G,) * 3
    modes = inputs.fourier_modes(9, m=24, kmax=8.0)
    dt = 0.25 * h[0]
    gfields = [inputs.fourier_field(modes, (G, G, G), (0, 0, 0), h, c) for c in range(L)]
    blocks = [block_views(f, (nbx,) * 3, (n, n, n)) for f in gfields]
    ext = [(n, n, n)] * nbx ** 3
    origins = [(bx * n * h[0], by * n * h[0], bz * n * h[0])
               for bz in range(nbx) for by in range(nbx) for bx in range(nbx)]
    bctx = bto.Context.batch(ext, origins, [h] * len(ext), [2] * len(ext), L)
    dev = [_dev(bc) for bc in blocks]
    ptrs = [torch.tensor([t.data_ptr() for t in fc], dtype=torch.int64, device="cuda") for fc in dev]
    for c in range(L):
        bctx.advect_batch(ptrs[c], dt)
    bo = {k: v.cpu().numpy() for k, v in bctx.end_interval().items()}
    gctx = bto.Context((G, G, G), (0, 0, 0), h, 2, L)
    go = run_gpu_interval(gctx, _dev(gfields), dt)
    gref = oracle.run_interval(oracle.Grid.make((G, G, G), (0, 0, 0), h), 2, L, dt, lambda c: gfields[c])
    rep = compare(go, gref, h)
    assert rep["both_valid"] > 0.5 * rep["n"]
    # map each block seed to its global canonical id
    S = n // 2
    gid = []
    for bz in range(nbx):
        for by in range(nbx):
            for bx in range(nbx):
                j = np.arange(S ** 3)
                jx, jy, jz = j % S + bx * S, (j // S) % S + by * S, j // (S * S) + bz * S
                gid.append(jx + G // 2 * (jy + G // 2 * jz))
    gid = np.concatenate(gid)
    assert np.max(np.abs(bo["seeds"] - go["seeds"][gid]) / h[0]) < 1e-5
    v = bo["valid"] == 1
    assert np.all(go["valid"][gid][v] == 1)
    assert np.max(np.abs(bo["ends"][v] - go["ends"][gid][v]) / h[0]) < 1e-4
    frac = 1.0 - v.mean()
    assert 0.0 < frac < 0.6
    bctx.close(); gctx.close()


@pytest.mark.parametrize("layout,offset_floats", [(bto.BTO_FIELD_F3_AOS, 1), (bto.BTO_FIELD_F3_AOS, 2),
                                                  (bto.BTO_FIELD_F3_AOS, 3), (bto.BTO_FIELD_F4_AOS, 4)])
def test_field_base_alignment_does_not_change_results(abc_case, layout, offset_floats):
    # Field bases of any 4-byte alignment must give bitwise the same results.
    import torch
    fields, _ = abc_case
    arrs = fields if layout == bto.BTO_FIELD_F3_AOS else [to_f4(f) for f in fields]
    aligned = _dev(arrs)
    shifted = []
    for a in arrs:
        buf = torch.empty(a.size + 8, dtype=torch.float32, device="cuda")
        buf[offset_floats:offset_floats + a.size] = torch.from_numpy(a.ravel()).cuda()
        shifted.append(buf[offset_floats:])
    outs = []
    for fl in (aligned, shifted):
        ctx = bto.Context(N1, (0, 0, 0), H1, S1, L1)
        ctx.set_layout(layout)
        outs.append(run_gpu_interval(ctx, [f.data_ptr() for f in fl], DT1))
        ctx.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_last_node_pairs_near_array_end():
    # Particles in the cells at the far corner read the last nodes of the
    # field: an F3 gather with wide loads must not read past them.
    n, h, L, dt = (9, 7, 5), (0.1, 0.1, 0.1), 6, 0.02
    f = np.zeros((6, 8, 10, 3), dtype=np.float32)
    f[..., 0] = -0.5
    f[..., 1] = -0.5
    f[..., 2] = -0.5
    rng = np.random.default_rng(3)
    f += rng.uniform(-0.05, 0.05, f.shape).astype(np.float32)
    g = oracle.Grid.make(n, (0, 0, 0), h)
    ref = oracle.run_interval(g, 1, L, dt, lambda c: f)
    ctx = bto.Context(n, (0, 0, 0), h, 1, L)
    gpu = run_gpu_interval(ctx, _dev([f] * L), dt)
    compare(gpu, ref, h)
    ctx.close()


def test_autotune_keeps_results_and_reports_every_shape():
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt = 6, 0.006
    modes = inputs.fourier_modes(12, m=8, kmax=5.0)
    devf = [_dev([inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(len(ext))])
            for c in range(L)]
    table = torch.tensor([t.data_ptr() for fc in devf for t in fc], dtype=torch.int64, device="cuda")
    nb = len(ext)
    ref = bto.Context.batch(ext, origins, spac, strides, L)
    for c in range(L):
        ref.advect_batch(table[c * nb:(c + 1) * nb], dt)
    r0 = {k: v.cpu().numpy() for k, v in ref.end_interval().items()}
    ctx = bto.Context.batch(ext, origins, spac, strides, L)
    ctx.advect_batch(table[:nb], dt)
    with pytest.raises(bto.BtoError) as e:                 # only at cycle 0
        ctx.autotune(table, L, dt)
    assert e.value.status == bto.BTO_ERR_STATE
    ctx.close()
    ctx = bto.Context.batch(ext, origins, spac, strides, L)
    rep = ctx.autotune(table, L, dt)
    assert len(rep["ms_per_cycle"]) == 12 and all(v > 0 for v in rep["ms_per_cycle"].values())
    assert ctx.launch() == rep["best"]
    for c in range(L):
        ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
    r1 = {k: v.cpu().numpy() for k, v in ctx.end_interval().items()}
    for k in r0:
        assert np.array_equal(r0[k], r1[k]), k
    ref.check(); ctx.check()
    ref.close(); ctx.close()


def test_ingest_gives_identical_results():
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt = 10, 0.006
    modes = inputs.fourier_modes(13, m=12, kmax=5.0)
    devf = [_dev([inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(len(ext))])
            for c in range(L)]
    table = torch.tensor([t.data_ptr() for fc in devf for t in fc], dtype=torch.int64, device="cuda")
    nb = len(ext)
    outs = []
    for ingest in (0, 1):
        ctx = bto.Context.batch(ext, origins, spac, strides, L)
        ctx.set_ingest(ingest)
        for rep in range(2):                          # two intervals: buffers reused
            for c in range(L):
                ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
            outs.append({k: v.cpu().numpy() for k, v in ctx.end_interval().items()})
        if ingest:
            with pytest.raises(bto.BtoError) as e:
                ctx.interval_graph(table, dt)
            assert e.value.status == bto.BTO_ERR_UNSUPPORTED
            with pytest.raises(bto.BtoError):
                ctx.set_layout(bto.BTO_FIELD_F4_AOS)
        ctx.check()
        ctx.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[2][k]) and np.array_equal(outs[1][k], outs[3][k]), k
    # single block as well
    n, h, s_ = (30, 26, 22), (0.03, 0.035, 0.04), 1
    fields = [inputs.fourier_field(modes, n, (0, 0, 0), h, c) for c in range(L)]
    res = []
    for ingest in (0, 1):
        ctx = bto.Context(n, (0, 0, 0), h, s_, L)
        ctx.set_ingest(ingest)
        res.append(run_gpu_interval(ctx, _dev(fields), dt))
        ctx.close()
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]), k


def test_exit_locations_match_oracle_and_closed_form(abc_case):
    import torch
    fields, ref = abc_case                       # every particle leaves the 32^3 ABC block
    ctx = bto.Context(N1, (0, 0, 0), H1, S1, L1)
    for f in _dev(fields):
        ctx.advect(f, DT1)
    out = ctx.end_interval(exits=True)
    ctx.check()
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    ctx.close()
    same = (g["exit_cycle"] == ref.exit_cycle) & (ref.min_margin >= 1e-4) & (ref.exit_cycle >= 0)
    assert same.sum() > 3000
    perr = np.max(np.abs(g["exit_pos"][same] - ref.exit_pos[same]) / np.asarray(H1))
    terr = np.max(np.abs(g["exit_time"][same] - ref.exit_time[same]))
    assert perr <= 1e-3 and terr <= 5e-3, (perr, terr)
    # on a face: some coordinate at 0 or 1
    on_face = np.min(np.minimum(np.abs(g["exit_pos"][same]), np.abs(g["exit_pos"][same] - 1.0)), axis=1)
    assert np.max(on_face) < 1e-5
    # straight flow: exact crossing x = 1 at time (1 - x0) / dt cycles
    n, h, L, dt = (32, 32, 32), (1.0 / 32,) * 3, 50, 0.0099
    ctx = bto.Context(n, (0, 0, 0), h, 2, L)
    for f in _dev([inputs.uniform_field(n, (1.0, 0.0, 0.0))] * L):
        ctx.advect(f, dt)
    o = {k: v.cpu().numpy() for k, v in ctx.end_interval(exits=True).items()}
    ctx.close()
    t = o["valid"] == 0
    assert t.sum() > 100 and np.all(np.isnan(o["exit_time"][~t]))
    assert np.max(np.abs(o["exit_pos"][t, 0] - 1.0)) < 1e-6
    assert np.max(np.abs(o["exit_time"][t] - (1.0 - o["seeds"][t, 0].astype(np.float64)) / dt)) < 1e-3


def test_lattice_fill_matches_oracle():
    import torch
    rng = np.random.default_rng(21)
    S = (37, 23, 19)
    P = S[0] * S[1] * S[2]
    ends = rng.standard_normal((P, 3)).astype(np.float32)
    # missing entries in clusters, like terminations near block faces
    valid = (rng.random(P) > 0.15).astype(np.uint8)
    valid.reshape(S[2], S[1], S[0])[:, :, 10:14] = 0
    valid.reshape(S[2], S[1], S[0])[5:8, :, :] = 0
    out_o, st_o = oracle.fill_lattice(S, ends.astype(np.float64), valid)
    d_out = torch.empty((P, 3), dtype=torch.float32, device="cuda")
    d_st = torch.empty((P,), dtype=torch.uint8, device="cuda")
    bto.bto_fill_lattice(S, torch.from_numpy(ends).cuda(), torch.from_numpy(valid).cuda(), d_out, d_st)
    torch.cuda.synchronize()
    st_g, out_g = d_st.cpu().numpy(), d_out.cpu().numpy()
    assert np.array_equal(st_g, st_o)
    ok = st_o > 0
    assert np.max(np.abs(out_g[ok] - out_o[ok])) < 1e-5
    assert np.all(np.isnan(out_g[~ok]))


def test_stitching_matches_oracle():
    import torch
    rng = np.random.default_rng(22)
    S, o, sp = (17, 13, 11), (0.2, -0.1, 0.3), (0.1, 0.12, 0.15)
    P = S[0] * S[1] * S[2]
    jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
    X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * np.asarray(sp) + np.asarray(o)
    ends = []
    for k in range(3):          # smooth random flow maps (+ a few missing entries)
        E = X + 0.05 * np.sin(3 * X[:, [1, 2, 0]] + k) + 0.02 * k
        E[rng.random(P) < 0.01] = np.nan
        ends.append(E.astype(np.float32))
    start = (np.asarray(o) + rng.random((500, 3)) * (np.asarray(S) - 1) * np.asarray(sp)).astype(np.float32)
    ref = oracle.stitch(S, o, sp, [e.astype(np.float64) for e in ends], start.astype(np.float64))
    dev_e = [torch.from_numpy(e).cuda() for e in ends]
    table = torch.tensor([t.data_ptr() for t in dev_e], dtype=torch.int64, device="cuda")
    path = torch.empty((4, 500, 3), dtype=torch.float32, device="cuda")
    bto.bto_stitch_pathlines(S, o, sp, 3, table, 500, torch.from_numpy(start).cuda(), path)
    torch.cuda.synchronize()
    g = path.cpu().numpy()
    assert np.array_equal(np.isnan(g), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.isnan(ref).any() and ok.any()
    assert np.max(np.abs(g[ok] - ref[ok])) < 1e-5


def test_barycentric_stitching_matches_oracle():
    # The Kuhn-tetrahedron barycentric interpolant on the GPU against the
    # oracle, with missing entries (a particle stops only when a vertex of
    # its own tetrahedron is missing) and starts on lattice points and on
    # the tie planes fx = fy = fz.
    import torch
    rng = np.random.default_rng(23)
    S, o, sp = (17, 13, 11), (0.2, -0.1, 0.3), (0.125, 0.25, 0.125)
    P = S[0] * S[1] * S[2]
    jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
    X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * np.asarray(sp) + np.asarray(o)
    ends = []
    for k in range(3):          # bilinear terms: the two interpolants differ
        E = X + 0.05 * np.sin(3 * X[:, [1, 2, 0]] + k) + 0.3 * X * X[:, [1, 2, 0]] + 0.02 * k
        E[rng.random(P) < 0.01] = np.nan
        ends.append(E.astype(np.float32))
    n_rand = 600
    u = rng.random((n_rand, 3)) * (np.asarray(S) - 1)
    u[:50] = np.floor(u[:50])                               # lattice points
    u[50:100, 1] = np.floor(u[50:100, 1]) + (u[50:100, 0] - np.floor(u[50:100, 0]))   # fx = fy
    u[100:150, 2] = np.floor(u[100:150, 2]) + (u[100:150, 0] - np.floor(u[100:150, 0]))  # fx = fz
    start = (np.asarray(o) + u * np.asarray(sp)).astype(np.float32)
    ref = oracle.stitch(S, o, sp, [e.astype(np.float64) for e in ends], start.astype(np.float64),
                        scheme="barycentric")
    tri = oracle.stitch(S, o, sp, [e.astype(np.float64) for e in ends], start.astype(np.float64))
    dev_e = [torch.from_numpy(e).cuda() for e in ends]
    table = torch.tensor([t.data_ptr() for t in dev_e], dtype=torch.int64, device="cuda")
    path = torch.empty((4, n_rand, 3), dtype=torch.float32, device="cuda")
    bto.bto_stitch_pathlines_ex(S, o, sp, 3, table, n_rand, torch.from_numpy(start).cuda(), path,
                                bto.BTO_STITCH_BARYCENTRIC)
    torch.cuda.synchronize()
    g = path.cpu().numpy()
    assert np.array_equal(np.isnan(g), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.isnan(ref).any() and ok.any()
    assert np.max(np.abs(g[ok] - ref[ok])) < 1e-5
    # the two interpolants differ (and barycentric keeps more pathlines)
    both = ok & ~np.isnan(tri)
    assert np.max(np.abs(ref[both] - tri[both])) > 1e-4
    assert ok.sum() > (~np.isnan(tri)).sum()


def test_batched_f4_graph_and_exits_equal_f3_per_cycle():
    # The batched form with F4 fields through the interval graph, with exit
    # locations, equals the batched F3 form driven cycle by cycle.
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt = 10, 0.006
    nb = len(ext)
    modes = inputs.fourier_modes(13, m=12, kmax=5.0)
    f3 = [[inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(nb)] for c in range(L)]
    dev3 = [_dev(fc) for fc in f3]
    dev4 = [_dev([to_f4(f) for f in fc]) for fc in f3]
    t3 = torch.tensor([t.data_ptr() for fc in dev3 for t in fc], dtype=torch.int64, device="cuda")
    t4 = torch.tensor([t.data_ptr() for fc in dev4 for t in fc], dtype=torch.int64, device="cuda")
    a = bto.Context.batch(ext, origins, spac, strides, L)
    for c in range(L):
        a.advect_batch(t3[c * nb:(c + 1) * nb], dt)
    ra = {k: v.cpu().numpy() for k, v in a.end_interval(exits=True).items()}
    b = bto.Context.batch(ext, origins, spac, strides, L)
    b.set_layout(bto.BTO_FIELD_F4_AOS)
    b.interval_graph(t4, dt)
    rb = {k: v.cpu().numpy() for k, v in b.end_interval(exits=True).items()}
    a.check(); b.check()
    for k in ra:
        assert np.array_equal(ra[k], rb[k], equal_nan=True), k
    assert (ra["valid"] == 0).any() and np.isfinite(ra["exit_pos"][ra["valid"] == 0]).all()
    a.close(); b.close()


def test_copy_active_lists_the_live_particles_of_each_block():
    # After c cycles the active list holds, per block, exactly the particles
    # whose exit cycle (from the finished interval) is -1 or >= c, each once,
    # at the positions the same interval reaches after c cycles.
    import torch
    ext, origins, spac, strides = _uneven_blocks()
    L, dt, stop = 12, 0.006, 7
    nb = len(ext)
    modes = inputs.fourier_modes(14, m=12, kmax=5.0)
    devf = [_dev([inputs.fourier_field(modes, ext[b], origins[b], spac[b], c) for b in range(nb)]) for c in range(L)]
    table = torch.tensor([t.data_ptr() for fc in devf for t in fc], dtype=torch.int64, device="cuda")
    full = bto.Context.batch(ext, origins, spac, strides, L)
    for c in range(L):
        full.advect_batch(table[c * nb:(c + 1) * nb], dt)
    ref = {k: v.cpu().numpy() for k, v in full.end_interval().items()}
    full.close()
    part = bto.Context.batch(ext, origins, spac, strides, stop)
    for c in range(stop):
        part.advect_batch(table[c * nb:(c + 1) * nb], dt)
    at_stop = {k: v.cpu().numpy() for k, v in part.end_interval().items()}
    # rerun the first `stop` cycles and read the list before the writer
    for c in range(stop):
        part.advect_batch(table[c * nb:(c + 1) * nb], dt)
    act = torch.empty((part.P, 4), dtype=torch.float32, device="cuda")
    live = part.copy_active(act)
    off = part.offsets()
    act = act.cpu().numpy()
    for blk in range(nb):
        ids = act[off[blk]:off[blk] + live[blk], 3].view(np.int32)
        e = ref["exit_cycle"][off[blk]:off[blk + 1]]
        want = np.flatnonzero((e < 0) | (e >= stop))
        assert np.array_equal(np.sort(ids), want), blk
        assert len(np.unique(ids)) == len(ids)
        # xi of the listed particles = the ends of the stop-cycle interval
        xi = act[off[blk]:off[blk] + live[blk], :3].astype(np.float64)
        phys = np.asarray(origins[blk]) + xi * np.asarray(spac[blk])
        ends = at_stop["ends"][off[blk]:off[blk + 1]][ids]
        assert np.max(np.abs(phys - ends) / np.asarray(spac[blk])) < 1e-4
    part.end_interval()
    part.check()
    part.close()
