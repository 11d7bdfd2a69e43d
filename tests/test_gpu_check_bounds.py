"""Bounds-checked build of libbto (BTO_CHECK_BOUNDS) on small cases.

The checked build tests every field-node index, group count, particle id,
destination tile and lattice index before using it; a failed test skips the
access, is counted, and raises the context's error word (no trap). This test
runs the same scenarios in a child process on the checked build and here on
the product build: the checked build must report itself, count no failed
check, leave every context's error word clear, and give bitwise the outputs
of the product build (the checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def scenarios():
    """Small intervals through every kernel family: ABC block (F3, F4, every
    particle leaves), a ragged turbulent block with exit locations, uneven
    batched blocks untiled and tiled, lattice and Delaunay fills, stitching."""
    import torch
    from paper_2004_02003_gb300 import bto, inputs
    torch.cuda.set_device(0)
    out = {}

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def run(ctx, fields, dt, exits=False, tag=""):
        for f in fields:
            ctx.advect(f, dt)
        o = ctx.end_interval(exits=exits)
        ctx.check()
        torch.cuda.synchronize()
        for k, v in o.items():
            out[tag + k] = v.cpu().numpy()

    n, h, L = (32, 32, 32), (1.0 / 32,) * 3, 30
    abc = [inputs.abc_field(n, (0, 0, 0), h, 0.01 * c) for c in range(L)]
    for layout, tag in ((bto.BTO_FIELD_F3_AOS, "abc3_"), (bto.BTO_FIELD_F4_AOS, "abc4_")):
        ctx = bto.Context(n, (0, 0, 0), h, 2, L)
        ctx.set_layout(layout)
        f = [dev(a if layout == bto.BTO_FIELD_F3_AOS else np.concatenate([a, np.zeros(a.shape[:-1] + (1,), np.float32)], -1))
             for a in abc]
        run(ctx, f, 0.01, tag=tag)
        ctx.close()
    n, origin, h, L = (45, 37, 29), (-0.3, 0.7, 1.1), (0.02, 0.025, 0.03), 24
    modes = inputs.fourier_modes(7, m=16, kmax=6.0)
    turb = [dev(inputs.fourier_field(modes, n, origin, h, c)) for c in range(L)]
    ctx = bto.Context(n, origin, h, 2, L)
    run(ctx, turb, 0.3 * min(h), exits=True, tag="turb_")
    ctx.close()
    ext = [(16, 24, 20), (33, 17, 9), (8, 8, 40)]
    strides = [1, 2, 4]
    org = [(0.1 * b, -0.2 * b, 0.05 * b) for b in range(3)]
    spc = [(0.02, 0.03, 0.025), (0.04, 0.02, 0.05), (0.03, 0.03, 0.01)]
    L = 12
    mod2 = inputs.fourier_modes(5, m=16, kmax=5.0)
    bf = [[dev(inputs.fourier_field(mod2, ext[b], org[b], spc[b], c)) for b in range(3)] for c in range(L)]
    table = torch.tensor([t.data_ptr() for fc in bf for t in fc], dtype=torch.int64, device="cuda")
    for tile, tag in ((None, "batch_"), ((8, 8, 8), "tiled_")):
        ctx = bto.Context.batch(ext, org, spc, strides, L)
        if tile:
            ctx.set_tiling(tile, 256)
        for c in range(L):
            ctx.advect_batch(table[3 * c:3 * c + 3], 0.006)
        o = ctx.end_interval()
        ctx.check()
        torch.cuda.synchronize()
        for k, v in o.items():
            out[tag + k] = v.cpu().numpy()
        ctx.close()
    # post hoc: lattice fill and stitching on the ABC block's basis flows
    S = (16, 16, 16)
    ends = torch.from_numpy(out["abc3_ends"]).cuda()
    valid = torch.from_numpy(out["abc3_valid"]).cuda()
    filled = torch.empty_like(ends)
    status = torch.empty_like(valid)
    bto.bto_fill_lattice(S, ends, valid, filled, status)
    table = torch.tensor([filled.data_ptr()] * 2, dtype=torch.int64, device="cuda")
    starts = torch.from_numpy(np.random.default_rng(3).uniform(0.0, 0.95, size=(500, 3)).astype(np.float32)).cuda()
    path = torch.empty((3, 500, 3), device="cuda")
    for scheme, tag in ((bto.BTO_STITCH_TRILINEAR, "tri_"), (bto.BTO_STITCH_BARYCENTRIC, "bary_")):
        bto.bto_stitch_pathlines_ex(S, (0, 0, 0), (1.0 / 8,) * 3, 2, table, 500, starts, path, scheme)
        torch.cuda.synchronize()
        out[tag + "path"] = path.cpu().numpy()
    out["fill_status"] = status.cpu().numpy()
    out["filled"] = filled.cpu().numpy()
    # the Delaunay fill of the same lattice (interior, face and edge entries)
    dfill = torch.empty_like(ends)
    dstat = torch.empty_like(valid)
    bto.bto_fill_delaunay(S, ends, valid, dfill, dstat)
    torch.cuda.synchronize()
    out["delaunay_status"] = dstat.cpu().numpy()
    out["delaunay_filled"] = dfill.cpu().numpy()
    return out


pytestmark = pytest.mark.gpu


def test_bounds_checked_build_counts_nothing_and_matches_product(cuda_device, tmp_path):
    from paper_2004_02003_gb300 import bto, build
    build.build()
    check_lib = build.build(check_bounds=True)
    dst = str(tmp_path / "checked.npz")
    env = dict(os.environ, BTO_LIBRARY=check_lib)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), dst], env=env, cwd=ROOT,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    assert r.returncode == 0, r.stdout.decode(errors="replace")[-3000:]
    bto.load()
    assert not bto.bto_check_bounds_build()
    assert bto.bto_bounds_failures() == 0
    want = scenarios()
    got = np.load(dst)
    assert set(got.files) == set(want)
    for k in want:
        assert np.array_equal(got[k], want[k], equal_nan=True), k


if __name__ == "__main__":
    # child: run the scenarios on the library named by BTO_LIBRARY
    from paper_2004_02003_gb300 import bto
    bto.load()
    assert bto.bto_check_bounds_build(), "BTO_LIBRARY is not the bounds-checked build"
    bto.bto_bounds_failures(reset=True)
    res = scenarios()
    fails = bto.bto_bounds_failures()
    assert fails == 0, f"{fails} bounds checks failed"
    np.savez(sys.argv[1], **res)
    print("checked build: 0 failed checks,", len(res), "outputs")
