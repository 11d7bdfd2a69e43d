"""Shared helpers of the GPU tests: run an interval through the C ABI and
compare it with the FP64 oracle under the parity rule.

Parity rule: for particles valid on both sides, every end-position component
agrees within 1e-3 cell widths; valid flags agree except for particles whose
oracle path (every tested stage point and end point) came within 1e-4 cell
widths of a block face; those are counted. Seeds agree to the FP32 rounding
of their physical coordinates (2^-23 |x|, plus 1e-6 cells).
"""
from __future__ import annotations

import numpy as np

END_TOL_CELLS = 1e-3
FACE_EPS_CELLS = 1e-4


def run_gpu_interval(ctx, fields_dev, dt, stream=None):
    """Advect one interval with per-cycle device fields; return numpy outputs."""
    import torch
    for f in fields_dev:
        ctx.advect(f, dt, stream)
    out = ctx.end_interval(stream=stream)
    ctx.check()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def compare(gpu, ref, h, tol=END_TOL_CELLS, face_eps=FACE_EPS_CELLS, ids=None):
    """Assert the parity rule; return a small report dict."""
    h = np.asarray(h, dtype=np.float64)
    g_ends = gpu["ends"].astype(np.float64)
    g_seeds = gpu["seeds"].astype(np.float64)
    g_valid = gpu["valid"]
    g_exit = gpu["exit_cycle"]
    if ids is not None:
        g_ends, g_seeds, g_valid, g_exit = g_ends[ids], g_seeds[ids], g_valid[ids], g_exit[ids]
    near = ref.min_margin < face_eps
    flag_diff = g_valid != ref.valid
    bad = flag_diff & ~near
    assert not bad.any(), f"{int(bad.sum())} valid flags differ away from faces"
    # seeds: the GPU writes origin + xi h in FP32 (one rounding, at most half
    # an ulp of |x|), the oracle the same sum in FP64 from the same inputs
    seed_excess = np.abs(g_seeds - ref.seeds) - (2.0 ** -23 * np.abs(ref.seeds) + 1e-6 * h)
    seed_err = float(np.max(seed_excess / h)) if seed_excess.size else 0.0
    assert seed_err <= 0.0, f"seed positions differ by {seed_err} cells beyond FP32 rounding"
    both = (g_valid == 1) & (ref.valid == 1)
    err = float(np.max(np.abs(g_ends[both] - ref.x[both]) / h)) if both.any() else 0.0
    assert err <= tol, f"end positions differ by {err} cells (tol {tol})"
    # terminated on both sides away from faces: same cycle, same last position
    term = (g_valid == 0) & (ref.valid == 0) & ~near
    assert np.array_equal(g_exit[term], ref.exit_cycle[term]), "exit cycles differ"
    terr = float(np.max(np.abs(g_ends[term] - ref.x[term]) / h)) if term.any() else 0.0
    assert terr <= tol, f"terminated end positions differ by {terr} cells"
    assert np.all(g_exit[g_valid == 1] == -1)
    return {"n": int(g_valid.size), "valid": int((g_valid == 1).sum()), "both_valid": int(both.sum()),
            "max_err_cells": err, "near_face": int(near.sum()),
            "flag_diff_near_face": int(flag_diff.sum())}


def block_views(global_field, nb_axis, n):
    """Split a global node-grid field (Z+1, Y+1, X+1, 3) into blocks of n cells
    (shared faces), block-major with x fastest."""
    out = []
    for bz in range(nb_axis[2]):
        for by in range(nb_axis[1]):
            for bx in range(nb_axis[0]):
                out.append(np.ascontiguousarray(
                    global_field[bz * n[2]: bz * n[2] + n[2] + 1,
                                 by * n[1]: by * n[1] + n[1] + 1,
                                 bx * n[0]: bx * n[0] + n[0] + 1]))
    return out


def to_f4(field_np, pad_value=np.nan):
    f = np.empty(field_np.shape[:-1] + (4,), dtype=np.float32)
    f[..., :3] = field_np
    f[..., 3] = pad_value
    return f
