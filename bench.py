#!/usr/bin/env python3
"""Benchmark: RK4 particle-steps/s of BTO flow-map extraction on GB300.

Workload (default, ``turb256``): a 256^3-cell domain split into 2x2x2 blocks of
128^3 cells (129^3 shared-face nodes each), FP32 float3 divergence-free
Fourier-mode turbulence (64 modes, |k| in [1,16], amplitude |k|^-5/6, phases
drifting per cycle, seed 20040204), one seed per 2^3 cells (262,144 per block,
2,097,152 in all), an interval of 100 cycles, dt = 0.25 cell / max|u|.

One bench STEP is one interval of the whole hot path over that input: 100
advection cycles of all 8 blocks (one persistent launch per cycle) and the
interval end (basis-flow writer and reseed). The 100 per-cycle fields
(8 x 100 x 25.7 MB = 20.6 GB, F3 layout) are synthesised in HBM before the
timed region, so every cycle reads a field larger than L2 that was not
recently touched.

Printed JSON (one line, rank 0): value = particle-steps per second over the
whole step, roofline of the advection kernel against the measured HBM copy
peak, the FP64 CPU oracle's rate on a bounded sample, and an end-to-end
figure with the fields copied from pinned host memory every cycle.

Also reported: the same workload as 8 separate single-block contexts
(``plain``), as one CUDA graph per interval (``graph``), the paper's metric
that excludes the write cycle, and the accuracy cost of BTO against the
in-GPU global flow map in which particles cross blocks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SEED = 20040204
GLOBAL_CELLS = 256
BLOCK_CELLS = 128
STRIDE = 2
INTERVAL = 100
NMODES = 64
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain/graph/global-map/e2e legs")
    ap.add_argument("--no-large", action="store_true", help="skip the 134M-particle in situ emulation leg")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--layout", default="f3", choices=["f3", "f4"],
                    help="field layout handed to the library (f4 pads each node to 16 bytes)")
    ap.add_argument("--ingest", action="store_true", help="repack F3 fields to 16-byte nodes per block (H1)")
    ap.add_argument("--launch", default="", help="threads,ppt,ctas_per_sm,reg_cap (default: library's)")
    ap.add_argument("--e2e-streams", type=int, default=1, help="copy streams of the end-to-end leg")
    ap.add_argument("--only", default="", choices=["", "batched"],
                    help="run one workload leg alone and print its JSON (for profiling)")
    ap.add_argument("--no-plain", action="store_true", help="batched leg: skip the 512-context plain comparison")
    ap.add_argument("--tile", default="", help="tx,ty,tz[,threads]: tiled advection kernel (default: off)")
    ap.add_argument("--stride", type=int, default=STRIDE,
                    help="seed stride of the main leg, to profile it at other densities "
                         "(other than 2 it skips the other legs)")
    ap.add_argument("--fields", type=int, default=INTERVAL,
                    help="distinct per-cycle fields kept in HBM (cycle c uses field c %% N); "
                         "fewer fields make a small case for profiling")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no data-path collective)
# ---------------------------------------------------------------------------
def dist_init(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device="cuda"):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world, device="cuda"):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(units, seconds, world, device="cuda"):
    """Whole-job throughput: units of all ranks over the slowest rank's time.
    Host-side reporting only; the per-cycle path has no collective."""
    total = sum_over_ranks(float(units), world, device)
    slowest = max_over_ranks(float(seconds), world, device)
    return total, slowest, total / slowest


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = getattr(self, "t_start", 0.0), getattr(self, "t_end", float("inf"))
        inside = [ln for (t, ln) in self.lines if lo <= t <= hi + 0.05]
        if not inside and self.lines:
            # timed region shorter than the sampling period: nearest sample
            mid = 0.5 * (lo + hi)
            inside = [min(self.lines, key=lambda tl: abs(tl[0] - mid))[1]]
        for ln in inside:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def block_layout(rank=0, world=1):
    """Blocks of one rank. The job's domain is (2*world) x 2 x 2 blocks of
    128^3 cells (each rank's 2x2x2 share is a 256^3-cell cube); rank r owns
    the blocks with bx in {2r, 2r+1}. Weak scaling: every rank has the same
    work, and the blocks of different ranks never overlap."""
    nbx = GLOBAL_CELLS // BLOCK_CELLS
    h = 1.0 / GLOBAL_CELLS
    blocks = []
    for bz in range(nbx):
        for by in range(nbx):
            for bx in range(nbx):
                blocks.append((bx + nbx * rank, by, bz))
    ext = [(BLOCK_CELLS,) * 3] * len(blocks)
    org = [(b[0] * BLOCK_CELLS * h, b[1] * BLOCK_CELLS * h, b[2] * BLOCK_CELLS * h) for b in blocks]
    spc = [(h, h, h)] * len(blocks)
    return blocks, ext, org, spc


def synth_fields(modes, blocks, cycles, device, with_global=False):
    """Per-cycle block fields (F3, contiguous) generated in device memory: the
    rank's 256^3-cell cube is synthesised whole (257^3 nodes) and cut into its
    8 blocks with shared faces."""
    import torch
    from paper_2004_02003_gb300 import inputs
    G = GLOBAL_CELLS
    h = 1.0 / G
    n = BLOCK_CELLS
    bx0 = min(b[0] for b in blocks)
    x0 = bx0 * n * h
    per_cycle, glob = [], []
    for c in range(cycles):
        gf = inputs.fourier_field_torch(modes, (G, G, G), (x0, 0, 0), (h, h, h), c, device)
        row = []
        for (bx, by, bz) in blocks:
            bx -= bx0
            row.append(gf[bz * n: bz * n + n + 1, by * n: by * n + n + 1, bx * n: bx * n + n + 1].contiguous())
        per_cycle.append(row)
        if with_global:
            glob.append(gf)
        else:
            del gf
    torch.cuda.synchronize()
    return per_cycle, glob


def count_particle_steps(exit_cycle, L):
    """Particle-steps of an interval: each particle attempts one step per cycle
    while live at the cycle's start, i.e. L steps if valid, exit+1 otherwise."""
    e = exit_cycle.astype(np.int64)
    return int(np.where(e < 0, L, e + 1).sum())


def live_per_cycle(exit_cycle, L):
    e = exit_cycle.astype(np.int64)
    steps = np.where(e < 0, L, e + 1)
    return np.array([(steps > c).sum() for c in range(L)], dtype=np.int64)


def touched_nodes(ctx, act, n_cells, nb):
    """Nodes of the cells that hold a live particle at the start of the current
    cycle, summed over blocks: the nodes the cycle's first RK4 stage must read
    (a lower bound of all nodes the cycle touches: later stage points may
    reach a neighbour cell)."""
    import torch
    live = ctx.copy_active(act)
    off = ctx.offsets()
    n = n_cells
    total = 0
    for b in range(nb):
        x = act[off[b]:off[b] + live[b], :3]
        if x.shape[0] == 0:
            continue
        cell = torch.clamp(torch.floor(x).to(torch.int64), 0, n - 1)
        mark = torch.zeros((n + 1) ** 3, dtype=torch.bool, device=act.device)
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    idx = (cell[:, 0] + dx) + (n + 1) * ((cell[:, 1] + dy) + (n + 1) * (cell[:, 2] + dz))
                    mark[idx] = True
        total += int(mark.sum().item())
    return total


def terminated_per_cycle(exit_cycle, L):
    """Particles whose step in cycle c terminated them (exit cycle c)."""
    e = exit_cycle.astype(np.int64)
    return np.bincount(e[e >= 0], minlength=L)[:L].astype(np.int64)


def algorithmic_bytes(exit_cycle, nodes_touched, L):
    """Algorithmic bytes of cycle c (what the method must move):
    12 * nodes touched + 24 * live at start + 17 * terminated in the cycle."""
    return (12 * np.asarray(nodes_touched, dtype=np.int64) + 24 * live_per_cycle(exit_cycle, L)
            + 17 * terminated_per_cycle(exit_cycle, L))


def hbm_peak():
    """HBM bandwidth denominator (GB/s): the measured copy bandwidth of this
    pool's GB300s when the measurement file is present, else 6800 GB/s."""
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk)) if os.path.exists(pk) else {}
    if "hbm_gbs" in peaks:
        return float(peaks["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha256():
    """Hash of the advection kernel's sources (kernel file + shared device
    functions): ties a recorded ncu capture to the code it measured."""
    import hashlib
    h = hashlib.sha256()
    for name in ("bto_kernels.cu", "bto_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2004_02003_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def measured_traffic(launch):
    """DRAM bytes (read + write) of one advect launch from the committed ncu
    captures (one per launch shape), or None when the kernel source has
    changed since the captures or none was of this launch shape."""
    rec = os.path.join(ROOT, "profiles", "advect_turb256_traffic.json")
    if not os.path.exists(rec):
        return None
    d = json.load(open(rec))
    if not kernel_source_sha256().startswith(d["kernel_source_sha256_prefix"]):
        return None
    shape = [launch["threads_per_cta"], launch["particles_per_thread"], launch["reg_cap"]]
    for c in d.get("captures", []):
        if c.get("launch_shape") == shape:
            return c["dram_bytes_per_launch"]
    return None


def run_ours(args):
    import torch
    from paper_2004_02003_gb300 import bto, inputs
    from paper_2004_02003_gb300 import build as lib_build

    rank, world, local = dist_init(args.gpus)
    lib_build.build()
    bto.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    if args.stride != STRIDE:          # a profiling variant of the main leg only
        args.no_extras = args.no_large = True
        args.cpu_seconds = 0.0

    modes = inputs.fourier_modes(SEED, m=NMODES, kmin=1.0, kmax=16.0, drift_max=0.05)
    h = 1.0 / GLOBAL_CELLS
    dt = 0.25 * h  # max|u| = 1 after normalisation -> 0.25 cells per step at max speed
    blocks, ext, org, spc = block_layout(rank, world)
    nb = len(blocks)
    L = INTERVAL
    nf = max(1, min(args.fields, L))
    fields, gfields = synth_fields(modes, blocks, nf, dev, with_global=(rank == 0 and not args.no_extras))
    if args.layout == "f4":
        fields = [[torch.nn.functional.pad(f, (0, 1)).contiguous() for f in row] for row in fields]
    fields = [fields[c % nf] for c in range(L)]
    gfields = [gfields[c % nf] for c in range(L)] if gfields else gfields
    table = torch.tensor([f.data_ptr() for row in fields for f in row], dtype=torch.int64, device=dev)
    field_bytes_cycle = sum(f.numel() * 4 for f in fields[0])

    ctx = bto.Context.batch(ext, org, spc, [args.stride] * nb, L)
    layout = bto.BTO_FIELD_F4_AOS if args.layout == "f4" else bto.BTO_FIELD_F3_AOS
    ctx.set_layout(layout)
    if args.ingest:
        ctx.set_ingest(1)
    if args.launch:
        ctx.set_launch(*[int(v) for v in args.launch.split(",")])
        tune = None
    else:
        # the library's autotuner picks the launch shape on this workload
        # (each of its 12 shapes runs one whole interval; then reseeded)
        tune = ctx.autotune(table, L, dt)
    if args.tile:
        tv = [int(v) for v in args.tile.split(",")]
        ctx.set_tiling(tv[:3], tv[3] if len(tv) > 3 else 256)
    P = ctx.P
    out = ctx.alloc_outputs(dev)

    end_ev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]

    block_ev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]

    def one_step(timing=False, launch_events=None):
        # timing: events around the block of L advection launches and around
        # the interval end, none between launches (so each launch still
        # overlaps the previous one's tail); launch_events: one pair around
        # every launch (the launches then run one after the other)
        if timing:
            block_ev[0].record(stream)
        for c in range(L):
            if launch_events is not None:
                launch_events[c][0].record(stream)
            ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
            if launch_events is not None:
                launch_events[c][1].record(stream)
        if timing:
            block_ev[1].record(stream)
            end_ev[0].record(stream)
        ctx.end_interval(out)
        if timing:
            end_ev[1].record(stream)

    # untimed reference interval: exit cycles define the units of every step,
    # and the live particles' cells give the field nodes each cycle touches
    act = torch.empty((P, 4), dtype=torch.float32, device=dev)
    nodes_touched = np.zeros(L, dtype=np.int64)
    for c in range(L):
        nodes_touched[c] = touched_nodes(ctx, act, BLOCK_CELLS, nb)
        ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
    ctx.end_interval(out)
    torch.cuda.synchronize()
    ctx.check()
    exit_np = out["exit_cycle"].cpu().numpy()
    valid_np = out["valid"].cpu().numpy()
    psteps = count_particle_steps(exit_np, L)
    nodes_total = nb * (BLOCK_CELLS + 1) ** 3

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(L)]
    launch_ms = []
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)            # let the sampler start before the timed region
        clk.mark("t_start")
        t0.record(stream)
        for k in range(args.steps):
            # events around the launch block and the interval end in the last
            # timed step only (same work every step)
            one_step(timing=k == args.steps - 1)
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark("t_end")
    barrier(world)
    elapsed = t0.elapsed_time(t1) / 1e3
    block_ms = block_ev[0].elapsed_time(block_ev[1])
    # one more (untimed) interval with events around every launch: the
    # launch-by-launch profile across the interval
    one_step(launch_events=ev)
    torch.cuda.synchronize()
    launch_ms = [ev[c][0].elapsed_time(ev[c][1]) for c in range(L)]
    ctx.check()
    # every step computes the same interval: check it reproduced the units
    assert np.array_equal(out["exit_cycle"].cpu().numpy(), exit_np), "steps differ"

    total_psteps, elapsed_max, value = aggregate(psteps * args.steps, elapsed, world)
    # the advection kernel's time in the last timed step: its L launches back
    # to back, as a user runs them
    advect_s = block_ms / 1e3
    # the paper's per-cycle metric leaves out the interval-end work (writer
    # and reseed), timed by its own events in the last step
    end_s = end_ev[0].elapsed_time(end_ev[1]) / 1e3
    cycles_s = elapsed / args.steps - end_s

    # roofline of the advection kernel (dominant): algorithmic bytes of each
    # launch (12 B per touched node, 24 B per live particle, 17 B per
    # termination) over the measured launch durations
    peak, peak_src = hbm_peak()
    algo = algorithmic_bytes(exit_np, nodes_touched, L)
    traffic = None if args.tile else measured_traffic(ctx.launch())
    achieved = float(algo.sum()) / advect_s / 1e9
    frac = achieved / peak

    res = {
        "metric": "RK4 particle-steps/s on 1 GB300 (% of mem roofline); batched & adjoint vs plain",
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed_max / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            **workload_config(args.stride, P, nb, L, dt, args.layout, field_bytes_cycle),
            "ingest": bool(args.ingest),
            "l2": f"inputs larger than L2: each cycle reads a 206 MB field; {nf} distinct fields resident",
            "launch": ctx.launch(),
            "tiling": ctx.tiling(),
            "autotune_ms_per_cycle": tune["ms_per_cycle"] if tune else None,
            "parallelism": f"weak: {world} rank(s), each the full workload, no collective",
        },
        "units_per_step": psteps,
        "nodes_touched_frac": float(nodes_touched.mean() / nodes_total),
        "paper_metric_value": float(psteps) / cycles_s if cycles_s > 0 else None,
        "interval_end_ms": end_s * 1e3,
        "terminated_frac": float(1.0 - valid_np.mean()),
        "gpu_launches": args.steps * (L + 3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": frac,
                     "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": float(algo.mean()),
                     "avg_launch_ms": block_ms / L,
                     "time_base": "CUDA events around the block of 100 launches in the last timed step "
                                  "(none between launches)",
                     "per_launch_events": {
                         "avg_launch_ms": float(np.mean(launch_ms)),
                         "launch_ms_by_decile": [round(float(np.mean(launch_ms[k:k + L // 10])), 4)
                                                 for k in range(0, L, L // 10)],
                         "note": "an extra untimed interval with events around every launch"}},
        "clocks": clk.summary(),
    }

    if not args.no_extras:
        res.update(extras(args, ctx, fields, gfields, table, out, exit_np, psteps, dt, dev, stream, rank, world,
                          ext, org, spc))
    if rank == 0 and world == 1:
        if args.cpu_seconds > 0:
            res["cpu_baseline"] = cpu_baseline(fields, dt, args.cpu_seconds, org)
    ctx.close()
    res["summary"] = summary(res)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def summary(res):
    """The figures of every workload in a few short keys, printed last so
    that a reader of the line's tail sees them: headline value and roofline
    fraction, batched (512 blocks) and large (134M particles) values and
    fractions, adjoint forward + backward against the plain interval."""
    def get(*keys):
        d = res
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) and abs(d) < 10 else d
    iv = (res.get("large") or {}).get("intervals") or [{}]
    return {"value": get("value"), "frac": get("roofline", "frac"), "graph": get("graph_value"),
            "batched_value": get("batched", "batched_value"), "batched_frac": get("batched", "roofline", "frac"),
            "large_value": get("large", "batched_value"), "large_frac": get("large", "roofline", "frac"),
            "accuracy_percent_lattice_delaunay": [
                get("accuracy_vs_global", "reconstructed", "lattice", "accuracy_percent_C_h"),
                get("accuracy_vs_global", "reconstructed", "delaunay", "accuracy_percent_C_h")],
            "large_accuracy_percent_lattice_delaunay": [iv[0].get("accuracy_percent"),
                                                        (iv[0].get("delaunay") or {}).get("accuracy_percent")],
            "adjoint_fwd_bwd_vs_plain": get("adjoint", "forward_backward_vs_plain"),
            "e2e": get("e2e", "value")}


def ctx_layout(args):
    from paper_2004_02003_gb300 import bto
    return bto.BTO_FIELD_F4_AOS if args.layout == "f4" else bto.BTO_FIELD_F3_AOS


def extras(args, ctx, fields, gfields, table, out, exit_ref, psteps, dt, dev, stream, rank, world, ext, org, spc):
    import torch
    from paper_2004_02003_gb300 import bto
    L = INTERVAL
    nb = len(ext)
    res = {}
    # (0) end to end on the headline's own context, right after the headline:
    # fields copied from pinned host memory every cycle, basis flows copied
    # back every interval; copies overlap compute on a second stream with a
    # two-slot device ring.
    res["e2e"] = e2e(args, ctx, fields, dt, dev, stream, nb, world)
    # (1) plain: one single-block context per block, one launch per block and cycle
    plain = [bto.Context(ext[b], org[b], spc[b], STRIDE, L) for b in range(nb)]
    shape = ctx.launch()
    for p in plain:
        p.set_layout(ctx_layout(args))
        p.set_launch(shape["threads_per_cta"], shape["particles_per_thread"], 0, shape["reg_cap"])
    outs = [p.alloc_outputs(dev) for p in plain]

    def plain_step():
        for c in range(L):
            for b in range(nb):
                plain[b].advect(fields[c][b], dt)
        for b in range(nb):
            plain[b].end_interval(outs[b])

    for _ in range(max(1, args.warmup)):
        plain_step()
    torch.cuda.synchronize()
    barrier(world)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        plain_step()
    t1.record(stream)
    torch.cuda.synchronize()
    res["plain_value"] = aggregate(psteps * args.steps, t0.elapsed_time(t1) / 1e3, world)[2]
    for p in plain:
        p.check(); p.close()

    # (2) graph: the interval's cycles as one CUDA graph
    g = bto.Context.batch(ext, org, spc, [STRIDE] * nb, L)
    g.set_layout(ctx_layout(args))
    g.set_launch(shape["threads_per_cta"], shape["particles_per_thread"], 0, shape["reg_cap"])
    gout = g.alloc_outputs(dev)
    for _ in range(max(1, args.warmup)):
        g.interval_graph(table, dt)
        g.end_interval(gout)
    torch.cuda.synchronize()
    barrier(world)
    t0.record(stream)
    for _ in range(args.steps):
        g.interval_graph(table, dt)
        g.end_interval(gout)
    t1.record(stream)
    torch.cuda.synchronize()
    g.check()
    assert np.array_equal(gout["exit_cycle"].cpu().numpy(), exit_ref)
    res["graph_value"] = aggregate(psteps * args.steps, t0.elapsed_time(t1) / 1e3, world)[2]
    g.close()

    # (3) accuracy cost vs the global flow map (rank 0, untimed)
    if rank == 0 and gfields:
        G = GLOBAL_CELLS
        h = 1.0 / G
        gc = bto.Context((G, G, G), (0, 0, 0), (h, h, h), STRIDE, L)
        for c in range(L):
            gc.advect(gfields[c], dt)
        go = gc.end_interval()
        gc.check()
        torch.cuda.synchronize()
        gv = go["valid"].cpu().numpy()
        ge = go["ends"].cpu().numpy().astype(np.float64)
        gce = go["exit_cycle"].cpu().numpy()
        gc.close()
        # global id of each block seed
        n = BLOCK_CELLS // STRIDE
        GS = G // STRIDE
        nbx = G // BLOCK_CELLS
        gid = []
        for bz in range(nbx):
            for by in range(nbx):
                for bx in range(nbx):
                    j = np.arange(n ** 3)
                    jx, jy, jz = j % n + bx * n, (j // n) % n + by * n, j // (n * n) + bz * n
                    gid.append(jx + GS * (jy + GS * jz))
        gid = np.concatenate(gid)
        bv = out["valid"].cpu().numpy()
        be = out["ends"].cpu().numpy().astype(np.float64)
        ok = bv == 1
        dev_cells = float(np.max(np.abs(be[ok] - ge[gid][ok])) / h) if ok.any() else 0.0
        res["accuracy_vs_global"] = {
            "terminated_frac_bto": float(1 - bv.mean()),
            "terminated_frac_global": float(1 - gv.mean()),
            "bto_valid_but_global_invalid": int((ok & (gv[gid] == 0)).sum()),
            "max_valid_end_deviation_cells": dev_cells,
            "global_particle_steps": count_particle_steps(gce, L),
            "reconstructed": reconstruction_metrics(bto, GS, h, STRIDE, gid, be, bv, ge, gv, dev),
        }

    # (4) adjoint and batched workloads against the plain path (rank 0)
    if rank == 0:
        res["tiled_ablation"] = tiled_leg(args, ext, org, spc, table, dt, out, dev, stream)
        res["adjoint"] = adjoint_leg(args, dev, stream)
    res["batched"] = batched_leg(args, dev, stream, rank, world)
    if rank == 0 and not args.no_large:
        res["large"] = large_leg(args, dev, stream)
    return res


def adjoint_leg(args, dev, stream):
    """Adjoint workload (64^3 ABC block on [0, 2 pi]^3, 32^3 seeds, 200 cycles,
    dt 0.01, checkpoints every 16): the plain interval against the tape's
    forward and forward + backward (seed and node-velocity gradients of
    sum over valid particles of |end - seed|^2), same GPU, same fields."""
    import torch
    from paper_2004_02003_gb300 import adjoint, bto, inputs
    n, L, dt, stride, K = (64, 64, 64), 200, 0.01, 2, 16
    h = (2 * np.pi / 64,) * 3
    F = torch.stack([inputs.abc_field_torch(n, (0, 0, 0), h, c * dt, dev) for c in range(L)]).contiguous()
    ctx = bto.Context(n, (0, 0, 0), h, stride, L)
    out = ctx.alloc_outputs(dev)

    def plain():
        for c in range(L):
            ctx.advect(F[c], dt)
        ctx.end_interval(out)

    plain()
    torch.cuda.synchronize()
    seeds = out["seeds"].clone()
    P = seeds.shape[0]
    tape = adjoint.Tape(n, (0, 0, 0), h, P, L, K)

    def fwd():
        return adjoint.flow_map(seeds, F, tape, dt)

    def fwd_bwd():
        s = seeds.clone().requires_grad_(True)
        Fg = F.detach().requires_grad_(True)
        ends, valid, _ = adjoint.flow_map(s, Fg, tape, dt)
        loss = (((ends - s) ** 2).sum(dim=1) * valid.to(torch.float32)).sum()
        loss.backward()
        return s.grad, Fg.grad

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, min(args.steps, 10))
    t_plain = timed(plain, reps)
    t_fwd = timed(fwd, reps)
    t_fb = timed(fwd_bwd, reps)
    ctx.check()
    ex = out["exit_cycle"].cpu().numpy()
    psteps = count_particle_steps(ex, L)
    tape.close()
    ctx.close()
    return {"workload": "64^3 ABC on [0,2pi]^3, 32,768 seeds (stride 2), 200 cycles, dt 0.01, checkpoints every 16",
            "plain_ms": t_plain, "tape_forward_ms": t_fwd, "forward_backward_ms": t_fb,
            "forward_backward_vs_plain": t_fb / t_plain,
            "plain_particle_steps_per_s": psteps / (t_plain / 1e3),
            "valid_frac": float((ex < 0).mean())}


def batched_layout(seed=20040206, nb=512):
    """512 uneven blocks: a 16 x 8 x 4 arrangement of slots over
    [0, 2] x [0, 1] x [0, 1]; block b fills its slot with n_a ~ U{16..96}
    cells per axis (redrawn until max/min <= 3) and a seed stride drawn from
    {1, 2, 4}."""
    rng = np.random.default_rng(seed)
    size = (2.0 / 16, 1.0 / 8, 1.0 / 4)
    ext, org, spc, strides = [], [], [], []
    for k in range(nb):
        ix, iy, iz = k % 16, (k // 16) % 8, k // 128
        while True:
            n = rng.integers(16, 97, size=3)
            if n.max() / n.min() <= 3:
                break
        ext.append(tuple(int(v) for v in n))
        org.append((ix * size[0], iy * size[1], iz * size[2]))
        spc.append(tuple(size[a] / int(n[a]) for a in range(3)))
        strides.append(int(rng.choice([1, 2, 4])))
    return ext, org, spc, strides


def tiled_leg(args, ext, org, spc, table, dt, ref_out, dev, stream,
              shapes=((32, 8, 8, 256), (16, 16, 8, 256), (16, 8, 8, 128))):
    """Ablation on the headline workload: the tiled advection kernel (field
    tiles staged in shared memory by bulk copies, per-step rebinning) against
    the untiled kernel, advect time only, and a bitwise comparison of every
    output with the untiled interval."""
    import torch
    from paper_2004_02003_gb300 import bto
    nb, L = len(ext), INTERVAL
    rows = []
    for sh in shapes:
        ctx = bto.Context.batch(ext, org, spc, [STRIDE] * nb, L)
        ctx.set_tiling(sh[:3], sh[3])
        out = ctx.alloc_outputs(dev)
        for rep in range(2):
            ev = [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(L)]
            for c in range(L):
                ev[c][0].record(stream)
                ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
                ev[c][1].record(stream)
            ctx.end_interval(out)
        torch.cuda.synchronize()
        ctx.check()
        ms = sum(e[0].elapsed_time(e[1]) for e in ev)
        same = all(torch.equal(out[k], ref_out[k]) for k in ("seeds", "ends", "valid", "exit_cycle"))
        psteps = count_particle_steps(out["exit_cycle"].cpu().numpy(), L)
        rows.append({"tile_cells": list(sh[:3]), "threads": sh[3], "tiling": ctx.tiling(),
                     "advect_us_per_cycle": ms * 1e3 / L, "particle_steps_per_s": psteps / (ms / 1e3),
                     "bitwise_equal_untiled": bool(same)})
        ctx.close()
    return rows


def batched_leg(args, dev, stream, rank=0, world=1):
    """Batched workload: 512 uneven blocks in one persistent launch per cycle
    (and as one CUDA graph per interval) against 512 single-block contexts,
    after the native autotuner has picked the launch shape. Under several
    ranks each rank takes its share of the 512 blocks (whole blocks, by
    estimated work) and the values are whole-job figures (strong scaling of
    this fixed workload)."""
    import torch
    from paper_2004_02003_gb300 import bto, inputs
    from paper_2004_02003_gb300.partition import block_work, partition_blocks
    ext_all, org_all, spc_all, strides_all = batched_layout()
    L, NF = 64, max(1, min(4, args.fields))
    parts = partition_blocks(block_work(ext_all, strides_all, L), world)
    mine = parts[rank]
    ext = [ext_all[b] for b in mine]
    org = [org_all[b] for b in mine]
    spc = [spc_all[b] for b in mine]
    strides = [strides_all[b] for b in mine]
    nb = len(ext)
    modes = inputs.fourier_modes(SEED + 2, m=32, kmin=1.0, kmax=16.0, drift_max=0.05)
    vmax = np.pi * inputs.DG_A * 1.5 + 0.1      # bound of |u| (gyre + scaled turbulence)
    dt = 0.25 * min(min(h) for h in spc_all) / vmax
    if nb == 0:      # more ranks than blocks: take part in the collectives only
        for _ in range(3):
            barrier(world)
        for _ in range(3):
            aggregate(0, 0.0, world)
        return None
    fields = [[inputs.double_gyre_fourier_torch(modes, ext[b], org[b], spc[b], c * dt, c, dev)
               for b in range(nb)] for c in range(NF)]
    table = torch.tensor([fields[c % NF][b].data_ptr() for c in range(L) for b in range(nb)],
                         dtype=torch.int64, device=dev)
    nodes = sum((n[0] + 1) * (n[1] + 1) * (n[2] + 1) for n in ext)
    ctx = bto.Context.batch(ext, org, spc, strides, L)
    tune = ctx.autotune(table, 16, dt)
    out = ctx.alloc_outputs(dev)

    def run_batched():
        for c in range(L):
            ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
        ctx.end_interval(out)

    def run_graph():
        ctx.interval_graph(table, dt)
        ctx.end_interval(out)

    def timed(fn, reps, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, min(args.steps, 10))
    barrier(world)
    t_b = timed(run_batched, reps)
    ex = out["exit_cycle"].cpu().numpy()
    psteps = count_particle_steps(ex, L)
    barrier(world)
    t_g = timed(run_graph, reps)
    ctx.check()
    plain = [] if args.no_plain else [bto.Context(ext[b], org[b], spc[b], strides[b], L) for b in range(nb)]
    pouts = [p.alloc_outputs(dev) for p in plain]

    def run_plain():
        for c in range(L):
            for b in range(nb):
                plain[b].advect(fields[c % NF][b], dt)
        for b in range(nb):
            plain[b].end_interval(pouts[b])

    barrier(world)
    t_p = timed(run_plain, 1, warm=1) if not args.no_plain else float("nan")
    for p in plain:
        p.check()
        p.close()
    P = ctx.P
    # whole-job values: all ranks' particle-steps over the slowest rank's time
    v_b = aggregate(psteps, t_b / 1e3, world)[2]
    v_g = aggregate(psteps, t_g / 1e3, world)[2]
    v_p = aggregate(psteps, t_p / 1e3, world)[2]
    # roofline of the batched launch: algorithmic bytes (12 per node of the
    # cells holding a live particle, 24 per live particle, 17 per
    # termination) over the advect-only time of one interval. The touched
    # nodes are counted in an untimed interval at every 8th cycle (held in
    # between); the time is the block of 64 launches with events around the
    # block only, so each launch overlaps the previous one's tail
    act = torch.empty((P, 4), dtype=torch.float32, device=dev)
    touched = np.zeros(L, dtype=np.int64)
    for c in range(L):
        if c % 8 == 0:
            touched[c] = touched_nodes_multi(ctx, act, ext)
        else:
            touched[c] = touched[c - 1]
        ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
    ctx.end_interval(out)
    torch.cuda.synchronize()
    del act
    bev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
    advect_ms = []
    for _ in range(reps):
        bev[0].record(stream)
        for c in range(L):
            ctx.advect_batch(table[c * nb:(c + 1) * nb], dt)
        bev[1].record(stream)
        ctx.end_interval(out)
        torch.cuda.synchronize()
        advect_ms.append(bev[0].elapsed_time(bev[1]))
    ctx.check()
    advect_ms = float(np.median(advect_ms))
    algo = algorithmic_bytes(out["exit_cycle"].cpu().numpy(), touched, L)
    peak, peak_src = hbm_peak()
    achieved = float(algo.sum()) / (advect_ms / 1e3) / 1e9
    ctx.close()
    return {"workload": "512 uneven blocks (16..96 cells per axis, aspect <= 3), strides {1,2,4}, "
                        "double gyre + 32 Fourier modes, interval 64",
            "blocks": nb, "particles": P, "nodes": nodes, "dt": dt, "autotune": tune,
            "ranks": world, "blocks_per_rank": [len(p) for p in parts],
            "batched_value": v_b, "graph_value": v_g, "plain_value": v_p, "batched_vs_plain": v_b / v_p,
            "ms_per_interval": {"batched": t_b, "graph": t_g, "plain": t_p},
            "terminated_frac": float((ex >= 0).mean()),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src, "advect_ms_per_interval": advect_ms,
                         "nodes_touched_frac": float(touched.mean() / nodes)}}


def touched_nodes_multi(ctx, act, ext):
    """touched_nodes for blocks of any extents: the nodes of the cells that
    hold a live particle at the start of the current cycle, all blocks."""
    import torch
    live = ctx.copy_active(act)
    off = ctx.offsets()
    dev = act.device
    nb = len(ext)
    n = torch.tensor(ext, dtype=torch.int64, device=dev)                   # (nb, 3) cells
    nn = n + 1
    nodes = nn.prod(dim=1)
    base = torch.cumsum(nodes, 0) - nodes
    idx = torch.cat([torch.arange(off[b], off[b] + live[b], device=dev) for b in range(nb) if live[b] > 0])
    bid = torch.repeat_interleave(torch.arange(nb, device=dev),
                                  torch.tensor(live, dtype=torch.int64, device=dev))
    x = act[idx, :3]
    cell = torch.minimum(torch.clamp(torch.floor(x).to(torch.int64), min=0), n[bid] - 1)
    mark = torch.zeros(int(nodes.sum().item()), dtype=torch.bool, device=dev)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                k = (cell[:, 0] + dx) + nn[bid, 0] * ((cell[:, 1] + dy) + nn[bid, 1] * (cell[:, 2] + dz))
                mark[base[bid] + k] = True
    return int(mark.sum().item())


def large_leg(args, dev, stream):
    """Large in situ emulation: a 512^3-cell domain as 4 x 4 x 4 blocks of 128^3
    cells, one seed per cell (134,217,728 particles), 128 Fourier modes,
    dt = 0.2 cell / max|u|, 3 intervals of 50 cycles. Every cycle the
    stand-in simulation writes that cycle's field on the device (the global
    513^3 node grid in single precision and its 64 block copies, timed
    separately), then the batched form (one launch), the plain form (64
    contexts, 64 launches) and the global flow map (one block over the whole
    domain: particles cross the block faces) each take one cycle, and 1000
    new pathlines take one RK4 step through the same field (ground truth for
    the stitching of f3)."""
    import torch
    from paper_2004_02003_gb300 import adjoint, bto, inputs
    G, n, S, L, NI = 512, 128, 1, 50, 3
    h = 1.0 / G
    dt = 0.2 * h
    nbx = G // n
    modes = inputs.fourier_modes(SEED + 4, m=128, kmin=1.0, kmax=16.0, drift_max=0.05)
    blocks = [(bx, by, bz) for bz in range(nbx) for by in range(nbx) for bx in range(nbx)]
    ext = [(n, n, n)] * len(blocks)
    org = [(b[0] * n * h, b[1] * n * h, b[2] * n * h) for b in blocks]
    spc = [(h, h, h)] * len(blocks)
    nb = len(blocks)

    def simulate(cyc):
        gf = inputs.fourier_field_torch(modes, (G, G, G), (0, 0, 0), (h, h, h), cyc, dev, dtype=torch.float32)
        bf = [gf[bz * n: bz * n + n + 1, by * n: by * n + n + 1, bx * n: bx * n + n + 1].contiguous()
              for (bx, by, bz) in blocks]
        return gf, bf

    bctx = bto.Context.batch(ext, org, spc, [S] * nb, L)
    # the library's autotuner picks the batched launch shape on cycle 0's
    # field (each of its shapes advances 4 cycles of it)
    gf, bf = simulate(0)
    tune_table = torch.tensor([t.data_ptr() for t in bf] * 4, dtype=torch.int64, device=dev)
    tune = bctx.autotune(tune_table, 4, dt)
    del gf, bf, tune_table
    gctx = bto.Context((G, G, G), (0, 0, 0), (h, h, h), S, L)
    plain = [bto.Context(ext[b], org[b], spc[b], S, L) for b in range(nb)]
    bout, gout = bctx.alloc_outputs(dev), gctx.alloc_outputs(dev)
    pouts = [p.alloc_outputs(dev) for p in plain]
    # global id of each block seed (stride 1: seeds are the block's nodes)
    j = torch.arange(n ** 3, device=dev)
    jx, jy, jz = j % n, (j // n) % n, j // (n * n)
    gid = torch.cat([(jx + b[0] * n) + G * ((jy + b[1] * n) + G * (jz + b[2] * n)) for b in blocks])
    # new pathlines: starts well inside the domain (150 steps of at most
    # 0.2 cells cannot reach a face), one RK4 step per cycle (1-cycle tape)
    nq = 1000
    starts = torch.from_numpy(np.random.default_rng(SEED + 5).uniform(0.1, 0.9, size=(nq, 3)).astype(np.float32)).to(dev)
    tape = adjoint.Tape((G, G, G), (0, 0, 0), (h, h, h), nq, 1, 1)
    cur, truth = starts.clone(), [starts.clone()]
    tval = torch.empty((nq,), dtype=torch.uint8, device=dev)
    t_sim = t_b = t_p = t_g = t_wb = 0.0
    report = []
    filled_sets, global_sets = [], []
    psteps_total = 0
    algo_total = 0
    # touched nodes for the roofline: counted (untimed) before every 10th
    # cycle of the batched context and held in between
    act = torch.empty((bctx.P, 4), dtype=torch.float32, device=dev)
    for k in range(NI):
        evs = []
        touched = np.zeros(L, dtype=np.int64)
        for c in range(L):
            touched[c] = touched_nodes(bctx, act, n, nb) if c % 10 == 0 else touched[c - 1]
            e = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
            e[0].record(stream)
            gf, bf = simulate(k * L + c)
            table = torch.tensor([t.data_ptr() for t in bf], dtype=torch.int64, device=dev)
            e[1].record(stream)
            e[2].record(stream)
            bctx.advect_batch(table, dt)
            e[3].record(stream)
            e[4].record(stream)
            for b in range(nb):
                plain[b].advect(bf[b], dt)
            e[5].record(stream)
            e[6].record(stream)
            gctx.advect(gf, dt)
            e[7].record(stream)
            ftab = torch.tensor([gf.data_ptr()], dtype=torch.int64, device=dev)
            nxt = torch.empty_like(cur)
            bto.bto_tape_forward(tape.handle, cur, ftab, dt, nxt, tval, None)
            cur = nxt
            evs.append(e)
            del gf, bf
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        bctx.end_interval(bout)
        w1.record(stream)
        for b in range(nb):
            plain[b].end_interval(pouts[b])
        gctx.end_interval(gout)
        torch.cuda.synchronize()
        truth.append(cur.clone())
        for e in evs:
            t_sim += e[0].elapsed_time(e[1])
            t_b += e[2].elapsed_time(e[3])
            t_p += e[4].elapsed_time(e[5])
            t_g += e[6].elapsed_time(e[7])
        t_wb += w0.elapsed_time(w1)
        bv = bout["valid"] == 1
        gv = gout["valid"][gid] == 1
        both = bv & gv          # a BTO-valid particle can leave the domain in the global map only by rounding
        d = ((bout["ends"][both] - gout["ends"][gid][both]).abs().amax(dim=1) / h).double()
        q = torch.quantile(d[torch.randperm(d.numel(), device=dev)[:1 << 24]],
                           torch.tensor([0.5, 0.99, 0.9999], dtype=torch.float64, device=dev)).tolist()
        dev_max = d.max().item()
        ex = bout["exit_cycle"].cpu().numpy()
        psteps_total += count_particle_steps(ex, L)
        algo_total += int(algorithmic_bytes(ex, touched, L).sum())
        # reconstruction of the missing BTO basis flows on the global seed
        # lattice (f2) and the paper's accuracy metrics against the global
        # map (Sec. 4.3: total average L2, max L2, Accuracy% with C = h)
        lat_e = torch.empty((G ** 3, 3), dtype=torch.float32, device=dev)
        lat_v = torch.empty((G ** 3,), dtype=torch.uint8, device=dev)
        lat_e[gid] = bout["ends"]
        lat_v[gid] = bout["valid"]
        filled = torch.empty_like(lat_e)
        status = torch.empty_like(lat_v)
        bto.bto_fill_lattice((G, G, G), lat_e, lat_v, filled, status)
        ok = (gout["valid"] == 1) & (status > 0)
        err = (filled[ok].double() - gout["ends"][ok].double()).norm(dim=1)
        l2, mx = err.mean().item(), err.max().item()
        filled_sets.append(filled)
        global_sets.append(gout["ends"].clone())
        # the paper's own reconstruction: Delaunay triangulation of the valid
        # basis flows of all blocks, barycentric interpolation (Sec. 3.2);
        # first interval only (a post hoc step of seconds)
        delaunay = None
        if k == 0:
            delaunay = delaunay_fill_report(bto, G, h, lat_e, lat_v, gout, filled, status, ok, stream)
        del lat_e, lat_v
        report.append({"interval": k, "terminated_frac_bto": float(1 - bv.float().mean().item()),
                       "terminated_frac_global": float(1 - (gout["valid"] == 1).float().mean().item()),
                       "bto_valid_not_global_valid": int((bv & ~gv).sum().item()),
                       "max_valid_end_deviation_cells": dev_max,
                       "valid_end_deviation_cells_p50_p99_p9999": q,
                       "still_missing_after_fill": int((status == 0).sum().item()),
                       "total_average_l2": l2, "max_l2": mx,
                       "accuracy_percent": (h - l2) / h * 100.0,
                       **({"delaunay": delaunay} if delaunay else {})})
    tape.close()
    del act
    for p in plain:
        p.check()
    bctx.check(); gctx.check()
    P = bctx.P
    for p in plain:
        p.close()
    bctx.close(); gctx.close()
    # new pathlines (Sec. 3.2 / 4.3 second context): stitched through the 3
    # intervals' basis flows of BTO (reconstructed) and of the global map,
    # against the RK4 ground truth advected without interval resets
    # (trilinear over the lattice cell, and the paper's barycentric
    # coordinates in the cell's Kuhn tetrahedron)
    paths = {}
    for name, sets in (("bto", filled_sets), ("global", global_sets)):
        table = torch.tensor([t.data_ptr() for t in sets], dtype=torch.int64, device=dev)
        for scheme, suffix in ((bto.BTO_STITCH_TRILINEAR, ""), (bto.BTO_STITCH_BARYCENTRIC, "_barycentric")):
            path = torch.empty((NI + 1, nq, 3), dtype=torch.float32, device=dev)
            bto.bto_stitch_pathlines_ex((G, G, G), (0, 0, 0), (h, h, h), NI, table, nq, starts, path, scheme)
            paths[name + suffix] = path
    torch.cuda.synchronize()
    path_err = []
    for k in range(1, NI + 1):
        row = {"after_interval": k}
        for name in ("bto", "global", "bto_barycentric", "global_barycentric"):
            e = (paths[name][k] - truth[k]).double().norm(dim=1) / h
            fin = torch.isfinite(e)
            row[name + "_mean_l2_cells"] = e[fin].mean().item() if fin.any() else None
            row[name + "_max_l2_cells"] = e[fin].max().item() if fin.any() else None
            row[name + "_pathlines"] = int(fin.sum().item())
        path_err.append(row)
    maxes = [r["max_l2"] for r in report]
    cyc = NI * L
    peak, peak_src = hbm_peak()
    return {"workload": "512^3 cells as 4x4x4 blocks of 128^3, 1 seed per cell, 128 Fourier modes, "
                        "3 intervals of 50 cycles, dt = 0.2 cell/max|u|; each cycle's field generated on the "
                        "device before the cycle (single-precision Fourier sum, timed separately)",
            "particles": P, "batched_launch": tune["best"],
            "batched_value": psteps_total / (t_b / 1e3), "plain_value": psteps_total / (t_p / 1e3),
            "batched_advect_ms_per_cycle": t_b / cyc, "plain_advect_ms_per_cycle": t_p / cyc,
            "global_advect_ms_per_cycle": t_g / cyc, "simulation_ms_per_cycle": t_sim / cyc,
            "batched_writer_ms_per_interval": t_wb / NI,
            "roofline": {"bound": "hbm", "achieved": algo_total / (t_b / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": algo_total / (t_b / 1e3) / 1e9 / peak, "peak_source": peak_src,
                         "algorithmic_bytes_per_cycle": algo_total / cyc,
                         "time_base": "CUDA events around each batched launch (one launch per cycle)"},
            "intervals": report,
            "greatest_max_l2": max(maxes), "average_max_l2": float(np.mean(maxes)),
            "pathlines_vs_rk4_ground_truth": path_err}


def reconstruction_metrics(bto, GS, h, stride, gid, be, bv, ge, gv, dev):
    """The paper's accuracy metrics (Sec. 4.3) of one interval's BTO basis
    flows against the global map after the missing entries of the global seed
    lattice (GS^3) are filled, by the lattice fill and by the Delaunay fill:
    total average L2 and max L2 over the entries valid in the global map and
    filled, Accuracy% with C = h and with C = stride * h (the seed spacing)."""
    import torch
    P = GS ** 3
    lat_e = torch.full((P, 3), float("nan"), dtype=torch.float32, device=dev)
    lat_v = torch.zeros((P,), dtype=torch.uint8, device=dev)
    gidt = torch.from_numpy(gid).to(dev)
    lat_e[gidt] = torch.from_numpy(be.astype(np.float32)).to(dev)
    lat_v[gidt] = torch.from_numpy(bv).to(dev)
    gvt = torch.from_numpy(gv).to(dev) == 1
    get = torch.from_numpy(ge).to(dev)
    outm = {}
    for name, fill in (("lattice", bto.bto_fill_lattice), ("delaunay", bto.bto_fill_delaunay)):
        f = torch.empty_like(lat_e)
        st = torch.empty_like(lat_v)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fill((GS, GS, GS), lat_e, lat_v, f, st)
        e1.record()
        torch.cuda.synchronize()
        okm = gvt & (st > 0)
        err = (f[okm].double() - get[okm]).norm(dim=1)
        l2, mx = err.mean().item(), err.max().item()
        outm[name] = {"total_average_l2": l2, "max_l2": mx,
                      "accuracy_percent_C_h": (h - l2) / h * 100.0,
                      "accuracy_percent_C_seed_spacing": (stride * h - l2) / (stride * h) * 100.0,
                      "filled": int((st == 2).sum().item()), "still_missing": int((st == 0).sum().item()),
                      "still_missing_valid_in_global_map": int(((st == 0) & gvt).sum().item()),
                      "fill_ms": e0.elapsed_time(e1)}
    return outm


def delaunay_fill_report(bto, G, h, lat_e, lat_v, gout, filled, status, ok, stream):
    """The Delaunay reconstruction (bto_fill_delaunay) of one interval's
    global seed lattice, its accuracy against the global map (Sec. 4.3) and
    its time, beside the lattice fill's on the entries both fill."""
    import torch
    dfill = torch.empty_like(lat_e)
    dstat = torch.empty_like(lat_v)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    bto.bto_fill_delaunay((G, G, G), lat_e, lat_v, dfill, dstat)
    d1.record(stream)
    torch.cuda.synchronize()
    okd = (gout["valid"] == 1) & (dstat > 0)
    errd = (dfill[okd].double() - gout["ends"][okd].double()).norm(dim=1)
    l2d, mxd = errd.mean().item(), errd.max().item()
    both_f = okd & ok & (status == 2) & (dstat == 2)
    el = (filled[both_f].double() - gout["ends"][both_f].double()).norm(dim=1)
    ed = (dfill[both_f].double() - gout["ends"][both_f].double()).norm(dim=1)
    # where the entries left missing lie: on the lattice's boundary faces,
    # and how many of them the global map keeps valid (lattice fill, Delaunay)
    j = torch.arange(G ** 3, device=dstat.device, dtype=torch.int32)
    jx, jy, jz = j % G, (j // G) % G, j // (G * G)
    face = (jx == 0) | (jx == G - 1) | (jy == 0) | (jy == G - 1) | (jz == 0) | (jz == G - 1)
    del j, jx, jy, jz
    gval = gout["valid"] == 1
    miss_d = dstat == 0
    return {"total_average_l2": l2d, "max_l2": mxd, "accuracy_percent": (h - l2d) / h * 100.0,
            "still_missing_after_fill": int(miss_d.sum().item()), "filled": int((dstat == 2).sum().item()),
            "still_missing_on_boundary_faces": int((miss_d & face).sum().item()),
            "still_missing_valid_in_global_map_lattice_delaunay": [int(((status == 0) & gval).sum().item()),
                                                                   int((miss_d & gval).sum().item())],
            "still_missing_valid_in_global_map_on_boundary_faces": int((miss_d & gval & face).sum().item()),
            "fill_ms": d0.elapsed_time(d1),
            "filled_by_both": int(both_f.sum().item()),
            "mean_l2_on_entries_both_fill_lattice_delaunay": [el.mean().item(), ed.mean().item()],
            "max_l2_on_entries_both_fill_lattice_delaunay": [el.max().item(), ed.max().item()]}


def e2e(args, ctx, fields, dt, dev, stream, nb, world=1):
    import torch
    L = INTERVAL
    R = 8  # pinned host ring of per-cycle fields (cycle c uses host[c % R])
    # each cycle's block fields lie side by side, on the host and in the two
    # device slots, so that a copy stream moves its share in one copy
    shape = tuple(fields[0][0].shape)
    host = [torch.empty((nb,) + shape, dtype=torch.float32, pin_memory=True) for _ in range(R)]
    for r in range(R):
        for b in range(nb):
            host[r][b].copy_(fields[r][b])
    slots = [torch.empty((nb,) + shape, dtype=torch.float32, device=dev) for _ in range(2)]
    slot_ptrs = [torch.tensor([slot[b].data_ptr() for b in range(nb)], dtype=torch.int64, device=dev)
                 for slot in slots]
    def host_out():
        return {"seeds": torch.empty((ctx.P, 3), dtype=torch.float32, pin_memory=True),
                "ends": torch.empty((ctx.P, 3), dtype=torch.float32, pin_memory=True),
                "valid": torch.empty((ctx.P,), dtype=torch.uint8, pin_memory=True),
                "exit_cycle": torch.empty((ctx.P,), dtype=torch.int32, pin_memory=True)}
    out_host = [host_out(), host_out()]      # interval k's results land in out_host[k % 2]
    # each cycle's block fields are split over K copy streams, one copy of
    # contiguous blocks each (concurrent copies contend for the host link:
    # one stream measured fastest)
    K = max(1, min(args.e2e_streams, nb))
    chunks = [(j * nb // K, (j + 1) * nb // K) for j in range(K)]
    copy_streams = [torch.cuda.Stream(device=dev) for _ in range(K)]
    out_dev = ctx.alloc_outputs(dev)
    copied = [[torch.cuda.Event() for _ in range(K)] for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    landed = [torch.cuda.Event() for _ in range(2)]
    h2d_bytes = host[0].numel() * 4
    d2h_bytes = sum(t.numel() * t.element_size() for t in out_host[0].values())
    gc = [0]                                   # cycles enqueued so far (slot parity)

    def enqueue(k):
        """Interval k: per cycle, the fields' host-to-device copies (two-slot
        device ring, copies of the next cycle overlap the current advection),
        the advection, then the writer and the results' copy back."""
        for c in range(L):
            s = gc[0] & 1
            for j, cs in enumerate(copy_streams):
                with torch.cuda.stream(cs):
                    if gc[0] >= 2:
                        cs.wait_event(consumed[s])
                    b0, b1 = chunks[j]
                    slots[s][b0:b1].copy_(host[c % R][b0:b1], non_blocking=True)
                    copied[s][j].record(cs)
            for j in range(K):
                stream.wait_event(copied[s][j])
            ctx.advect_batch(slot_ptrs[s], dt)
            consumed[s].record(stream)
            gc[0] += 1
        ctx.end_interval(out_dev)
        for key in out_dev:
            out_host[k % 2][key].copy_(out_dev[key], non_blocking=True)
        landed[k % 2].record(stream)

    def run(n):
        """n intervals, each enqueued before the previous one's results are
        read on the host, so that the copy engines never wait for the host."""
        units = 0
        for k in range(n + 1):
            if k < n:
                enqueue(k)
            if k >= 1:
                landed[(k - 1) % 2].synchronize()
                units += count_particle_steps(out_host[(k - 1) % 2]["exit_cycle"].numpy(), L)
        return units

    run(max(1, args.warmup))
    barrier(world)
    t = time.perf_counter()
    units = run(args.steps)
    el = time.perf_counter() - t
    # whole job: all ranks' units over the slowest rank's time
    _, _, value = aggregate(units, el, world)
    # this machine's host link: the same per-cycle copies alone, one interval's
    # worth back to back on the copy stream (no kernels), and the end-to-end
    # rate those copies would allow
    cs = copy_streams[0]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c0.record(cs)
    with torch.cuda.stream(cs):
        for c in range(L):
            slots[c & 1].copy_(host[c % R], non_blocking=True)
    c1.record(cs)
    torch.cuda.synchronize()
    link_gbs = h2d_bytes * L / (c0.elapsed_time(c1) * 1e-3) / 1e9
    per_interval = units / max(1, args.steps)
    return {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d_bytes * L,
            "d2h_bytes_per_step": d2h_bytes, "host_field_ring": R, "copy_streams": K,
            "h2d_gbs_copies_alone": link_gbs,
            "ceiling_value_from_copies_alone": per_interval * world / (h2d_bytes * L / (link_gbs * 1e9))}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------
def cpu_baseline(fields, dt, seconds, org):
    """The oracle on the same workload (every block, all 100 cycles), block
    by block, until ``seconds`` of oracle time have been spent."""
    import oracle
    h = 1.0 / GLOBAL_CELLS
    nthreads = oracle.max_threads()
    steps, spent, done = 0, 0.0, []
    for b in range(len(org)):
        if spent >= seconds:
            break
        g = oracle.Grid.make((BLOCK_CELLS,) * 3, org[b], (h, h, h))
        st = oracle.State(oracle.seeds(g, STRIDE))
        c = 0
        while c < INTERVAL and spent < seconds:
            f = fields[c][b].cpu().numpy()
            live = int((st.exit_cycle < 0).sum())
            t = time.perf_counter()
            oracle.cycle(g, f, dt, c, st)
            spent += time.perf_counter() - t
            steps += live
            c += 1
        done.append(f"block {b}: cycles 0..{c - 1}")
    return {"value": steps / spent, "unit": "particle-steps/s", "cores": nthreads, "host_cpus": os.cpu_count(),
            "kind": "oracle",
            "sample": f"turb256 workload, {'; '.join(done)} ({steps} particle-steps, {spent:.1f} s of oracle time)",
            "other_configs": oracle_other_configs()}


def oracle_other_configs():
    """The oracle's rate on the ABC block (all 4096 seeds, 50 cycles) and on
    the adjoint workload (4096 of its 32,768 seeds, 200 cycles: forward, and
    forward plus the discrete adjoint)."""
    import oracle
    from paper_2004_02003_gb300 import inputs
    res = {}
    n, h, L, dt = (32, 32, 32), (1.0 / 32,) * 3, 50, 0.01
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    g = oracle.Grid.make(n, (0, 0, 0), h)
    t = time.perf_counter()
    st = oracle.run_interval(g, 2, L, dt, lambda c: fields[c])
    el = time.perf_counter() - t
    res["abc_32"] = {"particle_steps": count_particle_steps(st.exit_cycle, L),
                     "particle_steps_per_s": count_particle_steps(st.exit_cycle, L) / el}
    n, L, dt = (64, 64, 64), 200, 0.01
    h = (2 * np.pi / 64,) * 3
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    g = oracle.Grid.make(n, (0, 0, 0), h)
    seeds = oracle.seeds(g, 2)
    ids = np.sort(np.random.default_rng(SEED + 9).choice(seeds.shape[0], size=4096, replace=False))
    t = time.perf_counter()
    st, _ = oracle.forward_with_history(g, lambda c: fields[c], dt, seeds[ids], L)
    t_f = time.perf_counter() - t
    up = 2.0 * (st.x - seeds[ids]) * st.valid[:, None]
    t = time.perf_counter()
    oracle.vjp(g, lambda c: fields[c], dt, seeds[ids], L, up, want_field_grads=True)
    t_fb = time.perf_counter() - t
    ps = count_particle_steps(st.exit_cycle, L)
    res["adjoint_64"] = {"sample_seeds": 4096, "particle_steps": ps, "forward_particle_steps_per_s": ps / t_f,
                         "forward_backward_s": t_fb, "forward_backward_particle_steps_per_s": ps / t_fb}
    return res


def workload_config(stride, P, nb, L, dt, layout, field_bytes_cycle):
    """The keys that define the benchmark's workload, shared by both arms."""
    return {
        "workload": "turb256: 256^3 cells as 2x2x2 blocks of 128^3, Fourier turbulence (64 modes), "
                    f"stride {stride} ({P:,} particles), interval {L}, dt=0.25 cell/max|u|",
        "blocks": nb, "particles": P, "interval_cycles": L, "dt": dt,
        "field_layout": layout.upper() + "_AOS", "field_bytes_per_cycle": field_bytes_cycle,
    }


def run_reference(args):
    """The oracle timed as the reference arm (rank 0 only, bounded sample)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    from paper_2004_02003_gb300 import inputs
    import oracle
    oracle.build()
    modes = inputs.fourier_modes(SEED, m=NMODES, kmin=1.0, kmax=16.0, drift_max=0.05)
    h = 1.0 / GLOBAL_CELLS
    dt = 0.25 * h
    g = oracle.Grid.make((BLOCK_CELLS,) * 3, (0, 0, 0), (h, h, h))
    nb = len(block_layout(0, 1)[0])
    # a bounded sample per step: 8192 particles of block 0 over the full interval
    rng = np.random.default_rng(SEED)
    ids = np.sort(rng.choice(oracle.num_seeds(g, STRIDE), size=8192, replace=False))
    fields = [inputs.fourier_field(modes, (BLOCK_CELLS,) * 3, (0, 0, 0), (h, h, h), c) for c in range(INTERVAL)]

    def step():
        st = oracle.State(oracle.seeds(g, STRIDE, ids))
        n = 0
        for c in range(INTERVAL):
            n += int((st.exit_cycle < 0).sum())
            oracle.cycle(g, fields[c], dt, c, st)
        return n

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units += step()
    el = time.perf_counter() - t
    v = units / el
    print(json.dumps({
        "impl": "reference", "metric": "RK4 particle-steps/s on 1 GB300 (% of mem roofline); batched & adjoint vs plain",
        "value": v, "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(STRIDE, nb * oracle.num_seeds(g, STRIDE), nb, INTERVAL, dt, "f3",
                                  nb * (BLOCK_CELLS + 1) ** 3 * 12),
        "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": "8192 random particles of block 0 of 8, all 100 cycles, per step"},
        "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_only(args):
    """One workload leg alone on one GPU (its own JSON line, not the
    benchmark's): a short command to capture that leg's kernels."""
    import torch
    from paper_2004_02003_gb300 import bto
    from paper_2004_02003_gb300 import build as lib_build
    lib_build.build()
    bto.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    if args.only == "batched":
        print(json.dumps({"leg": "batched", "result": batched_leg(args, dev, stream)}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
