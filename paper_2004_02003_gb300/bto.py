"""Thin ctypes binding of libbto (include/bto.h): argument marshalling only.

Every function keeps the C name and forwards to the CUDA library; nothing is
computed here. Device buffers may be given as torch CUDA tensors (their
``data_ptr()`` is passed) or as integer device addresses. Streams default to
torch's current stream on the current device.

The library must have been built (``paper_2004_02003_gb300.build.build()`` or
``__graft_entry__.build()``); importing works without it, but the first call
raises :class:`BtoError` if ``libbto.so`` is missing. There is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbto.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bto.h")

BTO_OK = 0
BTO_ERR_INVALID_ARG = 1
BTO_ERR_STATE = 2
BTO_ERR_CUDA = 3
BTO_ERR_OOM = 4
BTO_ERR_TIMEOUT = 5
BTO_ERR_UNSUPPORTED = 6
BTO_ERR_BOUNDS = 7
BTO_FIELD_F3_AOS = 0
BTO_FIELD_F4_AOS = 1
BTO_STITCH_TRILINEAR = 0
BTO_STITCH_BARYCENTRIC = 1

_lib = None

# C types of the device allocator hook (include/bto.h)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
# Every allocator callback pair ever installed, kept alive for the life of
# the process: a context or tape keeps the hook it was created with and may
# free through it after another hook (or none) has been installed.
_allocator_refs = []


class BtoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status) if _lib else status} (status {status})")


def _declare(lib):
    c_i32p = ctypes.POINTER(ctypes.c_int32)
    c_i64p = ctypes.POINTER(ctypes.c_int64)
    c_u64p = ctypes.POINTER(ctypes.c_uint64)
    c_fp = ctypes.POINTER(ctypes.c_float)
    vp = ctypes.c_void_p
    sig = {
        "bto_create": ([c_i32p, c_fp, c_fp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)], ctypes.c_int),
        "bto_batch_create": ([ctypes.c_int32, c_i32p, c_fp, c_fp, c_i32p, ctypes.c_int32,
                              ctypes.POINTER(vp)], ctypes.c_int),
        "bto_set_field_layout": ([vp, ctypes.c_int], ctypes.c_int),
        "bto_set_ingest": ([vp, ctypes.c_int32], ctypes.c_int),
        "bto_num_seeds": ([vp], ctypes.c_int64),
        "bto_num_blocks": ([vp], ctypes.c_int32),
        "bto_batch_offsets": ([vp, c_i64p], ctypes.c_int),
        "bto_advect_cycle": ([vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "bto_batch_advect_cycle": ([vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "bto_end_interval": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_end_interval_ex": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_launch_interval_graph": ([vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "bto_set_launch": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "bto_get_launch": ([vp, c_i32p], ctypes.c_int),
        "bto_set_tiling": ([vp, c_i32p, ctypes.c_int32], ctypes.c_int),
        "bto_get_tiling": ([vp, c_i32p], ctypes.c_int),
        "bto_test_wait_timeout": ([vp, ctypes.c_int32], ctypes.c_int),
        "bto_autotune": ([vp, vp, ctypes.c_int32, ctypes.c_float, vp, c_i32p, c_fp], ctypes.c_int),
        "bto_copy_active": ([vp, vp, c_i32p, vp], ctypes.c_int),
        "bto_last_error": ([vp], ctypes.c_int),
        "bto_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "bto_interval_noalloc": ([c_i32p, c_fp, c_fp, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_float,
                                  vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_destroy": ([vp], None),
        "bto_set_device_allocator": ([ALLOC_FN, FREE_FN, vp], ctypes.c_int),
        "bto_check_bounds_build": ([], ctypes.c_int32),
        "bto_bounds_failures": ([c_u64p, ctypes.c_int32], ctypes.c_int),
        "bto_fill_lattice": ([c_i32p, vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_fill_delaunay": ([c_i32p, vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_stitch_pathlines": ([c_i32p, c_fp, c_fp, ctypes.c_int32, vp, ctypes.c_int64, vp, vp, vp],
                                 ctypes.c_int),
        "bto_stitch_pathlines_ex": ([c_i32p, c_fp, c_fp, ctypes.c_int32, vp, ctypes.c_int64, vp, vp,
                                     ctypes.c_int32, vp], ctypes.c_int),
        "bto_tape_create": ([c_i32p, c_fp, c_fp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                             ctypes.POINTER(vp)], ctypes.c_int),
        "bto_tape_num_particles": ([vp], ctypes.c_int64),
        "bto_tape_forward": ([vp, vp, vp, ctypes.c_float, vp, vp, vp, vp], ctypes.c_int),
        "bto_tape_backward": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "bto_tape_jacobian": ([vp, vp, vp], ctypes.c_int),
        "bto_tape_ftle": ([vp, vp, vp, vp], ctypes.c_int),
        "bto_tape_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


def load():
    """Load libbto.so (raises BtoError if it has not been built). The
    environment variable BTO_LIBRARY names another build of the same library
    to load instead (the bounds-checked build, for instance)."""
    global _lib
    if _lib is None:
        path = os.environ.get("BTO_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise BtoError(BTO_ERR_UNSUPPORTED, f"libbto not built ({path} missing)")
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
    return _lib


def header_functions() -> list:
    """Names of the functions declared in include/bto.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bto_[a-z_0-9]+)\s*\(", text)))


def status_string(status: int) -> str:
    return load().bto_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != BTO_OK:
        raise BtoError(status, where)


def _addr(buf) -> int:
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    return int(buf.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _arr(ctype, values):
    values = list(values)
    return (ctype * len(values))(*values)


def bto_create(extent_cells, origin, spacing, seed_stride: int, interval_cycles: int) -> int:
    out = ctypes.c_void_p()
    _check(load().bto_create(_arr(ctypes.c_int32, extent_cells), _arr(ctypes.c_float, origin),
                             _arr(ctypes.c_float, spacing), int(seed_stride), int(interval_cycles),
                             ctypes.byref(out)), "bto_create")
    return out.value


def bto_batch_create(extents, origins, spacings, strides, interval_cycles: int) -> int:
    ext = [int(v) for e in extents for v in e]
    org = [float(v) for o in origins for v in o]
    spc = [float(v) for s in spacings for v in s]
    nb = len(strides)
    if len(ext) != 3 * nb or len(org) != 3 * nb or len(spc) != 3 * nb:
        raise BtoError(BTO_ERR_INVALID_ARG, "bto_batch_create: array lengths")
    out = ctypes.c_void_p()
    _check(load().bto_batch_create(nb, _arr(ctypes.c_int32, ext), _arr(ctypes.c_float, org),
                                   _arr(ctypes.c_float, spc), _arr(ctypes.c_int32, strides),
                                   int(interval_cycles), ctypes.byref(out)), "bto_batch_create")
    return out.value


def bto_set_field_layout(ctx: int, layout: int) -> None:
    _check(load().bto_set_field_layout(ctx, int(layout)), "bto_set_field_layout")


def bto_set_ingest(ctx: int, enable: int) -> None:
    _check(load().bto_set_ingest(ctx, int(enable)), "bto_set_ingest")


def bto_num_seeds(ctx: int) -> int:
    return int(load().bto_num_seeds(ctx))


def bto_num_blocks(ctx: int) -> int:
    return int(load().bto_num_blocks(ctx))


def bto_batch_offsets(ctx: int) -> list:
    nb = bto_num_blocks(ctx)
    buf = (ctypes.c_int64 * (nb + 1))()
    _check(load().bto_batch_offsets(ctx, buf), "bto_batch_offsets")
    return list(buf)


def bto_advect_cycle(ctx: int, d_field, dt: float, stream=None) -> None:
    _check(load().bto_advect_cycle(ctx, _addr(d_field), float(dt), _stream(stream)), "bto_advect_cycle")


def bto_batch_advect_cycle(ctx: int, d_fields, dt: float, stream=None) -> None:
    _check(load().bto_batch_advect_cycle(ctx, _addr(d_fields), float(dt), _stream(stream)),
           "bto_batch_advect_cycle")


def bto_end_interval(ctx: int, d_seeds, d_ends, d_valid, d_exit_cycle=None, stream=None) -> None:
    _check(load().bto_end_interval(ctx, _addr(d_seeds), _addr(d_ends), _addr(d_valid),
                                   _addr(d_exit_cycle), _stream(stream)), "bto_end_interval")


def bto_end_interval_ex(ctx: int, d_seeds, d_ends, d_valid, d_exit_cycle=None, d_exit_pos=None,
                        d_exit_time=None, stream=None) -> None:
    _check(load().bto_end_interval_ex(ctx, _addr(d_seeds), _addr(d_ends), _addr(d_valid), _addr(d_exit_cycle),
                                      _addr(d_exit_pos), _addr(d_exit_time), _stream(stream)),
           "bto_end_interval_ex")


def bto_launch_interval_graph(ctx: int, d_field_table, dt: float, stream=None) -> None:
    _check(load().bto_launch_interval_graph(ctx, _addr(d_field_table), float(dt), _stream(stream)),
           "bto_launch_interval_graph")


def bto_set_launch(ctx: int, threads_per_cta: int, particles_per_thread: int, ctas_per_sm: int = 0,
                   reg_cap: int = 0) -> None:
    _check(load().bto_set_launch(ctx, int(threads_per_cta), int(particles_per_thread), int(ctas_per_sm),
                                 int(reg_cap)), "bto_set_launch")


def bto_get_launch(ctx: int) -> dict:
    buf = (ctypes.c_int32 * 5)()
    _check(load().bto_get_launch(ctx, buf), "bto_get_launch")
    return {"threads_per_cta": buf[0], "particles_per_thread": buf[1], "ctas_per_sm": buf[2],
            "reg_cap": buf[3], "grid": buf[4]}


def bto_set_tiling(ctx: int, tile_cells, threads_per_cta: int = 256) -> None:
    """tile_cells = None or (0, 0, 0) switches tiling off."""
    arr = None if tile_cells is None else _arr(ctypes.c_int32, [int(v) for v in tile_cells])
    _check(load().bto_set_tiling(ctx, arr, int(threads_per_cta)), "bto_set_tiling")


def bto_test_wait_timeout(ctx: int, cycles: int) -> None:
    _check(load().bto_test_wait_timeout(ctx, int(cycles)), "bto_test_wait_timeout")


def bto_get_tiling(ctx: int) -> dict:
    buf = (ctypes.c_int32 * 8)()
    _check(load().bto_get_tiling(ctx, buf), "bto_get_tiling")
    return {"tile_cells": (buf[0], buf[1], buf[2]), "threads_per_cta": buf[3], "grid": buf[4], "tiles": buf[5],
            "buffers": buf[6], "records_staged": buf[7]}


AUTOTUNE_SHAPES = [(t, p, c) for t in (128, 256) for p in (1, 2, 4) for c in (0, 1)]


def bto_autotune(ctx: int, d_field_table, cycles: int, dt: float, stream=None) -> dict:
    best = (ctypes.c_int32 * 5)()
    ms = (ctypes.c_float * 12)()
    _check(load().bto_autotune(ctx, _addr(d_field_table), int(cycles), float(dt), _stream(stream), best, ms),
           "bto_autotune")
    return {"best": {"threads_per_cta": best[0], "particles_per_thread": best[1], "ctas_per_sm": best[2],
                     "reg_cap": best[3], "grid": best[4]},
            "ms_per_cycle": {f"{t}x{p}{'c' if c else ''}": round(ms[k], 5)
                             for k, (t, p, c) in enumerate(AUTOTUNE_SHAPES)}}


def bto_copy_active(ctx: int, d_out, stream=None) -> list:
    nb = bto_num_blocks(ctx)
    live = (ctypes.c_int32 * nb)()
    _check(load().bto_copy_active(ctx, _addr(d_out), live, _stream(stream)), "bto_copy_active")
    return list(live)


def bto_last_error(ctx: int) -> int:
    return int(load().bto_last_error(ctx))


def bto_interval_noalloc(extent_cells, origin, spacing, seed_stride: int, interval_cycles: int,
                         d_field_table, dt: float, d_seeds, d_ends, d_valid, d_exit_cycle=None,
                         stream=None) -> None:
    """One whole interval of one block with no device allocation by the
    library (state in a static device array; see include/bto.h)."""
    _check(load().bto_interval_noalloc(_arr(ctypes.c_int32, extent_cells), _arr(ctypes.c_float, origin),
                                       _arr(ctypes.c_float, spacing), int(seed_stride), int(interval_cycles),
                                       _addr(d_field_table), float(dt), _addr(d_seeds), _addr(d_ends),
                                       _addr(d_valid), _addr(d_exit_cycle), _stream(stream)),
           "bto_interval_noalloc")


def bto_set_device_allocator(alloc=None, free=None) -> None:
    """Install Python callables as the library's device allocator:
    alloc(nbytes) -> device address (int) or 0, free(address) -> None.
    Both None restores cudaMalloc / cudaFree."""
    if alloc is None and free is None:
        _check(load().bto_set_device_allocator(ALLOC_FN(), FREE_FN(), None), "bto_set_device_allocator")
        return
    a = ALLOC_FN(lambda nbytes, user: int(alloc(int(nbytes))) or None)
    f = FREE_FN(lambda ptr, user: free(int(ptr)))
    _allocator_refs.append((a, f))
    _check(load().bto_set_device_allocator(a, f, None), "bto_set_device_allocator")


def bto_check_bounds_build() -> bool:
    return bool(load().bto_check_bounds_build())


def bto_bounds_failures(reset: bool = False) -> int:
    v = ctypes.c_uint64(0)
    _check(load().bto_bounds_failures(ctypes.byref(v), int(bool(reset))), "bto_bounds_failures")
    return int(v.value)


def bto_fill_lattice(lattice, d_ends, d_valid, d_out, d_status=None, stream=None) -> None:
    _check(load().bto_fill_lattice(_arr(ctypes.c_int32, lattice), _addr(d_ends), _addr(d_valid), _addr(d_out),
                                   _addr(d_status), _stream(stream)), "bto_fill_lattice")


def bto_fill_delaunay(lattice, d_ends, d_valid, d_out, d_status=None, stream=None) -> None:
    _check(load().bto_fill_delaunay(_arr(ctypes.c_int32, lattice), _addr(d_ends), _addr(d_valid), _addr(d_out),
                                    _addr(d_status), _stream(stream)), "bto_fill_delaunay")


def bto_stitch_pathlines(lattice, origin, spacing, intervals: int, d_ends_table, nq: int, d_start, d_path,
                         stream=None) -> None:
    _check(load().bto_stitch_pathlines(_arr(ctypes.c_int32, lattice), _arr(ctypes.c_float, origin),
                                       _arr(ctypes.c_float, spacing), int(intervals), _addr(d_ends_table), int(nq),
                                       _addr(d_start), _addr(d_path), _stream(stream)), "bto_stitch_pathlines")


def bto_stitch_pathlines_ex(lattice, origin, spacing, intervals: int, d_ends_table, nq: int, d_start, d_path,
                            scheme: int, stream=None) -> None:
    _check(load().bto_stitch_pathlines_ex(_arr(ctypes.c_int32, lattice), _arr(ctypes.c_float, origin),
                                          _arr(ctypes.c_float, spacing), int(intervals), _addr(d_ends_table),
                                          int(nq), _addr(d_start), _addr(d_path), int(scheme), _stream(stream)),
           "bto_stitch_pathlines_ex")


def bto_tape_create(extent_cells, origin, spacing, num_particles: int, cycles: int,
                    checkpoint_every: int) -> int:
    out = ctypes.c_void_p()
    _check(load().bto_tape_create(_arr(ctypes.c_int32, extent_cells), _arr(ctypes.c_float, origin),
                                  _arr(ctypes.c_float, spacing), int(num_particles), int(cycles),
                                  int(checkpoint_every), ctypes.byref(out)), "bto_tape_create")
    return out.value


def bto_tape_num_particles(tape: int) -> int:
    return int(load().bto_tape_num_particles(tape))


def bto_tape_forward(tape: int, d_seeds, d_field_table, dt: float, d_ends, d_valid, d_exit_cycle=None,
                     stream=None) -> None:
    _check(load().bto_tape_forward(tape, _addr(d_seeds), _addr(d_field_table), float(dt), _addr(d_ends),
                                   _addr(d_valid), _addr(d_exit_cycle), _stream(stream)), "bto_tape_forward")


def bto_tape_backward(tape: int, d_grad_ends, d_grad_seeds, d_grad_field_table=None, stream=None) -> None:
    _check(load().bto_tape_backward(tape, _addr(d_grad_ends), _addr(d_grad_seeds), _addr(d_grad_field_table),
                                    _stream(stream)), "bto_tape_backward")


def bto_tape_jacobian(tape: int, d_jac, stream=None) -> None:
    _check(load().bto_tape_jacobian(tape, _addr(d_jac), _stream(stream)), "bto_tape_jacobian")


def bto_tape_ftle(tape: int, d_jac, d_ftle, stream=None) -> None:
    _check(load().bto_tape_ftle(tape, _addr(d_jac), _addr(d_ftle), _stream(stream)), "bto_tape_ftle")


def bto_tape_destroy(tape: int) -> None:
    if tape:
        load().bto_tape_destroy(tape)


def bto_status_string(status: int) -> str:
    return status_string(status)


def bto_destroy(ctx: int) -> None:
    if ctx:
        load().bto_destroy(ctx)


class Context:
    """Owning handle of a libbto context with torch-allocated outputs.

    ``Context(extent, origin, spacing, stride, interval)`` for one block, or
    ``Context.batch(extents, origins, spacings, strides, interval)``.
    """

    def __init__(self, extent, origin, spacing, stride, interval, _handle=None):
        self.handle = _handle if _handle is not None else bto_create(extent, origin, spacing, stride, interval)
        self.interval = int(interval)
        self.P = bto_num_seeds(self.handle)
        self.nb = bto_num_blocks(self.handle)

    @classmethod
    def batch(cls, extents, origins, spacings, strides, interval):
        h = bto_batch_create(extents, origins, spacings, strides, interval)
        return cls(None, None, None, None, interval, _handle=h)

    def offsets(self):
        return bto_batch_offsets(self.handle)

    def set_layout(self, layout):
        bto_set_field_layout(self.handle, layout)

    def set_ingest(self, enable):
        bto_set_ingest(self.handle, int(enable))

    def set_launch(self, threads, ppt, ctas_per_sm=0, reg_cap=0):
        bto_set_launch(self.handle, threads, ppt, ctas_per_sm, reg_cap)

    def launch(self):
        return bto_get_launch(self.handle)

    def set_tiling(self, tile_cells, threads=256):
        bto_set_tiling(self.handle, tile_cells, threads)

    def tiling(self):
        return bto_get_tiling(self.handle)

    def advect(self, field, dt, stream=None):
        bto_advect_cycle(self.handle, field, dt, stream)

    def advect_batch(self, field_ptrs, dt, stream=None):
        bto_batch_advect_cycle(self.handle, field_ptrs, dt, stream)

    def interval_graph(self, field_table, dt, stream=None):
        bto_launch_interval_graph(self.handle, field_table, dt, stream)

    def alloc_outputs(self, device=None):
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        return {"seeds": torch.empty((self.P, 3), dtype=torch.float32, device=dev),
                "ends": torch.empty((self.P, 3), dtype=torch.float32, device=dev),
                "valid": torch.empty((self.P,), dtype=torch.uint8, device=dev),
                "exit_cycle": torch.empty((self.P,), dtype=torch.int32, device=dev)}

    def end_interval(self, out=None, stream=None, exits=False):
        """Basis flows of the interval (dict of tensors); with exits=True also
        the clipped termination locations and times."""
        out = out if out is not None else self.alloc_outputs()
        if exits:
            import torch
            dev = out["seeds"].device
            out.setdefault("exit_pos", torch.empty((self.P, 3), dtype=torch.float32, device=dev))
            out.setdefault("exit_time", torch.empty((self.P,), dtype=torch.float32, device=dev))
            bto_end_interval_ex(self.handle, out["seeds"], out["ends"], out["valid"], out.get("exit_cycle"),
                                out["exit_pos"], out["exit_time"], stream)
        else:
            bto_end_interval(self.handle, out["seeds"], out["ends"], out["valid"],
                             out.get("exit_cycle"), stream)
        return out

    def autotune(self, field_table, cycles, dt, stream=None):
        return bto_autotune(self.handle, field_table, cycles, dt, stream)

    def copy_active(self, d_out, stream=None):
        return bto_copy_active(self.handle, d_out, stream)

    def check(self):
        _check(bto_last_error(self.handle), "bto_last_error")

    def close(self):
        if self.handle:
            bto_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
