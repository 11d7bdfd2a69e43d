"""FP64 CPU oracle for BTO Lagrangian flow-map extraction.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(the CUDA library and its binding) never does, and this package imports
nothing from it.

The arithmetic lives in ``bto_oracle.c`` (plain C, IEEE double, one particle
at a time, OpenMP over particles). This module only marshals numpy arrays
into it and strings the per-cycle calls into an interval, in the order the
paper states (Sec. 2.3 and 3.1): seed on a uniform lattice, advance every live
particle one RK4 step per cycle on that cycle's field, terminate on leaving
the block, and write seed / end / valid at the end of the interval.

Parity pins: every function here is pinned by tests that do not call the
oracle's own formulas (closed forms for affine and rotating fields, brute
force exit cycles, the Eq. (hx) invariant); see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bto_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libbto_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``bto_oracle.c`` with gcc into ``oracle/_build``.

    ``-ffp-contract=off`` keeps the double arithmetic free of fused
    multiply-adds, so x86 and Arm hosts give identical results.
    """
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.bto_oracle_num_seeds.argtypes = [i64p, ctypes.c_int64]
    lib.bto_oracle_num_seeds.restype = ctypes.c_int64
    lib.bto_oracle_seeds.argtypes = [i64p, dp, dp, ctypes.c_int64, ctypes.c_int64, i64p, dp]
    lib.bto_oracle_seeds.restype = None
    lib.bto_oracle_sample.argtypes = [fp, i64p, dp, dp, ctypes.c_int64, dp, dp]
    lib.bto_oracle_sample.restype = None
    lib.bto_oracle_cycle.argtypes = [fp, i64p, dp, dp, ctypes.c_double, ctypes.c_int32,
                                     ctypes.c_int64, dp, i32p, dp, dp, dp, ctypes.c_int32]
    lib.bto_oracle_cycle.restype = None
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.bto_oracle_adjoint_cycle.argtypes = [fp, i64p, dp, dp, ctypes.c_double, ctypes.c_int64, dp, u8p, dp,
                                             dp, ctypes.c_int32]
    lib.bto_oracle_adjoint_cycle.restype = None
    lib.bto_oracle_delaunay.argtypes = [i64p, u8p, ctypes.c_int64, i32p]
    lib.bto_oracle_delaunay.restype = ctypes.c_int64
    lib.bto_oracle_max_threads.argtypes = []
    lib.bto_oracle_max_threads.restype = ctypes.c_int32
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass(frozen=True)
class Grid:
    """One block of a uniform grid (reading R5): ``n`` cells per axis,
    ``n + 1`` nodes per axis at ``origin + i * h``.

    ``origin`` and ``h`` hold the float32 values the GPU receives, widened to
    double, so both sides start from the same numbers.
    """
    n: tuple
    origin: tuple
    h: tuple

    @staticmethod
    def make(n, origin, h) -> "Grid":
        o32 = np.asarray(origin, dtype=np.float32).astype(np.float64)
        h32 = np.asarray(h, dtype=np.float32).astype(np.float64)
        return Grid(tuple(int(v) for v in n), tuple(float(v) for v in o32),
                    tuple(float(v) for v in h32))

    def _arrays(self):
        return (np.ascontiguousarray(self.n, dtype=np.int64),
                np.ascontiguousarray(self.origin, dtype=np.float64),
                np.ascontiguousarray(self.h, dtype=np.float64))

    @property
    def node_shape(self):
        """numpy shape of a field for this block: (nz+1, ny+1, nx+1, 3)."""
        return (self.n[2] + 1, self.n[1] + 1, self.n[0] + 1, 3)


def max_threads() -> int:
    return int(_load().bto_oracle_max_threads())


def num_seeds(grid: Grid, stride: int) -> int:
    n, _, _ = grid._arrays()
    return int(_load().bto_oracle_num_seeds(_ptr(n, ctypes.c_int64), int(stride)))


def seeds(grid: Grid, stride: int, ids=None) -> np.ndarray:
    """Seed positions (physical), canonical order, shape (m, 3) float64."""
    lib = _load()
    n, o, h = grid._arrays()
    if ids is None:
        m = num_seeds(grid, stride)
        idp = None
    else:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        m = ids.shape[0]
        idp = _ptr(ids, ctypes.c_int64)
    out = np.empty((m, 3), dtype=np.float64)
    lib.bto_oracle_seeds(_ptr(n, ctypes.c_int64), _ptr(o, ctypes.c_double),
                         _ptr(h, ctypes.c_double), int(stride), m, idp,
                         _ptr(out, ctypes.c_double))
    return out


def _check_field(grid: Grid, field: np.ndarray) -> np.ndarray:
    field = np.ascontiguousarray(field, dtype=np.float32)
    want = int(np.prod(grid.node_shape))
    if field.size != want:
        raise ValueError(f"field has {field.size} values, block needs {want}")
    return field


def sample(grid: Grid, field: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Trilinear velocity at physical points q (m, 3) -> (m, 3) float64."""
    lib = _load()
    field = _check_field(grid, field)
    n, o, h = grid._arrays()
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
    v = np.empty_like(q)
    lib.bto_oracle_sample(_ptr(field, ctypes.c_float), _ptr(n, ctypes.c_int64),
                          _ptr(o, ctypes.c_double), _ptr(h, ctypes.c_double),
                          q.shape[0], _ptr(q, ctypes.c_double), _ptr(v, ctypes.c_double))
    return v


class State:
    """Particle state of one interval: positions, exit cycle, min margin."""

    def __init__(self, x0: np.ndarray):
        self.x = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 3).copy()
        self.seeds = self.x.copy()
        m = self.x.shape[0]
        self.exit_cycle = np.full(m, -1, dtype=np.int32)
        self.min_margin = np.full(m, np.inf, dtype=np.float64)
        self.exit_pos = np.full((m, 3), np.nan, dtype=np.float64)
        self.exit_time = np.full(m, np.nan, dtype=np.float64)

    @property
    def valid(self) -> np.ndarray:
        return (self.exit_cycle < 0).astype(np.uint8)


def cycle(grid: Grid, field: np.ndarray, dt: float, c: int, state: State,
          nthreads: int = 0) -> None:
    """Advance every live particle of ``state`` by one RK4 step (in place)."""
    lib = _load()
    field = _check_field(grid, field)
    n, o, h = grid._arrays()
    lib.bto_oracle_cycle(_ptr(field, ctypes.c_float), _ptr(n, ctypes.c_int64),
                         _ptr(o, ctypes.c_double), _ptr(h, ctypes.c_double),
                         float(dt), int(c), state.x.shape[0],
                         _ptr(state.x, ctypes.c_double),
                         _ptr(state.exit_cycle, ctypes.c_int32),
                         _ptr(state.min_margin, ctypes.c_double),
                         _ptr(state.exit_pos, ctypes.c_double), _ptr(state.exit_time, ctypes.c_double),
                         int(nthreads))


def run_interval(grid: Grid, stride: int, cycles: int, dt: float, field_of_cycle,
                 ids=None, c0: int = 0, nthreads: int = 0) -> State:
    """One interval (Sec. 2.3 / 3.1): seed, then ``cycles`` RK4 cycles.

    ``field_of_cycle(c)`` returns the float32 field of cycle c (absolute cycle
    index, starting at ``c0``); exit cycles are recorded relative to the
    interval (0 .. cycles-1). ``ids`` restricts the run to those canonical
    seeds (each particle is independent, so a subset gives the same numbers).
    """
    st = State(seeds(grid, stride, ids))
    for c in range(cycles):
        cycle(grid, field_of_cycle(c0 + c), dt, c, st, nthreads)
    return st


# ---------------------------------------------------------------------------
# Discrete adjoint (gradients of a loss on end positions)
# ---------------------------------------------------------------------------
def adjoint_cycle(grid: Grid, field: np.ndarray, dt: float, x: np.ndarray, alive: np.ndarray,
                  lam: np.ndarray, grad_field=None, nthreads: int = 0) -> None:
    """Reverse of one cycle: lam (m, 3) holds dL/dx after the cycle on entry
    and dL/dx before it on return, for particles whose step was taken
    (alive = 1). grad_field, if given, is a float64 array shaped like the
    field and is accumulated."""
    lib = _load()
    field = _check_field(grid, field)
    n, o, h = grid._arrays()
    x = np.ascontiguousarray(x, dtype=np.float64)
    alive = np.ascontiguousarray(alive, dtype=np.uint8)
    assert lam.dtype == np.float64 and lam.flags.c_contiguous
    gp = None
    if grad_field is not None:
        assert grad_field.dtype == np.float64 and grad_field.flags.c_contiguous
        assert grad_field.size == field.size
        gp = _ptr(grad_field, ctypes.c_double)
    lib.bto_oracle_adjoint_cycle(_ptr(field, ctypes.c_float), _ptr(n, ctypes.c_int64),
                                 _ptr(o, ctypes.c_double), _ptr(h, ctypes.c_double), float(dt),
                                 x.shape[0], _ptr(x, ctypes.c_double), _ptr(alive, ctypes.c_uint8),
                                 _ptr(lam, ctypes.c_double), gp, int(nthreads))


def forward_with_history(grid: Grid, field_of_cycle, dt: float, x0: np.ndarray, cycles: int):
    """Forward from arbitrary start positions, keeping every cycle's
    positions: returns (state, xs) with xs[c] the positions at the start of
    cycle c (xs[cycles] = end positions)."""
    st = State(x0)
    xs = [st.x.copy()]
    for c in range(cycles):
        cycle(grid, field_of_cycle(c), dt, c, st)
        xs.append(st.x.copy())
    return st, xs


def vjp(grid: Grid, field_of_cycle, dt: float, x0: np.ndarray, cycles: int, grad_end: np.ndarray,
        want_field_grads: bool = False):
    """Gradient of <grad_end, x_end(x0, F)> with respect to x0 (and, if asked,
    to every cycle's node velocities), by the discrete adjoint. A terminated
    particle's end is its last in-block position, reached by the steps
    before its exit cycle."""
    st, xs = forward_with_history(grid, field_of_cycle, dt, x0, cycles)
    lam = np.ascontiguousarray(grad_end, dtype=np.float64).reshape(-1, 3).copy()
    gF = [None] * cycles
    for c in reversed(range(cycles)):
        alive = ((st.exit_cycle < 0) | (st.exit_cycle > c)).astype(np.uint8)
        g = np.zeros(grid.node_shape, dtype=np.float64) if want_field_grads else None
        adjoint_cycle(grid, field_of_cycle(c), dt, xs[c], alive, lam, g)
        gF[c] = g
    return st, lam, gF


# ---------------------------------------------------------------------------
# Post hoc reconstruction of missing basis flows (Sec. 3.2; Eq. 2)
# ---------------------------------------------------------------------------
def fill_lattice(S, ends: np.ndarray, valid: np.ndarray):
    """Lattice stand-in for the paper's neighbourhood reconstruction: each
    missing entry J takes, along the axis whose nearest valid neighbours on
    both sides are closest (ties x, y, z), the linear interpolant of Eq. (1)
    between them at J. Returns (filled ends, status: 1 valid, 2 filled,
    0 missing). Plain loops, test sizes only."""
    Sx, Sy, Sz = (int(v) for v in S)
    E = np.asarray(ends, dtype=np.float64).reshape(Sz, Sy, Sx, 3)
    V = np.asarray(valid).reshape(Sz, Sy, Sx).astype(bool)
    out = np.full_like(E, np.nan)
    status = np.zeros((Sz, Sy, Sx), dtype=np.uint8)
    out[V] = E[V]
    status[V] = 1
    dims = (Sx, Sy, Sz)
    for jz, jy, jx in zip(*np.nonzero(~V)):
        j = [jx, jy, jz]
        best = None
        for ax in range(3):
            def at(off):
                jj = list(j)
                jj[ax] += off
                return jj
            a = 1
            while j[ax] - a >= 0 and not V[tuple(reversed(at(-a)))]:
                a += 1
            if j[ax] - a < 0:
                continue
            b = 1
            while j[ax] + b < dims[ax] and not V[tuple(reversed(at(b)))]:
                b += 1
            if j[ax] + b >= dims[ax]:
                continue
            if best is None or a + b < best[1] + best[2]:
                best = (ax, a, b, at(-a), at(b))
        if best is None:
            continue
        ax, a, b, jl, jr = best
        x0, x1, x = -a, b, 0.0
        fl, fr = E[tuple(reversed(jl))], E[tuple(reversed(jr))]
        # Eq. (1): L(x) = (x - x0)/(x1 - x0) f(x1) + (x1 - x)/(x1 - x0) f(x0)
        out[jz, jy, jx] = (x - x0) / (x1 - x0) * fr + (x1 - x) / (x1 - x0) * fl
        status[jz, jy, jx] = 2
    return out.reshape(-1, 3), status.reshape(-1)


def stitch(S, origin, spacing, ends_list, start, scheme: str = "trilinear"):
    """Pathline stitching (Sec. 3.2) on a seed lattice: in interval k the next
    position interpolates the end positions of the basis flows around the
    particle's lattice cell. ``scheme``:

    * ``"trilinear"``: Eq. 1 per axis over the cell's 8 corners;
    * ``"barycentric"``: the paper's barycentric coordinates in a Delaunay
      tetrahedron of the start points. The 8 corners of a lattice cell lie on
      one sphere, so every face-conforming split of the cells is a Delaunay
      triangulation; this is the Kuhn split (6 tetrahedra sharing the main
      diagonal). With the fractional coordinates sorted t_a >= t_b >= t_c
      (ties kept in axis order), the particle's tetrahedron has vertices
      0, e_a, e_a + e_b, (1, 1, 1) and its barycentric weights are
      1 - t_a, t_a - t_b, t_b - t_c, t_c.

    Outside the lattice, or when an entry the interpolant uses is missing
    (NaN), the particle stops (NaN). Returns (intervals + 1, nq, 3)."""
    if scheme not in ("trilinear", "barycentric"):
        raise ValueError(scheme)
    S = [int(v) for v in S]
    o = np.asarray(origin, dtype=np.float32).astype(np.float64)
    sp = np.asarray(spacing, dtype=np.float32).astype(np.float64)
    x = np.asarray(start, dtype=np.float64).reshape(-1, 3).copy()
    path = [x.copy()]
    for E in ends_list:
        E = np.asarray(E, dtype=np.float64).reshape(S[2], S[1], S[0], 3)
        nxt = np.full_like(x, np.nan)
        for i in range(x.shape[0]):
            u = (x[i] - o) / sp
            if not np.all(np.isfinite(u)) or np.any(u < 0) or np.any(u > np.array(S) - 1):
                continue
            cell = [min(int(np.floor(u[a])), max(S[a] - 2, 0)) for a in range(3)]
            t = [u[a] - cell[a] for a in range(3)]
            acc = np.zeros(3)
            if scheme == "trilinear":
                for c in range(2):
                    for b in range(2):
                        for a in range(2):
                            w = (t[0] if a else 1 - t[0]) * (t[1] if b else 1 - t[1]) * (t[2] if c else 1 - t[2])
                            j = [min(cell[0] + a, S[0] - 1), min(cell[1] + b, S[1] - 1), min(cell[2] + c, S[2] - 1)]
                            acc += w * E[j[2], j[1], j[0]]
            else:
                axes = sorted(range(3), key=lambda a: -t[a])        # stable: ties keep x, y, z
                ts = [t[a] for a in axes]
                weights = [1 - ts[0], ts[0] - ts[1], ts[1] - ts[2], ts[2]]
                j = list(cell)
                for m in range(4):
                    if m > 0:
                        j[axes[m - 1]] = min(j[axes[m - 1]] + 1, S[axes[m - 1]] - 1)
                    acc += weights[m] * E[j[2], j[1], j[0]]
            nxt[i] = acc
        x = nxt
        path.append(x.copy())
    return np.stack(path)


# ---------------------------------------------------------------------------
# Accuracy metrics (Sec. 4.3): b = BTO positions, m = reference positions.
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Post hoc reconstruction over a Delaunay triangulation (Sec. 3.2)
# ---------------------------------------------------------------------------
def delaunay(S, valid: np.ndarray) -> np.ndarray:
    """Delaunay triangulation (Bowyer-Watson, exact predicates, ties broken
    by the lifted-weight perturbation described in bto_oracle.c) of the
    valid points of the seed lattice S (x fastest). Returns (T, 4) canonical
    lattice ids, each tetrahedron positively oriented."""
    lib = _load()
    S64 = np.asarray(S, dtype=np.int64)
    v = np.ascontiguousarray(np.asarray(valid).reshape(-1), dtype=np.uint8)
    cap = 16 * int(v.sum()) + 64
    out = np.empty((cap, 4), dtype=np.int32)
    nt = lib.bto_oracle_delaunay(_ptr(S64, ctypes.c_int64), _ptr(v, ctypes.c_uint8), cap,
                                 _ptr(out, ctypes.c_int32))
    if nt < 0:
        raise RuntimeError(f"bto_oracle_delaunay failed ({nt})")
    return out[:nt].copy()


def lattice_coords(S, ids: np.ndarray) -> np.ndarray:
    S = [int(v) for v in S]
    ids = np.asarray(ids, dtype=np.int64)
    return np.stack([ids % S[0], (ids // S[0]) % S[1], ids // (S[0] * S[1])], axis=-1).astype(np.float64)


def delaunay_interpolate(S, tets: np.ndarray, ends: np.ndarray, q: np.ndarray, tol: float = 1e-9):
    """Barycentric interpolation of the end positions over the tetrahedron
    of ``tets`` that holds each query point q (lattice coordinates, (m, 3)).
    Returns (values (m, 3), found (m,) bool); a point held by no tetrahedron
    (outside the hull of the valid points) gets NaN."""
    E = np.asarray(ends, dtype=np.float64).reshape(-1, 3)
    V = lattice_coords(S, tets)                       # (T, 4, 3)
    A = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1))   # columns v1 - v0, v2 - v0, v3 - v0
    Ainv = np.linalg.inv(A)
    q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
    vals = np.full((q.shape[0], 3), np.nan)
    found = np.zeros(q.shape[0], dtype=bool)
    for i in range(q.shape[0]):
        l123 = np.einsum("tij,tj->ti", Ainv, q[i] - V[:, 0, :])
        lam = np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)
        hit = np.flatnonzero(np.all(lam >= -tol, axis=1))
        if hit.size == 0:
            continue
        t = hit[0]
        vals[i] = lam[t] @ E[tets[t]]
        found[i] = True
    return vals, found


def fill_delaunay(S, ends: np.ndarray, valid: np.ndarray):
    """Reconstruction of the missing basis flows of a seed lattice over the
    Delaunay triangulation of the valid ones (Sec. 3.2): each missing entry
    takes the barycentric interpolant at its own lattice point over the
    tetrahedron that holds it. An entry on the lattice's boundary faces lies
    on a face of that tetrahedron (its weight on the vertex off the face is
    zero); an entry outside the hull of the valid points stays missing. A
    lattice one point thick along some axis has no tetrahedra, and its
    missing entries stay missing.
    Returns (filled ends, status: 1 valid, 2 filled, 0 missing)."""
    v = np.asarray(valid).reshape(-1).astype(bool)
    E = np.asarray(ends, dtype=np.float64).reshape(-1, 3).copy()
    status = np.where(v, 1, 0).astype(np.uint8)
    miss = np.flatnonzero(~v)
    E[miss] = np.nan
    if miss.size and v.sum() >= 4 and min(int(a) for a in S) > 1:
        tets = delaunay(S, v)
        vals, found = delaunay_interpolate(S, tets, E, lattice_coords(S, miss))
        E[miss] = vals
        status[miss[found]] = 2
    return E, status


def total_average_l2(b: np.ndarray, m: np.ndarray) -> float:
    """Total average L2 norm, (1/p) sum_i ||b_i - m_i|| (Sec. 4.3). The sum
    runs over the p particles (the printed bounds i = 0..p are read as the p
    particles, matching the 1/p factor)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    if b.shape[0] == 0:
        return 0.0
    return float(np.mean(np.sqrt(np.sum((b - m) ** 2, axis=1))))


def accuracy_percent(l2: float, cell_side: float) -> float:
    """Accuracy% = (C - L) / C * 100 (Sec. 4.3)."""
    return (cell_side - l2) / cell_side * 100.0


def max_l2(b: np.ndarray, m: np.ndarray) -> float:
    """Largest single-particle L2 error of one interval (Sec. 4.3)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    if b.shape[0] == 0:
        return 0.0
    return float(np.max(np.sqrt(np.sum((b - m) ** 2, axis=1))))


def greatest_and_average_max_l2(per_interval_max) -> tuple:
    """Greatest max L2 over intervals, and the mean of the per-interval
    maxima (Sec. 4.3)."""
    a = np.asarray(per_interval_max, dtype=np.float64)
    return float(a.max()), float(a.mean())
