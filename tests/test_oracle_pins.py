"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms for affine fields (trilinear interpolation, Eq. (1) per
axis, is exact on them), the RK4 stability polynomial, RK4's fourth-order
convergence, brute-force exit cycles in exact rational arithmetic, and the
Eq. (hx) statement that a seed farther from the boundary than the largest
per-interval displacement cannot reach it. Each is chosen so that a dropped
term, a swapped index or a sign error in the oracle fails at least one.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import inputs


# ----------------------------------------------------------------------------
# Trilinear interpolation (Eq. 1 per axis and component)
# ----------------------------------------------------------------------------
def test_sample_reproduces_node_values():
    rng = np.random.default_rng(1)
    n = (5, 4, 3)
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), (0.25, 0.5, 0.125))
    field = rng.standard_normal(g.node_shape).astype(np.float32)
    # every node, including the upper faces (t = 1 in the last cell)
    I, J, K = np.meshgrid(np.arange(n[0] + 1), np.arange(n[1] + 1), np.arange(n[2] + 1), indexing="ij")
    q = np.stack([I.ravel() * 0.25, J.ravel() * 0.5, K.ravel() * 0.125], axis=1)
    v = oracle.sample(g, field, q)
    want = field[K.ravel(), J.ravel(), I.ravel()].astype(np.float64)
    assert np.array_equal(v, want)


def test_sample_affine_field_is_exact():
    # A is not symmetric, so a transposed axis or a swapped weight fails.
    A = np.array([[0.5, -1.25, 0.375], [2.0, 0.25, -0.75], [-0.5, 1.5, 1.0]])
    b = np.array([0.25, -0.5, 1.75])
    n = (6, 5, 7)
    h = (0.125, 0.25, 0.0625)
    origin = (-0.5, 0.25, 1.0)
    g = oracle.Grid.make(n, origin, h)
    field = inputs.affine_field(n, origin, h, A, b)   # dyadic: exact in float32
    rng = np.random.default_rng(2)
    lo = np.array(origin)
    hi = lo + np.array(n) * np.array(h)
    q = lo + rng.random((2000, 3)) * (hi - lo)
    v = oracle.sample(g, field, q)
    assert np.max(np.abs(v - (q @ A.T + b))) < 1e-12


def test_sample_is_not_nearest_or_constant():
    # A quadratic field is NOT reproduced: the interpolant of x^2 on [0, 1]
    # is x, so the error at the midpoint is exactly 1/4 (Eq. 1 in 1D).
    n = (1, 1, 1)
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    field = np.zeros(g.node_shape, dtype=np.float32)
    field[:, :, 1, 0] = 1.0                      # u_x = x^2 at x in {0, 1}
    v = oracle.sample(g, field, np.array([[0.5, 0.3, 0.7]]))
    assert v[0, 0] == pytest.approx(0.5, abs=1e-15)   # interpolant x, not x^2
    assert v[0, 1] == 0.0 and v[0, 2] == 0.0


# ----------------------------------------------------------------------------
# RK4 step
# ----------------------------------------------------------------------------
def test_uniform_translation_is_exact():
    n = (16, 16, 16)
    h = (1.0 / 16,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    c = np.array([0.0078125, -0.00390625, 0.001953125])
    field = inputs.uniform_field(n, c)
    st = oracle.State(oracle.seeds(g, 4)[:, :] * 0.5 + 0.25)
    L, dt = 20, 0.5
    for k in range(L):
        oracle.cycle(g, field, dt, k, st)
    assert np.all(st.exit_cycle == -1)
    assert np.max(np.abs(st.x - (st.seeds + L * dt * c))) < 1e-14


def _phi(Z):
    I = np.eye(3)
    return I + Z / 2 + Z @ Z / 6 + Z @ Z @ Z / 24


def test_linear_field_matches_rk4_closed_form():
    # u = A x + b on a grid: trilinear is exact, so gridded RK4 must equal the
    # closed-form RK4 map x -> x + dt phi(dt A) (A x + b) for any A.
    A = np.array([[-0.75, 1.5, 0.25], [-1.25, 0.5, -0.5], [0.375, -0.25, -1.0]])
    b = np.array([0.5, -0.25, 0.125])
    n = (64, 64, 64)
    h = (0.25, 0.25, 0.25)
    origin = (-8.0, -8.0, -8.0)
    g = oracle.Grid.make(n, origin, h)
    field = inputs.affine_field(n, origin, h, A, b)
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-0.5, 0.5, size=(300, 3))
    st = oracle.State(x0)
    dt = 0.0625
    M = _phi(dt * A)
    x = x0.copy()
    for k in range(12):
        oracle.cycle(g, field, dt, k, st)
        x = x + dt * (x @ A.T + b) @ M.T
    assert np.all(st.exit_cycle == -1)
    assert np.max(np.abs(st.x - x)) < 1e-12


def test_rotation_amplification_factor():
    # Solid-body rotation: one RK4 step scales the radius by |P(i w dt)| with
    # P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, i.e.
    # sqrt(1 - (w dt)^6/72 + (w dt)^8/576).
    w, dt, L = 2.0, 0.2, 25
    n = (32, 32, 32)
    h = (1.0 / 8,) * 3
    center = (2.0, 2.0, 2.0)
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    field = inputs.rotation_field(n, (0.0, 0.0, 0.0), h, w, center)
    x0 = np.array([[2.0 + r, 2.0, 2.0 + 0.25 * r] for r in (0.25, 0.5, 1.0, 1.5)])
    st = oracle.State(x0)
    for k in range(L):
        oracle.cycle(g, field, dt, k, st)
    z = w * dt
    amp = np.sqrt(1 - z ** 6 / 72 + z ** 8 / 576)
    r0 = np.hypot(x0[:, 0] - 2.0, x0[:, 1] - 2.0)
    r = np.hypot(st.x[:, 0] - 2.0, st.x[:, 1] - 2.0)
    assert np.max(np.abs(r / r0 - amp ** L)) < 1e-13
    assert np.array_equal(st.x[:, 2], x0[:, 2])  # no motion along the axis


def test_rotation_fourth_order_convergence():
    # Global error of RK4 at a fixed end time drops ~16x when dt halves.
    w, T = 1.0, 2.0
    n = (32, 32, 32)
    h = (1.0 / 8,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    field = inputs.rotation_field(n, (0.0, 0.0, 0.0), h, w, (2.0, 2.0, 2.0))
    x0 = np.array([[3.0, 2.0, 2.0]])
    exact = np.array([2.0 + np.cos(w * T), 2.0 + np.sin(w * T), 2.0])
    errs = []
    for steps in (10, 20, 40):
        st = oracle.State(x0)
        for k in range(steps):
            oracle.cycle(g, field, T / steps, k, st)
        errs.append(np.linalg.norm(st.x[0] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14.0 < r1 < 18.0 and 14.5 < r2 < 17.5


# ----------------------------------------------------------------------------
# Termination (Sec. 3.1, Sec. 3.3; closed box, stage points tested)
# ----------------------------------------------------------------------------
def _brute_exit(x0, step, lo, hi, L):
    """First cycle whose end point leaves [lo, hi]^3 (exact rationals)."""
    x = [Fraction(v) for v in x0]
    for c in range(L):
        nxt = [x[a] + step[a] for a in range(3)]
        if any(not (lo[a] <= nxt[a] <= hi[a]) for a in range(3)):
            return c, x
        x = nxt
    return -1, x


@pytest.mark.parametrize("vel", [(1.0, 0.0, 0.0), (0.0, -0.5, 0.0), (0.25, 0.5, -1.0)])
def test_straight_line_exit_cycle_brute_force(vel):
    # h = dt = 3/8: every position, stage point and dt/6 is exact in binary,
    # so particles land exactly on faces, which count as inside.
    n = (8, 8, 8)
    h = (0.375,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    field = inputs.uniform_field(n, vel)
    dt, L = 0.375, 12
    st = oracle.State(oracle.seeds(g, 1))
    for k in range(L):
        oracle.cycle(g, field, dt, k, st)
    step = [Fraction(v) * Fraction(dt) for v in vel]
    on_face = 0
    for p in range(st.x.shape[0]):
        want_c, want_x = _brute_exit(st.seeds[p], step, [0] * 3, [3] * 3, L)
        assert st.exit_cycle[p] == want_c
        assert np.array_equal(st.x[p], np.array([float(v) for v in want_x]))
        on_face += any(v in (0, 3) for v in want_x) and want_c != 0
    assert on_face > 0   # the closed-box case was exercised


def test_directional_flow_terminates_exactly_the_near_face_seeds():
    n = (32, 32, 32)
    h = (1.0 / 32,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    field = inputs.uniform_field(n, (1.0, 0.0, 0.0))
    L, dt = 50, 0.0099                 # reach 0.495; no seed ties with a face
    st = oracle.run_interval(g, 2, L, dt, lambda c: field)
    x0 = st.seeds[:, 0]
    leave = x0 + L * dt > 1.0
    assert np.array_equal(st.valid == 0, leave)
    assert np.array_equal(st.exit_cycle[leave], np.floor((1.0 - x0[leave]) / dt).astype(int))
    assert np.all(st.exit_cycle[~leave] == -1)


def _one_cycle_1d(x, x_e, K, dt, n_cells=8):
    """Particle at (x, 4, 4) in u = (-K (x - x_e), 0, 0) on an 8^3 unit-cell block."""
    n = (n_cells,) * 3
    A = np.diag([-K, 0.0, 0.0])
    b = np.array([K * x_e, 0.0, 0.0])
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    field = inputs.affine_field(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), A, b)
    st = oracle.State(np.array([[x, 4.0, 4.0]]))
    oracle.cycle(g, field, dt, 7, st)
    return st


def test_termination_on_stage_point_p2():
    # K dt = 3: p2 - x_e = (1 - 3/2) d; x = 5, x_e = 1 -> p2 = -1 (outside),
    # while the full step would land at x' = 1 + 1.375 * 4 = 6.5 (inside).
    st = _one_cycle_1d(5.0, 1.0, 30.0, 0.1)
    assert st.exit_cycle[0] == 7 and st.x[0, 0] == 5.0
    assert st.min_margin[0] == pytest.approx(1.0)


def test_termination_on_stage_point_p3():
    # p3 - x_e = (1 - 3/2 + 9/4) d = 1.75 d: x = 7, x_e = 5 -> p3 = 8.5 (outside);
    # p2 = 4 and x' = 7.75 are inside.
    st = _one_cycle_1d(7.0, 5.0, 30.0, 0.1)
    assert st.exit_cycle[0] == 7 and st.x[0, 0] == 7.0
    assert st.min_margin[0] == pytest.approx(0.5)


def test_termination_on_stage_point_p4():
    # p4 - x_e = (1 - 3 + 9/2 - 27/4) d = -4.25 d: x = 5, x_e = 4 -> p4 = -0.25;
    # p2 = 3.5, p3 = 5.75 and x' = 5.375 are inside.
    st = _one_cycle_1d(5.0, 4.0, 30.0, 0.1)
    assert st.exit_cycle[0] == 7 and st.x[0, 0] == 5.0
    assert st.min_margin[0] == pytest.approx(0.25)


def test_overshooting_step_that_stays_inside_is_kept():
    # Same unstable K dt = 3 step with every stage point inside:
    # x = 4.5, x_e = 4: p2 = 3.75, p3 = 4.875, p4 = 1.875, x' = 4.6875.
    st = _one_cycle_1d(4.5, 4.0, 30.0, 0.1)
    assert st.exit_cycle[0] == -1
    assert st.x[0, 0] == pytest.approx(4.0 + 1.375 * 0.5, abs=1e-12)


# ----------------------------------------------------------------------------
# Seeds (Sec. 2.3) and the Eq. (hx) invariant (Sec. 3.3)
# ----------------------------------------------------------------------------
def test_seed_lattice_and_canonical_order():
    g = oracle.Grid.make((7, 10, 5), (1.0, -2.0, 0.5), (0.5, 0.25, 1.0))
    s = 2
    S = (4, 5, 3)                       # ceil(n / s), upper faces excluded
    assert oracle.num_seeds(g, s) == 4 * 5 * 3
    x = oracle.seeds(g, s)
    p = 0
    for jz in range(S[2]):
        for jy in range(S[1]):
            for jx in range(S[0]):
                want = (1.0 + jx * s * 0.5, -2.0 + jy * s * 0.25, 0.5 + jz * s * 1.0)
                assert tuple(x[p]) == want
                p += 1
    ids = np.array([5, 0, 59, 13])
    assert np.array_equal(oracle.seeds(g, s, ids), x[ids])


def test_eq_hx_far_seeds_stay_valid_on_abc():
    n = (32, 32, 32)
    h = (1.0 / 32,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    L, dt = 20, 0.002
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * dt) for c in range(L)]
    st = oracle.run_interval(g, 2, L, dt, lambda c: fields[c])
    vmax = max(inputs.max_speed(f) for f in fields)
    reach = L * dt * vmax
    d_face = np.min(np.minimum(st.seeds, 1.0 - st.seeds), axis=1)
    far = d_face > reach
    assert far.sum() > 0
    assert np.all(st.valid[far] == 1)
    assert (st.valid == 0).sum() > 0   # some near-face seeds did leave


def test_thread_count_does_not_change_results():
    n = (16, 16, 16)
    h = (1.0 / 16,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * 0.02) for c in range(10)]
    a = oracle.run_interval(g, 1, 10, 0.02, lambda c: fields[c], nthreads=1)
    b = oracle.run_interval(g, 1, 10, 0.02, lambda c: fields[c], nthreads=4)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.exit_cycle, b.exit_cycle)


def test_subset_run_equals_full_run():
    n = (16, 16, 16)
    h = (1.0 / 16,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    fields = [inputs.abc_field(n, (0, 0, 0), h, c * 0.02) for c in range(10)]
    full = oracle.run_interval(g, 1, 10, 0.02, lambda c: fields[c])
    ids = np.array([3, 4000, 17, 999, 4095])
    sub = oracle.run_interval(g, 1, 10, 0.02, lambda c: fields[c], ids=ids)
    assert np.array_equal(sub.x, full.x[ids])
    assert np.array_equal(sub.exit_cycle, full.exit_cycle[ids])


# ----------------------------------------------------------------------------
# Accuracy metrics (Sec. 4.3)
# ----------------------------------------------------------------------------
def test_metrics_by_hand():
    b = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    m = np.zeros((3, 3))
    assert oracle.total_average_l2(b, m) == pytest.approx((5.0 + 0.0 + 3.0) / 3)
    assert oracle.max_l2(b, m) == 5.0
    assert oracle.accuracy_percent(0.25, 1.0) == pytest.approx(75.0)
    assert oracle.greatest_and_average_max_l2([1.0, 3.0, 2.0]) == (3.0, 2.0)


# ----------------------------------------------------------------------------
# Termination locations (the paper's future work, Sec. 6; chord clipping)
# ----------------------------------------------------------------------------
def test_exit_location_of_straight_flow_is_the_exact_crossing():
    # Uniform u = (1, 0, 0): the chord is the path, so the clipped point is
    # the exact face crossing and the exit time (in cycles) is (1 - x0)/dt.
    n = (32, 32, 32)
    h = (1.0 / 32,) * 3
    g = oracle.Grid.make(n, (0.0, 0.0, 0.0), h)
    field = inputs.uniform_field(n, (1.0, 0.0, 0.0))
    L, dt = 50, 0.0099
    st = oracle.run_interval(g, 2, L, dt, lambda c: field)
    t = st.exit_cycle >= 0
    assert t.sum() > 100
    x0 = st.seeds[t]
    assert np.max(np.abs(st.exit_pos[t, 0] - 1.0)) < 1e-12
    assert np.array_equal(st.exit_pos[t, 1:], x0[:, 1:])
    assert np.max(np.abs(st.exit_time[t] - (1.0 - x0[:, 0]) / dt)) < 1e-9
    assert np.all(np.isnan(st.exit_time[~t]))


def test_exit_location_for_each_stage_by_hand():
    # The K dt = 3 linear-field cases of the stage-point pins above:
    # p2 = -1 from x = 5 (t = 5/6, f = 1/2); p3 = 8.5 from x = 7 (t = 2/3,
    # f = 1/2); p4 = -0.25 from x = 5 (t = 5/5.25, f = 1).
    for x, xe, face, t, f in ((5.0, 1.0, 0.0, 5 / 6, 0.5), (7.0, 5.0, 8.0, 2 / 3, 0.5),
                              (5.0, 4.0, 0.0, 5 / 5.25, 1.0)):
        st = _one_cycle_1d(x, xe, 30.0, 0.1)
        assert st.exit_pos[0, 0] == pytest.approx(face, abs=1e-12)
        assert tuple(st.exit_pos[0, 1:]) == (4.0, 4.0)
        assert st.exit_time[0] == pytest.approx(7 + t * f, abs=1e-12)


# ----------------------------------------------------------------------------
# BTO against the global flow map, and Eq. (hx) across block faces
# ----------------------------------------------------------------------------
def _decomposed_abc(L, dt):
    G, n, s = 32, 16, 2
    h = (1.0 / G,) * 3
    glob = [inputs.abc_field((G, G, G), (0, 0, 0), h, c * dt) for c in range(L)]
    gg = oracle.Grid.make((G, G, G), (0.0, 0.0, 0.0), h)
    gst = oracle.run_interval(gg, s, L, dt, lambda c: glob[c])
    blocks = []
    for bz in range(2):
        for by in range(2):
            for bx in range(2):
                o = (bx * n * h[0], by * n * h[1], bz * n * h[2])
                g = oracle.Grid.make((n, n, n), o, h)
                sl = [np.ascontiguousarray(f[bz * n:bz * n + n + 1, by * n:by * n + n + 1, bx * n:bx * n + n + 1])
                      for f in glob]
                blocks.append(((bx, by, bz), oracle.run_interval(g, s, L, dt, lambda c, sl=sl: sl[c])))
    vmax = max(inputs.max_speed(f) for f in glob)
    return G, n, s, h, gst, blocks, L * dt * vmax


def test_bto_valid_ends_equal_global_flow_map():
    # Sec. 3.1 / Sec. 5: a particle that never leaves its block sees the
    # same cells and node values as in the undecomposed domain (blocks share
    # their face nodes), so its basis flow is the global flow map's, up to
    # rounding; and it cannot have left the domain either.
    G, n, s, h, gst, blocks, reach = _decomposed_abc(20, 0.002)
    S, GS = n // s, G // s
    checked = 0
    for (bx, by, bz), st in blocks:
        j = np.arange(S ** 3)
        jx, jy, jz = j % S, (j // S) % S, j // (S * S)
        gid = (jx + bx * S) + GS * ((jy + by * S) + GS * (jz + bz * S))
        assert np.allclose(st.seeds, gst.seeds[gid], atol=1e-15)
        v = st.valid == 1
        assert np.all(gst.valid[gid][v] == 1)
        assert np.max(np.abs(st.x[v] - gst.x[gid][v])) < 1e-12
        checked += int(v.sum())
    assert checked > 0.5 * GS ** 3
    # BTO terminates more than the global map: particles that cross inner faces
    assert sum(int((st.valid == 0).sum()) for _, st in blocks) > int((gst.valid == 0).sum())


def test_eq_hx_gap_bound_across_block_faces():
    # Eq. (hx): missing basis flows lie within the largest displacement of a
    # face, so along the normal of a face two valid flows around a run of
    # missing ones are at most 2 h_x + 2 reach apart. Lines along one axis
    # whose other coordinates are farther than the reach from every face
    # normal to them can only lose flows near faces normal to the line.
    G, n, s, h, gst, blocks, reach = _decomposed_abc(20, 0.002)
    S, GS = n // s, G // s
    hx = s * h[0]
    lat = np.zeros((GS, GS, GS), dtype=np.uint8)        # (z, y, x)
    for (bx, by, bz), st in blocks:
        lat[bz * S:(bz + 1) * S, by * S:(by + 1) * S, bx * S:(bx + 1) * S] = st.valid.reshape(S, S, S)
    j = np.arange(GS) % S
    far = np.minimum(j, S - j) * hx > reach + 1e-12
    cross = far[:, None] & far[None, :]
    bound = 2.0 + 2.0 * reach / hx
    widest = 0
    for axis in range(3):
        lines = np.moveaxis(lat, axis, -1)[cross]
        assert lines.shape[0] > 0
        for line in lines[np.any(lines == 0, axis=1)]:
            ok = np.flatnonzero(line == 1)
            if ok.size >= 2:
                widest = max(widest, int(np.diff(ok).max()))
    assert 1 < widest <= bound, (widest, bound)
