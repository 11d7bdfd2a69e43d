"""Pins of the oracle's lattice reconstruction (Sec. 3.2, Eq. 1 and Eq. 2)."""
import numpy as np

import oracle


def test_affine_flow_map_is_reconstructed_exactly():
    # Linear interpolation reproduces an affine map, so every filled entry
    # must equal the map itself.
    rng = np.random.default_rng(3)
    S = (9, 7, 6)
    jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
    x0 = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3).astype(np.float64)
    M = np.array([[1.1, 0.2, -0.3], [0.05, 0.9, 0.4], [-0.2, 0.1, 1.3]])
    ends = x0 @ M.T + np.array([0.5, -1.0, 2.0])
    valid = (rng.random(x0.shape[0]) > 0.3).astype(np.uint8)
    out, status = oracle.fill_lattice(S, ends, valid)
    filled = status == 2
    assert filled.sum() > 50 and np.all(status[valid == 1] == 1)
    assert np.max(np.abs(out[filled] - ends[filled])) < 1e-12


def test_double_interpolation_identity():
    # Eq. (2): interpolating inside [x0, x1] through the value filled at x1
    # equals interpolating between x0 and x2 directly.
    rng = np.random.default_rng(4)
    f = rng.standard_normal((5, 3))
    ends = f.copy()
    valid = np.array([1, 0, 1, 1, 1], dtype=np.uint8)   # x0 = 0, x1 = 1 (missing), x2 = 2
    out, status = oracle.fill_lattice((5, 1, 1), ends, valid)
    assert status[1] == 2
    for x in np.linspace(0.0, 1.0, 7):
        through_fill = (x - 0) / (1 - 0) * out[1] + (1 - x) / (1 - 0) * out[0]
        direct = (x - 0) / (2 - 0) * f[2] + (2 - x) / (2 - 0) * f[0]
        assert np.allclose(through_fill, direct, atol=1e-14)


def test_axis_with_the_closest_neighbours_is_used():
    S = (7, 3, 1)
    ends = np.arange(21 * 3, dtype=np.float64).reshape(21, 3)
    valid = np.ones(21, dtype=np.uint8)
    c = 3 + 7 * 1                      # centre (3, 1)
    valid[[c, c - 1, c + 1, c - 2]] = 0  # x gap: a = 3, b = 2; y gap: a = b = 1
    out, status = oracle.fill_lattice(S, ends, valid)
    assert status[c] == 2
    assert np.allclose(out[c], 0.5 * (ends[c - 7] + ends[c + 7]))
    # an entry with no valid neighbour pair on any axis stays missing
    out2, status2 = oracle.fill_lattice((3, 1, 1), ends[:3], np.array([0, 1, 1], dtype=np.uint8))
    assert status2[0] == 0 and np.all(np.isnan(out2[0]))


def _affine_lattice(S, o, sp, M, b):
    jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
    X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * np.asarray(sp) + np.asarray(o)
    return X @ M.T + b


def test_stitching_composes_affine_flow_maps_exactly():
    # Trilinear interpolation reproduces affine maps, so stitching through the
    # basis flows of affine flow maps applies their composition exactly.
    S, o, sp = (12, 10, 9), (0.0, 0.0, 0.0), (0.5, 0.5, 0.5)   # dyadic: exact lattice
    M1 = np.array([[1.0, 0.05, 0.0], [-0.05, 1.0, 0.02], [0.0, 0.01, 0.98]])
    M2 = np.array([[0.97, 0.0, 0.03], [0.02, 1.01, 0.0], [0.0, -0.02, 1.0]])
    b1, b2 = np.array([0.1, -0.05, 0.2]), np.array([-0.1, 0.1, 0.05])
    E1, E2 = _affine_lattice(S, o, sp, M1, b1), _affine_lattice(S, o, sp, M2, b2)
    rng = np.random.default_rng(9)
    start = rng.uniform(1.5, 3.5, size=(50, 3))
    path = oracle.stitch(S, o, sp, [E1, E2], start)
    want1 = start @ M1.T + b1
    want2 = want1 @ M2.T + b2
    assert np.max(np.abs(path[1] - want1)) < 1e-12
    assert np.max(np.abs(path[2] - want2)) < 1e-12


def test_stitching_at_lattice_points_and_outside():
    S, o, sp = (4, 4, 4), (1.0, 1.0, 1.0), (0.25, 0.25, 0.25)
    rng = np.random.default_rng(10)
    E = rng.standard_normal((64, 3)) + 2.0
    start = np.array([[1.25, 1.5, 1.0], [0.5, 1.5, 1.5], [1.75, 1.75, 1.75]])
    path = oracle.stitch(S, o, sp, [E], start)
    assert np.allclose(path[1, 0], E[1 + 4 * (2 + 4 * 0)])
    assert np.all(np.isnan(path[1, 1]))                      # outside the lattice
    assert np.allclose(path[1, 2], E[3 + 4 * (3 + 4 * 3)])   # upper corner


def _quadratic_flow_map(X, T):
    # u = (x^2, 0, 0): x(T) = x0 / (1 - x0 T), y and z fixed
    out = X.copy()
    out[:, 0] = X[:, 0] / (1.0 - X[:, 0] * T)
    return out


def test_stitching_error_is_second_order_in_the_seed_spacing():
    # Sec. 3.3 (Eq. global): the post hoc interpolation of a flow map from
    # basis flows spaced h_x apart errs by O(h_x^2), bounded by the Hessian of
    # the flow map (d^2/8 h_x^2 max|H| for one interval). The flow map of
    # u = (x^2, 0, 0) over T is known in closed form and is not affine in x,
    # so its basis flows are taken exact and only the interpolation errs: the
    # mean error must fall about 4x each time h_x halves, stay under the 1D
    # bound h_x^2 / 8 max|F''| (which implies the paper's d^2/8 form), and y
    # and z (affine) must be reproduced to rounding.
    T, box = 0.5, 0.5
    F2_max = 2.0 * T / (1.0 - box * T) ** 3          # max of d^2/dx0^2 x0 / (1 - x0 T)
    rng = np.random.default_rng(11)
    start = rng.uniform(0.0, box, size=(4000, 3))
    exact = _quadratic_flow_map(start, T)
    means = []
    for n in (8, 16, 32, 64):
        S, hx = (n + 1,) * 3, box / n                  # dyadic spacing: exact lattice
        jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
        X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * hx
        path = oracle.stitch(S, (0.0, 0.0, 0.0), (hx, hx, hx), [_quadratic_flow_map(X, T)], start)
        err = np.abs(path[1] - exact)
        assert np.max(err[:, 1:]) < 1e-14
        assert np.max(err[:, 0]) <= hx * hx / 8.0 * F2_max * (1.0 + 1e-9)
        assert np.max(err[:, 0]) <= 9.0 / 8.0 * hx * hx * F2_max
        means.append(float(np.mean(err[:, 0])))
    ratios = [means[k] / means[k + 1] for k in range(len(means) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_stitched_pathline_error_stays_second_order_over_intervals():
    # Eq. (global) for n stitched intervals: the error grows with the number
    # of intervals but keeps the h_x^2 order. Three intervals of the same
    # closed-form map, lattice spacings 1/16 and 1/32 of the box.
    T, box = 0.25, 0.5
    rng = np.random.default_rng(12)
    start = rng.uniform(0.0, 0.2, size=(2000, 3))      # stays inside for 3 intervals
    exact = start.copy()
    for _ in range(3):
        exact = _quadratic_flow_map(exact, T)
    assert np.max(exact[:, 0]) < box
    errs = []
    for n in (16, 32):
        S, hx = (n + 1,) * 3, box / n
        jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
        X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * hx
        E = _quadratic_flow_map(X, T)
        path = oracle.stitch(S, (0.0, 0.0, 0.0), (hx, hx, hx), [E, E, E], start)
        assert np.all(np.isfinite(path[3]))
        errs.append(float(np.mean(np.abs(path[3] - exact)[:, 0])))
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def _unit_cell_lattice(E8):
    # corner (a, b, c) of the unit cell -> lattice entry, x fastest
    return np.asarray(E8, dtype=np.float64).reshape(8, 3)


def test_barycentric_stitching_worked_example():
    # Kuhn split of the unit cell (Sec. 3.2's barycentric coordinates over a
    # Delaunay tetrahedron). At (0.7, 0.2, 0.4): x > z > y, so the
    # tetrahedron is (0,0,0), (1,0,0), (1,0,1), (1,1,1) with weights
    # 1 - 0.7, 0.7 - 0.4, 0.4 - 0.2, 0.2. At the cell centre every fraction
    # is 1/2: the weights are 1/2 on (0,0,0) and on (1,1,1), nothing else.
    rng = np.random.default_rng(13)
    E = rng.standard_normal((8, 3))          # index a + 2b + 4c
    c000, c100, c101, c111 = E[0], E[1], E[1 + 4], E[7]
    path = oracle.stitch((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), [E],
                         np.array([[0.7, 0.2, 0.4], [0.5, 0.5, 0.5]]), scheme="barycentric")
    assert np.allclose(path[1, 0], 0.3 * c000 + 0.3 * c100 + 0.2 * c101 + 0.2 * c111, atol=1e-14)
    assert np.allclose(path[1, 1], 0.5 * c000 + 0.5 * c111, atol=1e-14)
    # bilinear data x*y: trilinear is exact at the centre (1/4), the Kuhn
    # tetrahedron gives the diagonal average (1/2)
    xy = np.array([[float(a * b)] * 3 for c in range(2) for b in range(2) for a in range(2)])
    centre = np.array([[0.5, 0.5, 0.5]])
    tri = oracle.stitch((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), [xy], centre)
    bary = oracle.stitch((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), [xy], centre, scheme="barycentric")
    assert np.allclose(tri[1, 0], 0.25) and np.allclose(bary[1, 0], 0.5)


def test_barycentric_stitching_composes_affine_maps_and_is_continuous():
    S, o, sp = (12, 10, 9), (0.0, 0.0, 0.0), (0.5, 0.5, 0.5)
    M1 = np.array([[1.0, 0.05, 0.0], [-0.05, 1.0, 0.02], [0.0, 0.01, 0.98]])
    M2 = np.array([[0.97, 0.0, 0.03], [0.02, 1.01, 0.0], [0.0, -0.02, 1.0]])
    b1, b2 = np.array([0.1, -0.05, 0.2]), np.array([-0.1, 0.1, 0.05])
    E1, E2 = _affine_lattice(S, o, sp, M1, b1), _affine_lattice(S, o, sp, M2, b2)
    rng = np.random.default_rng(14)
    start = rng.uniform(1.5, 3.5, size=(50, 3))
    path = oracle.stitch(S, o, sp, [E1, E2], start, scheme="barycentric")
    want1 = start @ M1.T + b1
    assert np.max(np.abs(path[1] - want1)) < 1e-12
    assert np.max(np.abs(path[2] - (want1 @ M2.T + b2))) < 1e-12
    # across the faces between tetrahedra (fx = fy, fy = fz) and between
    # cells the interpolant is continuous: points eps apart differ by O(eps)
    E = rng.standard_normal((S[0] * S[1] * S[2], 3))
    eps = 1e-9
    base = np.array([[1.3, 1.3, 2.2], [1.8, 2.1, 2.1], [2.0, 1.7, 1.1], [1.6, 1.6, 1.6]])
    for d in (np.array([eps, -eps, 0.0]), np.array([0.0, eps, -eps]), np.array([eps, 0.0, 0.0])):
        p_lo = oracle.stitch(S, o, sp, [E], base - d, scheme="barycentric")[1]
        p_hi = oracle.stitch(S, o, sp, [E], base + d, scheme="barycentric")[1]
        assert np.max(np.abs(p_hi - p_lo)) < 1e-6


def test_barycentric_stitching_is_second_order_and_uses_only_its_tetrahedron():
    T, box = 0.5, 0.5
    rng = np.random.default_rng(15)
    start = rng.uniform(0.0, box, size=(4000, 3))
    exact = _quadratic_flow_map(start, T)
    means = []
    for n in (8, 16, 32):
        S, hx = (n + 1,) * 3, box / n
        jz, jy, jx = np.meshgrid(np.arange(S[2]), np.arange(S[1]), np.arange(S[0]), indexing="ij")
        X = np.stack([jx, jy, jz], axis=-1).reshape(-1, 3) * hx
        path = oracle.stitch(S, (0.0, 0.0, 0.0), (hx, hx, hx), [_quadratic_flow_map(X, T)], start,
                             scheme="barycentric")
        err = np.abs(path[1] - exact)
        assert np.max(err[:, 1:]) < 1e-14
        means.append(float(np.mean(err[:, 0])))
    ratios = [means[k] / means[k + 1] for k in range(len(means) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios
    # a missing entry off the particle's tetrahedron does not stop it; one
    # on it does (trilinear stops for either)
    E = rng.standard_normal((8, 3))
    q = np.array([[0.7, 0.2, 0.4]])                      # tetrahedron 000, 100, 101, 111
    off, on = E.copy(), E.copy()
    off[2] = np.nan                                      # corner (0, 1, 0)
    on[5] = np.nan                                       # corner (1, 0, 1)
    grid = ((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    assert np.all(np.isfinite(oracle.stitch(*grid, [off], q, scheme="barycentric")[1]))
    assert np.all(np.isnan(oracle.stitch(*grid, [on], q, scheme="barycentric")[1]))
    assert np.all(np.isnan(oracle.stitch(*grid, [off], q)[1]))
