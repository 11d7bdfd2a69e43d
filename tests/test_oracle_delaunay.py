"""Pins of the oracle's Delaunay reconstruction (Sec. 3.2: a Delaunay
triangulation over the start locations of the valid basis flows, then
barycentric interpolation), independent of its code:

* the definition of a Delaunay triangulation, checked directly: the
  tetrahedra have positive volume, tile the convex hull of the valid points
  (their volumes add up to the hull volume from scipy's Qhull, and no point
  of the lattice lies in two interiors), and no valid point lies strictly
  inside a tetrahedron's circumsphere (floating point, with a tolerance);
* exactness of barycentric interpolation for affine flow maps;
* a closed form of the Delaunay property: filling data f(x) = |x|^2 at a
  missing lattice point j whose two neighbours along some axis are valid
  gives |j|^2 + 1 exactly (the lower convex hull of the lifted points is the
  smallest convex combination of |p|^2 over points p averaging to j; all
  valid points are at least 1 away from j and the pair j +- e_a reaches
  that bound), which a non-Delaunay triangulation of the same points misses;
* on the lattice's edges, the linear interpolant of the nearest valid
  neighbours along the edge (both bounding planes support the hull); a
  missing corner, or an edge entry with no valid neighbour on one side,
  stays missing; affine maps filled exactly on faces;
* a full lattice is returned unchanged;
* the tie-breaking reading: on small lattices, full and with holes, the
  tetrahedra equal those of a brute-force lower convex hull of the points
  lifted with explicit exact rational weights (a linear solve per 4-point
  set and a test against every other point, no determinant).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _holes(S, frac, seed, balls=0):
    rng = np.random.default_rng(seed)
    P = int(np.prod(S))
    v = rng.random(P) >= frac
    X = oracle.lattice_coords(S, np.arange(P))
    for _ in range(balls):
        c = rng.uniform(2, np.array(S) - 3)
        r = rng.uniform(1.0, 2.2)
        v &= np.linalg.norm(X - c, axis=1) > r
    return v


def _vol(V):
    return np.einsum("ti,ti->t", V[:, 1] - V[:, 0], np.cross(V[:, 2] - V[:, 0], V[:, 3] - V[:, 0])) / 6.0


@pytest.mark.parametrize("S,frac,balls,seed", [((7, 6, 5), 0.15, 0, 1), ((9, 8, 7), 0.05, 3, 2), ((6, 6, 6), 0.0, 2, 3)])
def test_triangulation_is_delaunay_and_tiles_the_hull(S, frac, balls, seed):
    from scipy.spatial import ConvexHull
    v = _holes(S, frac, seed, balls)
    T = oracle.delaunay(S, v)
    V = oracle.lattice_coords(S, T)
    vol = _vol(V)
    assert np.all(vol > 0)
    pts = oracle.lattice_coords(S, np.flatnonzero(v))
    assert abs(vol.sum() - ConvexHull(pts).volume) < 1e-9
    # every vertex is a valid point, every valid point is a vertex
    assert np.all(v[T.ravel()]) and set(np.unique(T)) == set(np.flatnonzero(v))
    # empty circumspheres: |p - c|^2 >= r^2 for every valid point p
    A = 2.0 * (V[:, 1:] - V[:, :1])
    b = (V[:, 1:] ** 2).sum(-1) - (V[:, :1] ** 2).sum(-1)
    c = np.linalg.solve(A, b[..., None])[..., 0]
    r2 = ((V[:, 0] - c) ** 2).sum(-1)
    d2 = ((pts[None, :, :] - c[:, None, :]) ** 2).sum(-1)
    assert np.all(d2 >= r2[:, None] - 1e-7)
    # no lattice point lies strictly inside two tetrahedra
    grid = oracle.lattice_coords(S, np.arange(int(np.prod(S)))) + 0.123 * np.array([1.0, 0.37, 0.21])
    Ainv = np.linalg.inv(np.transpose(V[:, 1:] - V[:, :1], (0, 2, 1)))
    l = np.einsum("tij,ptj->pti", Ainv, grid[:, None, :] - V[None, :, 0, :])
    inside = np.all(l > 1e-9, axis=2) & (l.sum(axis=2) < 1 - 1e-9)
    assert inside.sum(axis=1).max() <= 1


def test_affine_flow_map_is_reconstructed_exactly():
    S = (9, 8, 7)
    v = _holes(S, 0.1, 4, balls=2)
    M = np.array([[1.1, 0.2, -0.3], [0.05, 0.9, 0.4], [-0.2, 0.1, 1.3]])
    t = np.array([0.3, -0.7, 1.9])
    X = oracle.lattice_coords(S, np.arange(int(np.prod(S))))
    ends = X @ M.T + t
    f, st = oracle.fill_delaunay(S, np.where(v[:, None], ends, np.nan), v)
    ok = st > 0
    assert np.sum(st == 2) > 20
    assert np.max(np.abs(f[ok] - ends[ok])) < 1e-10


def test_quadratic_data_at_holes_with_a_valid_opposite_pair():
    S = (9, 9, 9)
    v = _holes(S, 0.12, 5)
    X = oracle.lattice_coords(S, np.arange(int(np.prod(S))))
    q = (X ** 2).sum(axis=1, keepdims=True) * np.ones((1, 3))
    f, st = oracle.fill_delaunay(S, q, v)
    P = int(np.prod(S))
    checked = 0
    for j in np.flatnonzero(~v):
        x = X[j].astype(int)
        pairs = []
        for a in range(3):
            lo, hi = x.copy(), x.copy()
            lo[a] -= 1; hi[a] += 1
            if lo[a] >= 0 and hi[a] < S[a]:
                il = lo[0] + S[0] * (lo[1] + S[1] * lo[2])
                ih = hi[0] + S[0] * (hi[1] + S[1] * hi[2])
                pairs.append(v[il] and v[ih])
        if any(pairs):
            assert st[j] == 2
            assert abs(f[j, 0] - ((X[j] ** 2).sum() + 1.0)) < 1e-9, (j, f[j, 0])
            checked += 1
    assert checked > 40


def test_boundary_edges_faces_and_corners():
    """On a lattice edge (two coordinates at the lattice's bounds) both
    bounding planes support the hull of the valid points, so the tetrahedron
    holding a missing entry meets the edge line in the segment between its
    nearest valid neighbours along the edge: the entry takes their linear
    interpolant, whatever the data. On a face an affine map is still filled
    exactly, a missing corner lies outside the hull and stays missing, and
    an edge entry with no valid neighbour on one side stays missing."""
    S = (9, 8, 7)
    rng = np.random.default_rng(12)
    P = int(np.prod(S))
    X = oracle.lattice_coords(S, np.arange(P)).astype(int)
    v = rng.random(P) >= 0.3
    ends = rng.standard_normal((P, 3))
    f, st = oracle.fill_delaunay(S, np.where(v[:, None], ends, np.nan), v)
    hi = np.array(S) - 1
    n_edge = 0
    for j in np.flatnonzero(~v):
        fixed = (X[j] == 0) | (X[j] == hi)
        if fixed.sum() == 3:
            assert st[j] == 0
        if fixed.sum() != 2:
            continue
        a = int(np.flatnonzero(~fixed)[0])
        line = [k for k in range(P) if np.all(np.delete(X[k], a) == np.delete(X[j], a)) and v[k]]
        below = [k for k in line if X[k][a] < X[j][a]]
        above = [k for k in line if X[k][a] > X[j][a]]
        if not below or not above:
            assert st[j] == 0
            continue
        lo = max(below, key=lambda k: X[k][a])
        up = min(above, key=lambda k: X[k][a])
        t = (X[j][a] - X[lo][a]) / (X[up][a] - X[lo][a])
        assert st[j] == 2
        assert np.max(np.abs(f[j] - ((1 - t) * ends[lo] + t * ends[up]))) < 1e-12
        n_edge += 1
    assert n_edge > 10
    # an affine map is filled exactly on faces too
    M = np.array([[0.7, -0.2, 0.1], [0.3, 1.2, -0.4], [0.05, 0.1, 0.9]])
    aff = X @ M.T + np.array([1.0, 2.0, -3.0])
    f, st = oracle.fill_delaunay(S, np.where(v[:, None], aff, np.nan), v)
    face = np.any((X == 0) | (X == hi), axis=1)
    assert np.sum((st == 2) & face) > 20
    assert np.max(np.abs(f[st > 0] - aff[st > 0])) < 1e-10


def test_flat_lattice_has_no_tetrahedra():
    S = (6, 5, 1)
    v = np.random.default_rng(13).random(30) >= 0.2
    f, st = oracle.fill_delaunay(S, np.zeros((30, 3)), v)
    assert np.all(st[~v] == 0) and np.all(np.isnan(f[~v])) and np.all(st[v] == 1)


def test_full_lattice_unchanged():
    S = (5, 4, 6)
    v = np.ones(int(np.prod(S)), dtype=bool)
    ends = np.random.default_rng(6).standard_normal((int(np.prod(S)), 3))
    f, st = oracle.fill_delaunay(S, ends, v)
    assert np.array_equal(f, ends) and np.all(st == 1)


def _regular_triangulation_brute_force(S, valid, t):
    """Lower convex hull of the valid lattice points lifted to
    w(j) = |j|^2 + t^(r + 1), r = the canonical lattice id, in exact
    rational arithmetic: a 4-point set is a tetrahedron of the regular
    triangulation when the affine function through its four lifted points
    lies strictly below every other lifted point. With t = 1e-6 the explicit
    weights order ties as the reading's infinitesimals do on a lattice this
    small (every cofactor is an integer below 100 in size, so a weight
    outweighs all later ones together, and all of them together stay below
    the unit step of an unperturbed determinant)."""
    from fractions import Fraction
    from itertools import combinations
    ids = [int(i) for i in np.flatnonzero(valid)]
    X = {i: [int(c) for c in oracle.lattice_coords(S, np.array([i]))[0]] for i in ids}
    w = {i: Fraction(sum(c * c for c in X[i])) + t ** (i + 1) for i in ids}

    def solve(rows, rhs):
        # Gauss-Jordan elimination over the rationals; None when singular
        m = [[Fraction(v) for v in r] + [rhs[k]] for k, r in enumerate(rows)]
        n = len(m)
        for c in range(n):
            piv = next((r for r in range(c, n) if m[r][c] != 0), None)
            if piv is None:
                return None
            m[c], m[piv] = m[piv], m[c]
            for r in range(n):
                if r != c and m[r][c] != 0:
                    f = m[r][c] / m[c][c]
                    m[r] = [a - f * b for a, b in zip(m[r], m[c])]
        return [m[r][n] / m[r][r] for r in range(n)]

    tets = set()
    for q in combinations(ids, 4):
        coef = solve([X[i] + [1] for i in q], [w[i] for i in q])
        if coef is None:          # coplanar points span no tetrahedron
            continue
        if all(w[e] > sum(a * b for a, b in zip(coef, X[e] + [1])) for e in ids if e not in q):
            tets.add(tuple(sorted(q)))
    return tets


@pytest.mark.parametrize("S,holes", [((3, 3, 2), []), ((3, 3, 3), [13]), ((3, 3, 3), [7, 13, 15]),
                                     ((4, 3, 2), [5, 18]), ((2, 2, 2), [])])
def test_tie_breaking_matches_the_lower_hull_with_exact_weights(S, holes):
    """Lattice points are cospherical in eights, so only the tie-breaking
    reading fixes the triangulation. The oracle's must be the brute-force
    lower hull of the lifted points with explicit weights ordered as the
    reading orders its infinitesimals (lowest canonical id largest)."""
    from fractions import Fraction
    v = np.ones(int(np.prod(S)), dtype=bool)
    v[holes] = False
    want = _regular_triangulation_brute_force(S, v, Fraction(1, 10 ** 6))
    got = {tuple(sorted(int(i) for i in t)) for t in oracle.delaunay(S, v)}
    assert got == want
