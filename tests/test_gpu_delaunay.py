"""GPU Delaunay reconstruction (bto_fill_delaunay) against the FP64 oracle's
Bowyer-Watson triangulation (oracle.fill_delaunay), through the C ABI.

Both sides decide with exact integer predicates under the same tie-breaking
reading, so they pick the same Delaunay tetrahedron (or, for a point on a
shared face, tetrahedra whose barycentric interpolants agree there): the
statuses must be identical and the filled ends agree to FP32 rounding of
the FP64 result (relative 1e-6 of the ends' scale).
"""
import numpy as np
import pytest

import oracle
from paper_2004_02003_gb300 import bto

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    from paper_2004_02003_gb300 import build
    build.build()
    bto.load()


def _holes(S, frac, seed, balls=0):
    rng = np.random.default_rng(seed)
    P = int(np.prod(S))
    v = rng.random(P) >= frac
    X = oracle.lattice_coords(S, np.arange(P))
    for _ in range(balls):
        c = rng.uniform(1, np.array(S) - 2)
        r = rng.uniform(1.0, 2.5)
        v &= np.linalg.norm(X - c, axis=1) > r
    return v


def _gpu_fill(S, ends, valid):
    import torch
    e = torch.from_numpy(np.ascontiguousarray(ends, dtype=np.float32)).cuda()
    v = torch.from_numpy(np.ascontiguousarray(valid, dtype=np.uint8)).cuda()
    out = torch.empty_like(e)
    st = torch.empty_like(v)
    bto.bto_fill_delaunay(S, e, v, out, st)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("S,frac,balls,seed", [((12, 11, 10), 0.08, 3, 11), ((9, 14, 8), 0.2, 0, 12),
                                              ((10, 10, 10), 0.02, 5, 13), ((6, 5, 4), 0.3, 1, 14),
                                              ((7, 9, 2), 0.25, 0, 15), ((20, 3, 16), 0.15, 2, 16)])
def test_delaunay_fill_matches_oracle(S, frac, balls, seed):
    v = _holes(S, frac, seed, balls)
    X = oracle.lattice_coords(S, np.arange(int(np.prod(S))))
    ends = np.stack([X[:, 0] + 0.3 * np.sin(0.7 * X[:, 1]), X[:, 1] + 0.2 * np.cos(0.5 * X[:, 2] + X[:, 0]),
                     X[:, 2] + 0.1 * X[:, 0] * X[:, 1] / 10.0], axis=1)
    ends_in = np.where(v[:, None], ends, np.nan).astype(np.float32)
    ref, st_o = oracle.fill_delaunay(S, ends_in.astype(np.float64), v)
    got, st_g = _gpu_fill(S, ends_in, v)
    bad = np.flatnonzero(st_g != st_o)
    if bad.size:
        P = np.flatnonzero(v)
        for j in bad[:12]:
            d = np.sqrt(((oracle.lattice_coords(S, P) - X[j]) ** 2).sum(axis=1)).min()
            print("mismatch at", X[j], "gpu", st_g[j], "oracle", st_o[j], "nearest valid %.2f" % d)
    assert bad.size == 0, f"{bad.size} statuses differ"
    filled = st_o == 2
    assert filled.sum() > 0
    scale = np.abs(ref[filled]).max()
    assert np.max(np.abs(got[filled] - ref[filled])) <= 2e-6 * scale
    assert np.array_equal(got[st_o == 1], ends_in[st_o == 1])
    assert np.all(np.isnan(got[st_o == 0]))


def test_delaunay_fill_affine_and_quadratic_closed_forms():
    S = (16, 15, 14)
    v = _holes(S, 0.06, 21, balls=4)
    X = oracle.lattice_coords(S, np.arange(int(np.prod(S))))
    M = np.array([[1.1, 0.2, -0.3], [0.05, 0.9, 0.4], [-0.2, 0.1, 1.3]])
    aff = (X @ M.T + np.array([0.5, -1.0, 2.0])).astype(np.float32)
    got, st = _gpu_fill(S, np.where(v[:, None], aff, np.nan), v)
    ok = st == 2
    assert ok.sum() > 50
    assert np.max(np.abs(got[ok] - aff[ok])) < 1e-4
    # |x|^2 at holes with a valid opposite neighbour pair: |j|^2 + 1 exactly
    q = ((X ** 2).sum(axis=1, keepdims=True) * np.ones((1, 3))).astype(np.float32)
    gq, sq = _gpu_fill(S, np.where(v[:, None], q, np.nan), v)
    n = 0
    for j in np.flatnonzero(~v):
        x = X[j].astype(int)
        for a in range(3):
            lo, hi = x.copy(), x.copy()
            lo[a] -= 1; hi[a] += 1
            if lo[a] < 0 or hi[a] >= S[a]:
                continue
            il = lo[0] + S[0] * (lo[1] + S[1] * lo[2])
            ih = hi[0] + S[0] * (hi[1] + S[1] * hi[2])
            if v[il] and v[ih]:
                assert sq[j] == 2 and gq[j, 0] == np.float32((X[j] ** 2).sum() + 1.0), j
                n += 1
                break
    assert n > 50


def test_boundary_entries_and_flat_lattice():
    """Entries on the lattice's faces and edges are filled over the face's
    triangles and the edge's segments, as the oracle's tetrahedra give them;
    corners stay missing; a lattice one point thick has no tetrahedra."""
    S = (11, 10, 9)
    rng = np.random.default_rng(17)
    P = int(np.prod(S))
    X = oracle.lattice_coords(S, np.arange(P)).astype(int)
    face = np.any((X == 0) | (X == np.array(S) - 1), axis=1)
    v = ~(face & (rng.random(P) < 0.35))           # holes on the faces only
    ends = rng.standard_normal((P, 3)).astype(np.float32)
    ends_in = np.where(v[:, None], ends, np.nan).astype(np.float32)
    ref, st_o = oracle.fill_delaunay(S, ends_in.astype(np.float64), v)
    got, st_g = _gpu_fill(S, ends_in, v)
    assert np.array_equal(st_g, st_o)
    fixed = ((X == 0) | (X == np.array(S) - 1)).sum(axis=1)
    assert np.sum((st_o == 2) & (fixed == 1)) > 50 and np.sum((st_o == 2) & (fixed == 2)) > 5
    assert np.all(st_o[(fixed == 3) & ~v] == 0)
    filled = st_o == 2
    assert np.max(np.abs(got[filled] - ref[filled])) <= 2e-6 * np.abs(ref[filled]).max()
    # one point thick: nothing to interpolate over
    S1 = (8, 6, 1)
    v1 = rng.random(48) >= 0.25
    g1, s1 = _gpu_fill(S1, np.zeros((48, 3), np.float32), v1)
    assert np.all(s1[~v1] == 0) and np.all(np.isnan(g1[~v1])) and np.all(s1[v1] == 1)


@pytest.mark.parametrize("S,k,seed", [((9, 8, 7), 12, 1), ((11, 10, 9), 15, 2)])
def test_entries_on_the_hull_of_the_valid_points(S, k, seed):
    """Valid points fill the half space x + y + z <= k, with half of the
    plane x + y + z = k and 5% of the rest missing: missing entries on that
    plane lie on facets of the hull, where the walk ends on a facet with a
    far starting point at weight 0 and has to certify the facet (wrapping
    across it to a Delaunay tetrahedron of the valid points); entries beyond
    the plane are outside the hull and stay missing."""
    P = int(np.prod(S))
    X = oracle.lattice_coords(S, np.arange(P))
    r = np.random.default_rng(seed)
    t = X.sum(axis=1)
    v = (t <= k) & ~((t == k) & (r.random(P) < 0.5)) & (r.random(P) > 0.05)
    ends = r.standard_normal((P, 3)).astype(np.float32)
    ends_in = np.where(v[:, None], ends, np.nan).astype(np.float32)
    ref, st_o = oracle.fill_delaunay(S, ends_in.astype(np.float64), v)
    got, st_g = _gpu_fill(S, ends_in, v)
    assert np.array_equal(st_g, st_o)
    on_plane = (t == k) & ~v
    assert np.sum(on_plane & (st_o == 2)) > 10 and np.all(st_o[(t > k) & ~v] == 0)
    filled = st_o == 2
    assert np.max(np.abs(got[filled] - ref[filled])) <= 2e-6 * np.abs(ref[filled]).max()


def test_large_lattice_sampled_against_local_oracle():
    """A 96 x 96 x 64 lattice with the hole pattern of block faces (slabs two
    points thick at 47-48 along x and along y, 2% random holes, four
    spherical voids) is filled whole on the GPU. For sampled missing entries
    at least 6 points from the lattice's faces, the oracle triangulates the
    13^3 neighbourhood around the entry. Where the tetrahedron holding the
    entry has a circumsphere that no lattice point outside the neighbourhood
    can enter, it is also the tetrahedron of the whole lattice, and the GPU
    must have filled the entry with the same interpolant."""
    S = (96, 96, 64)
    P = int(np.prod(S))
    X = oracle.lattice_coords(S, np.arange(P)).astype(np.int64)
    rng = np.random.default_rng(31)
    v = rng.random(P) > 0.02
    v &= ~np.isin(X[:, 0], (47, 48)) & ~np.isin(X[:, 1], (47, 48))
    for _ in range(4):
        c = rng.uniform(10, np.array(S) - 11)
        v &= np.linalg.norm(X - c, axis=1) > rng.uniform(2.0, 3.0)
    ends = np.stack([X[:, 0] + 0.3 * np.sin(0.21 * X[:, 1]), X[:, 1] + 0.2 * np.cos(0.17 * X[:, 2] + 0.1 * X[:, 0]),
                     X[:, 2] + 0.01 * X[:, 0] * X[:, 1] / 9.0], axis=1).astype(np.float32)
    got, st = _gpu_fill(S, np.where(v[:, None], ends, np.nan).astype(np.float32), v)
    inner = np.all((X >= 6) & (X <= np.array(S) - 7), axis=1) & ~v
    sample = rng.choice(np.flatnonzero(inner), size=32, replace=False)
    S2 = (13, 13, 13)
    off = oracle.lattice_coords(S2, np.arange(13 ** 3)).astype(np.int64) - 6
    checked = 0
    for j in sample:
        g = X[j] + off
        gid = g[:, 0] + S[0] * (g[:, 1] + S[1] * g[:, 2])
        tets = oracle.delaunay(S2, v[gid])
        V = oracle.lattice_coords(S2, tets)
        A = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1))
        lam3 = np.einsum("tij,tj->ti", np.linalg.inv(A), np.array([6.0, 6.0, 6.0]) - V[:, 0, :])
        lam = np.concatenate([1.0 - lam3.sum(axis=1, keepdims=True), lam3], axis=1)
        hit = np.flatnonzero(np.all(lam >= -1e-9, axis=1))
        if hit.size == 0:
            continue
        t = hit[0]
        M = 2.0 * (V[t, 1:] - V[t, :1])
        ctr = np.linalg.solve(M, (V[t, 1:] ** 2).sum(axis=1) - (V[t, 0] ** 2).sum())
        rad = np.sqrt(((V[t, 0] - ctr) ** 2).sum())
        if np.any(ctr - rad <= -1.0 + 1e-6) or np.any(ctr + rad >= 13.0 - 1e-6):
            continue
        want = lam[t] @ ends[gid[tets[t]]].astype(np.float64)
        assert st[j] == 2, (X[j], st[j])
        assert np.max(np.abs(got[j] - want)) <= 2e-6 * np.abs(ends).max(), (X[j], got[j], want)
        checked += 1
    assert checked >= 20, checked


def test_large_lattice_face_entries_against_local_oracle():
    """Face entries of the same kind of lattice: for sampled missing entries
    on the faces x = 0 and z = S_z - 1 (6 or more points from the face's
    edges), the oracle triangulates the 13 x 13 x 7 neighbourhood that the
    face bounds. The tetrahedron holding the entry meets the face in a
    triangle of the face's own triangulation; where that triangle's
    circumcircle stays inside the neighbourhood's extent on the face, it is
    the triangle of the whole lattice, and the GPU's value must equal the
    oracle's."""
    S = (64, 72, 48)
    P = int(np.prod(S))
    X = oracle.lattice_coords(S, np.arange(P)).astype(np.int64)
    rng = np.random.default_rng(37)
    face = (X[:, 0] == 0) | (X[:, 2] == S[2] - 1)
    v = ~(face & (rng.random(P) < 0.3)) & (rng.random(P) > 0.02)
    ends = np.stack([X[:, 0] + 0.2 * np.sin(0.3 * X[:, 1]), X[:, 1] + 0.1 * X[:, 2] / 7.0,
                     X[:, 2] + 0.25 * np.cos(0.2 * X[:, 0] + 0.1 * X[:, 1])], axis=1).astype(np.float32)
    got, st = _gpu_fill(S, np.where(v[:, None], ends, np.nan).astype(np.float32), v)
    checked = 0
    for fixed_axis, at in ((0, 0), (2, S[2] - 1)):
        free = [a for a in range(3) if a != fixed_axis]
        cand = (X[:, fixed_axis] == at) & ~v
        for a in free:
            cand &= (X[:, a] >= 6) & (X[:, a] <= S[a] - 7)
        for j in rng.choice(np.flatnonzero(cand), size=12, replace=False):
            S2 = [13, 13, 13]
            S2[fixed_axis] = 7
            lo = X[j].copy()
            for a in free:
                lo[a] -= 6
            lo[fixed_axis] = 0 if at == 0 else at - 6
            loc = oracle.lattice_coords(S2, np.arange(int(np.prod(S2)))).astype(np.int64)
            g = loc + lo
            gid = g[:, 0] + S[0] * (g[:, 1] + S[1] * g[:, 2])
            q = (X[j] - lo).astype(np.float64)
            tets = oracle.delaunay(S2, v[gid])
            V = oracle.lattice_coords(S2, tets)
            A = np.transpose(V[:, 1:, :] - V[:, :1, :], (0, 2, 1))
            lam3 = np.einsum("tij,tj->ti", np.linalg.inv(A), q - V[:, 0, :])
            lam = np.concatenate([1.0 - lam3.sum(axis=1, keepdims=True), lam3], axis=1)
            hit = np.flatnonzero(np.all(lam >= -1e-9, axis=1))
            if hit.size == 0:
                continue
            t = hit[0]
            on = np.flatnonzero(V[t, :, fixed_axis] == q[fixed_axis])
            if on.size != 3:
                continue
            W = V[t][on][:, free]
            M = 2.0 * (W[1:] - W[:1])
            ctr = np.linalg.solve(M, (W[1:] ** 2).sum(axis=1) - (W[0] ** 2).sum())
            rad = np.sqrt(((W[0] - ctr) ** 2).sum())
            if np.any(ctr - rad <= -1.0 + 1e-6) or np.any(ctr + rad >= 13.0 - 1e-6):
                continue
            want = lam[t] @ ends[gid[tets[t]]].astype(np.float64)
            assert st[j] == 2, (X[j], st[j])
            assert np.max(np.abs(got[j] - want)) <= 2e-6 * np.abs(ends).max(), (X[j], got[j], want)
            checked += 1
    assert checked >= 12, checked
