// Post hoc reconstruction of missing basis flows over a Delaunay
// triangulation of the valid ones (Sec. 3.2: a Delaunay triangulation over
// the start locations of the loaded basis flows, then barycentric
// interpolation), for sm_103a.
//
// The start locations are seed-lattice points j. The Delaunay tetrahedron
// that holds a point q is the lower facet, above q, of the convex hull of
// the points lifted to w(j) = |j|^2: equivalently, the optimal basis of the
// linear program
//     minimise   sum_i lambda_i w(j_i)
//     subject to sum_i lambda_i j_i = q,  sum_i lambda_i = 1,  lambda >= 0,
// whose optimal lambda are q's barycentric coordinates in that tetrahedron.
// Each warp solves this program for one missing lattice point at a time by
// the simplex method over the valid points of a window around it (the
// lanes share out the window's points): the basis is a tetrahedron holding
// q; a point inside the tetrahedron's circumsphere (below the plane through
// its lifted vertices) has a negative reduced cost and enters; the ratio
// test picks the vertex that leaves so that q stays inside. It starts from
// four far points around q and stops when no window point lies inside the
// circumsphere. The result is the Delaunay tetrahedron of all valid points
// when its circumsphere fits in the window (no lattice point outside the
// window can then lie inside it); otherwise the window grows (radius 2 to
// 8 lattice units) and the walk resumes.
//
// Entries on the lattice's outer faces lie on the hull of the valid points.
// There the face's plane supports the lifted point set, so the tetrahedra
// meet the face in the regular triangulation of the face's own points
// under the same weights (|j|^2 differs from the face's squared in-plane
// coordinates by a constant): such an entry is solved by the same simplex
// method in the face's two free coordinates, with triangles. On a lattice
// edge two planes support the hull, and the triangulation meets the edge
// line in the segments between consecutive valid points: the entry takes
// the linear interpolant of its nearest valid neighbours along the edge. A
// missing corner is outside the hull. A lattice one point thick along an
// axis has no tetrahedra; its missing entries stay missing.
//
// Cospherical lattice points (a cell's 8 corners) make the Delaunay
// triangulation non-unique. Ties are broken as if the lifted weights were
// |j|^2 + d_r(j), with infinitesimals d_0 >> d_1 >> ... > 0 ordered by the
// point's canonical lattice id (the four far points last): when the
// unperturbed predicate is zero, the term of the lowest-ranked point with a
// non-zero cofactor decides. Predicates are exact (integer arithmetic), and
// the simplex method takes the lowest-ranked entering point and breaks
// ratio ties by rank (Bland's rule), so it terminates.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"

namespace bto {
namespace {

typedef __int128 i128;

struct LPt {
    int64_t x, y, z;   // lattice coordinates relative to the query point
    int64_t rank;
};

// Magnitudes: window points lie within kMaxWindow of the query and the four
// starting points kFar from it, so coordinate differences are at most
// 2 kFar + 2 kMaxWindow < 2^12: a 3 x 3 determinant of differences stays
// below 6 * 2^36 and the lifted 4 x 4 determinant below 4 * 3 * 2^22 * 6 *
// 2^33 < 2^63, so 64-bit integers are exact; only the ratio test's cross
// products (two orientations) need 128 bits.
__device__ __forceinline__ int64_t det3(int64_t a0, int64_t a1, int64_t a2, int64_t b0, int64_t b1, int64_t b2,
                                        int64_t c0, int64_t c1, int64_t c2) {
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
}

// orientation: determinant of the rows b - a, c - a, d - a
__device__ __forceinline__ int64_t orient(const LPt &a, const LPt &b, const LPt &c, const LPt &d) {
    return det3(b.x - a.x, b.y - a.y, b.z - a.z, c.x - a.x, c.y - a.y, c.z - a.z, d.x - a.x, d.y - a.y,
                d.z - a.z);
}

__device__ __noinline__ int perturbed_sign(const LPt (&t)[4], const LPt &e);

// Sign of the 5 x 5 determinant with rows (x, y, z, w, 1) of t0..t3, e
// under the perturbed lifting: negative when e is inside the circumsphere of
// the positively oriented tetrahedron (t0, t1, t2, t3).
__device__ __noinline__ int lifted_sign(const LPt (&t)[4], const LPt &e) {
    // unperturbed: rows (p - e, |p - e|^2) of the tetrahedron, expanded
    // along the squared-length column
    int64_t r[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        r[i][0] = t[i].x - e.x;
        r[i][1] = t[i].y - e.y;
        r[i][2] = t[i].z - e.z;
        r[i][3] = r[i][0] * r[i][0] + r[i][1] * r[i][1] + r[i][2] * r[i][2];
    }
    int64_t d0 = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = (i + 1) & 3, b = (i + 2) & 3, c = (i + 3) & 3;
        // rows a, b, c in increasing order for the minor's sign
        int u0 = a, u1 = b, u2 = c;
        if (u0 > u1) { const int s = u0; u0 = u1; u1 = s; }
        if (u1 > u2) { const int s = u1; u1 = u2; u2 = s; }
        if (u0 > u1) { const int s = u0; u0 = u1; u1 = s; }
        const int64_t m = det3(r[u0][0], r[u0][1], r[u0][2], r[u1][0], r[u1][1], r[u1][2], r[u2][0], r[u2][1],
                               r[u2][2]);
        d0 += (((i + 3) & 1) ? -m : m) * r[i][3];
    }
    if (d0 != 0) return d0 > 0 ? 1 : -1;
    return perturbed_sign(t, e);
}

// The sign when the unperturbed determinant is zero: point k of
// (t0, t1, t2, t3, e) carries the term (-1)^(k+3) * (-orient(the other
// four, in order)); the lowest-ranked point with a non-zero term decides.
__device__ __noinline__ int perturbed_sign(const LPt (&t)[4], const LPt &e) {
    const LPt *p[5] = {&t[0], &t[1], &t[2], &t[3], &e};
    bool used[5] = {false, false, false, false, false};
    for (int round = 0; round < 5; ++round) {
        int k = -1;
        for (int m = 0; m < 5; ++m)
            if (!used[m] && (k < 0 || p[m]->rank < p[k]->rank)) k = m;
        used[k] = true;
        const LPt *q[4];
        for (int m = 0, n = 0; m < 5; ++m)
            if (m != k) q[n++] = p[m];
        const int64_t o = -orient(*q[0], *q[1], *q[2], *q[3]);
        if (o != 0) {
            const int64_t c = ((k + 3) & 1) ? -o : o;
            return c > 0 ? 1 : -1;
        }
    }
    return 0;
}

__device__ __forceinline__ int64_t lattice_rank(int3 S, int64_t x, int64_t y, int64_t z) {
    return x + (int64_t)S.x * (y + (int64_t)S.y * z);
}

constexpr int64_t kFar = 1024;   // distance of the four starting points, lattice units
constexpr int kMaxPivots = 512;
constexpr int kMaxWindow = 8;      // largest window radius, lattice units
constexpr int kMaxWindow2 = 12;    // on a face (a window of 25 x 25 points)
// Work limit (rows plus points) of the scan that shows that a facet (edge)
// through the query point bounds the hull of all valid points.
constexpr int64_t kHullScanWork = (int64_t)1 << 22;

// floor(n / d) and ceil(n / d) for d > 0.
__device__ __forceinline__ int64_t floor_div(int64_t n, int64_t d) { return n >= 0 ? n / d : -((-n + d - 1) / d); }
__device__ __forceinline__ int64_t ceil_div(int64_t n, int64_t d) { return n >= 0 ? (n + d - 1) / d : -((-n) / d); }

// The integers t in [lo, hi] with a t + b > 0, as [t0, t1]; false when none.
__device__ __forceinline__ bool positive_range(int64_t a, int64_t b, int64_t lo, int64_t hi, int64_t &t0,
                                               int64_t &t1) {
    if (a == 0) {
        t0 = lo;
        t1 = hi;
        return b > 0 && lo <= hi;
    }
    if (a > 0) {
        t0 = max(lo, floor_div(-b, a) + 1);
        t1 = hi;
    } else {
        t0 = lo;
        t1 = min(hi, ceil_div(b, -a) - 1);
    }
    return t0 <= t1;
}

// Outcome of one walk in a window of radius R around the lattice point c:
// 1 and the tetrahedron with q's barycentric coordinates, or 0 (no result
// in this window: q outside the hull of its valid points, circumsphere
// larger than the window, or the pivot limit).
// Circumsphere of T (centre and squared radius, FP64), for the filter that
// spares most points the exact predicate.
__device__ __noinline__ void circumsphere(const LPt (&T)[4], double (&ctr)[3], double &r2) {
    double A[3][3], b[3];
    const LPt &a = T[0];
    for (int m = 0; m < 3; ++m) {
        const LPt &p = T[m + 1];
        A[m][0] = 2.0 * (double)(p.x - a.x);
        A[m][1] = 2.0 * (double)(p.y - a.y);
        A[m][2] = 2.0 * (double)(p.z - a.z);
        b[m] = (double)(p.x - a.x) * (double)(p.x - a.x) + (double)(p.y - a.y) * (double)(p.y - a.y) +
               (double)(p.z - a.z) * (double)(p.z - a.z);
    }
    const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                       A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                       A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double c[3];
    for (int m = 0; m < 3; ++m) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) M[r][s] = s == m ? b[r] : A[r][s];
        c[m] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
    }
    ctr[0] = c[0] + (double)a.x; ctr[1] = c[1] + (double)a.y; ctr[2] = c[2] + (double)a.z;
    r2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
}

// The circumsphere of T for the walk's filter: centre and squared radius in
// FP32, relative to q. The 3 x 3 system 2 (p_m - a) . c = |p_m - a|^2 is
// solved by Cramer's rule in exact 64-bit integers (differences below 2^12:
// the determinant stays below 2^42 and the numerators below 2^55); only the
// conversions, the three quotients and the final sums are rounded, so the
// centre is within 3e-7 r of the exact one (T holds q, so |c - q| <= r).
__device__ __forceinline__ void circumsphere_f(const LPt (&T)[4], float (&c)[3], float &r2) {
    int64_t A[3][3], b[3];
    const LPt &a = T[0];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const LPt &p = T[m + 1];
        A[m][0] = 2 * (p.x - a.x);
        A[m][1] = 2 * (p.y - a.y);
        A[m][2] = 2 * (p.z - a.z);
        b[m] = (p.x - a.x) * (p.x - a.x) + (p.y - a.y) * (p.y - a.y) + (p.z - a.z) * (p.z - a.z);
    }
    const float det = (float)det3(A[0][0], A[0][1], A[0][2], A[1][0], A[1][1], A[1][2], A[2][0], A[2][1], A[2][2]);
    const float u0 = (float)det3(b[0], A[0][1], A[0][2], b[1], A[1][1], A[1][2], b[2], A[2][1], A[2][2]) / det;
    const float u1 = (float)det3(A[0][0], b[0], A[0][2], A[1][0], b[1], A[1][2], A[2][0], b[2], A[2][2]) / det;
    const float u2 = (float)det3(A[0][0], A[0][1], b[0], A[1][0], A[1][1], b[1], A[2][0], A[2][1], b[2]) / det;
    c[0] = u0 + (float)a.x;
    c[1] = u1 + (float)a.y;
    c[2] = u2 + (float)a.z;
    r2 = u0 * u0 + u1 * u1 + u2 * u2;
}

// Sets T to the four far starting points (positively oriented).
__device__ void start_tetrahedron(int64_t P, LPt (&T)[4]) {
    const int64_t far[4][3] = {{kFar, kFar, kFar}, {kFar, -kFar, -kFar}, {-kFar, kFar, -kFar}, {-kFar, -kFar, kFar}};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T[k].x = far[k][0]; T[k].y = far[k][1]; T[k].z = far[k][2];
        T[k].rank = P + k;
    }
    if (orient(T[0], T[1], T[2], T[3]) < 0) { const LPt s = T[0]; T[0] = T[1]; T[1] = s; }
}

// True when the circumsphere of T, centred at ctr (relative to the query
// point c) with squared radius r2, stays clear of every lattice plane just
// outside the window [x0, x1] x [y0, y1] x [z0, z1] that lies inside the
// lattice: then no lattice point outside the window is inside it.
__device__ bool sphere_fits(const double (&ctr)[3], double r2, int3 S, int64_t cx, int64_t cy, int64_t cz,
                            int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0, int64_t z1) {
    const double rad = sqrt(r2) * (1.0 + 1e-12) + 1e-9;
    const double lo[3] = {(double)(x0 - cx), (double)(y0 - cy), (double)(z0 - cz)};
    const double hi[3] = {(double)(x1 - cx), (double)(y1 - cy), (double)(z1 - cz)};
    const int64_t ext[3] = {S.x, S.y, S.z};
    const int64_t cc[3] = {cx, cy, cz};
    for (int m = 0; m < 3; ++m) {
        // a window edge on the lattice boundary needs no margin
        if (cc[m] + (int64_t)lo[m] > 0 && ctr[m] - rad <= lo[m] - 1.0) return false;
        if (cc[m] + (int64_t)hi[m] < ext[m] - 1 && ctr[m] + rad >= hi[m] + 1.0) return false;
    }
    return true;
}

// Every routine from here on is warp-cooperative: the 32 lanes of a warp
// solve one missing entry together. They hold the same simplex, split the
// window's points between them (point k of the window goes to lane k mod
// 32, k in rank order), and combine their findings with warp reductions,
// so every decision is warp-uniform and equal to that of a serial scan in
// rank order.
constexpr unsigned kAll = 0xffffffffu;
constexpr int64_t kNone = INT64_MAX;

__device__ __forceinline__ int64_t warp_min(int64_t v) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, (int64_t)__shfl_xor_sync(kAll, (long long)v, o));
    return v;
}
__device__ __forceinline__ int64_t warp_max(int64_t v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_xor_sync(kAll, (long long)v, o));
    return v;
}
__device__ __forceinline__ LPt shfl_xor_pt(const LPt &p, int o) {
    LPt r;
    r.x = __shfl_xor_sync(kAll, (long long)p.x, o);
    r.y = __shfl_xor_sync(kAll, (long long)p.y, o);
    r.z = __shfl_xor_sync(kAll, (long long)p.z, o);
    r.rank = __shfl_xor_sync(kAll, (long long)p.rank, o);
    return r;
}

__device__ __forceinline__ void positive_orientation(LPt (&t)[4]) {
    if (orient(t[0], t[1], t[2], t[3]) < 0) { const LPt s = t[0]; t[0] = t[1]; t[1] = s; }
}

// A lane's walk over a window of wx x wy x wz points in rank order: points
// k = lane, lane + 32, ..., with offsets (x, y, z) inside the window kept
// by additions (a window holds at most 25 x 25 or 17 x 17 x 17 points, and
// a lattice at most 2^31, so 32-bit indices suffice).
struct WinIter {
    int wx, wy, k, x, y, z;
    __device__ WinIter(int wx_, int wy_, int start) : wx(wx_), wy(wy_), k(start) {
        x = start % wx;
        const int q = start / wx;
        y = q % wy;
        z = q / wy;
    }
    __device__ __forceinline__ void step() {
        k += 32;
        x += 32;
        while (x >= wx) {
            x -= wx;
            if (++y == wy) { y = 0; ++z; }
        }
    }
};

// Pivot rule. The first kDeepPivots pivots enter the point deepest inside
// the circumsphere (largest r^2 - |p - c|^2 in FP32, ties to the lowest
// rank), which reaches q's simplex in few pivots; later pivots take the
// lowest-ranked point inside (Bland's rule), which cannot cycle, so every
// walk ends. Either way the entering point passes the exact predicate and
// the walk stops only when no window point is inside the circumsphere.
constexpr int kDeepPivots = 64;

// Warp-maximum key of a candidate: the FP32 depth's bits made monotone in
// the high word, the complement of the rank in the low word (ranks are
// below 2^31); 0 means none.
__device__ __forceinline__ unsigned long long depth_key(float depth, int64_t rank) {
    const unsigned bits = __float_as_uint(depth);
    const unsigned mono = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
    return ((unsigned long long)mono << 32) | (0xffffffffu - (unsigned)rank);
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kAll, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Lattice coordinates of the point of rank r (r < 2^31).
__device__ __forceinline__ void rank_coords(int3 S, int64_t r, int64_t (&p)[3]) {
    const int rr = (int)r;
    p[0] = rr % S.x;
    const int q = rr / S.x;
    p[1] = q % S.y;
    p[2] = q / S.y;
}

// The walk ended with one starting point (vertex kf of T) at weight exactly
// 0: q lies on the facet F of the other three vertices, and no window point
// is inside the sphere through F and the far starting point. F is a facet
// of the Delaunay triangulation of all valid points, and q's interpolant is
// the one over F, when (a) wrapping across F to the valid window point D on
// the other side whose sphere through F holds no other such point gives a
// tetrahedron whose sphere holds no valid window point at all and fits in
// the window, or (b) no valid point of the lattice lies strictly on the far
// side of F (F is then on the hull; shown within a work limit). Either way
// T[kf] is replaced by a valid point (D, or a vertex of F) with weight 0.
// Spheres through F order the points beyond it (a point inside the sphere
// through F and D comes before D), so the lanes' candidates D combine into
// the first one in any order.
__device__ __noinline__ bool across_facet(int3 S, const uint8_t *__restrict__ valid, int64_t cx, int64_t cy, int64_t cz,
                             int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0, int64_t z1, LPt (&T)[4],
                             int kf) {
    const int lane = threadIdx.x & 31;
    const int64_t o = orient(T[0], T[1], T[2], T[3]);
    const int wx = (int)(x1 - x0 + 1), wy = (int)(y1 - y0 + 1), W = wx * wy * (int)(z1 - z0 + 1);
    bool far_pt = false, have = false;
    LPt D = T[(kf + 1) & 3];
    for (WinIter w(wx, wy, lane); w.k < W; w.step()) {
        const int64_t x = x0 + w.x, y = y0 + w.y, z = z0 + w.z;
        const int64_t r = lattice_rank(S, x, y, z);
        if (!valid[r] || T[0].rank == r || T[1].rank == r || T[2].rank == r || T[3].rank == r) continue;
        const LPt p = {x - cx, y - cy, z - cz, r};
        LPt u[4] = {T[0], T[1], T[2], T[3]};
        u[kf] = p;
        const int64_t so = orient(u[0], u[1], u[2], u[3]);
        if (so == 0) continue;
        if ((so > 0) == (o > 0)) { far_pt = true; continue; }
        if (!have) { D = p; have = true; continue; }
        LPt t4[4] = {T[0], T[1], T[2], T[3]};
        t4[kf] = D;
        positive_orientation(t4);
        if (lifted_sign(t4, p) < 0) D = p;
    }
    far_pt = __any_sync(kAll, far_pt);
    for (int off = 16; off > 0; off >>= 1) {
        const LPt Do = shfl_xor_pt(D, off);
        const bool ho = __shfl_xor_sync(kAll, (int)have, off) != 0;
        if (!ho || Do.rank == D.rank) continue;
        if (!have) { D = Do; have = true; continue; }
        LPt t4[4] = {T[0], T[1], T[2], T[3]};
        t4[kf] = D;
        positive_orientation(t4);
        if (lifted_sign(t4, Do) < 0) D = Do;
    }
    if (have) {
        LPt t4[4] = {T[0], T[1], T[2], T[3]};
        t4[kf] = D;
        positive_orientation(t4);
        bool inside = false;
        for (WinIter w(wx, wy, lane); w.k < W && !inside; w.step()) {
            const int64_t x = x0 + w.x, y = y0 + w.y, z = z0 + w.z;
            const int64_t r = lattice_rank(S, x, y, z);
            if (!valid[r] || t4[0].rank == r || t4[1].rank == r || t4[2].rank == r || t4[3].rank == r) continue;
            const LPt p = {x - cx, y - cy, z - cz, r};
            inside = lifted_sign(t4, p) < 0;
        }
        inside = __any_sync(kAll, inside);
        double ctr[3], r2;
        circumsphere(t4, ctr, r2);
        if (!inside && sphere_fits(ctr, r2, S, cx, cy, cz, x0, x1, y0, y1, z0, z1)) {
            T[kf] = D;
            return true;
        }
    }
    // (b): no valid point of the lattice strictly on the far side of F. The
    // orientation with p in place of the starting point is affine in p,
    // n.p + d, so each lattice row holds its far-side points in one interval
    // and only those are visited (within kHullScanWork rows and points).
    if (!far_pt) {
        LPt u[4] = {T[0], T[1], T[2], T[3]};
        const LPt o0 = {0, 0, 0, -1}, ex = {1, 0, 0, -1}, ey = {0, 1, 0, -1}, ez = {0, 0, 1, -1};
        u[kf] = o0;
        const int64_t d = orient(u[0], u[1], u[2], u[3]);
        u[kf] = ex;
        const int64_t nx = orient(u[0], u[1], u[2], u[3]) - d;
        u[kf] = ey;
        const int64_t ny = orient(u[0], u[1], u[2], u[3]) - d;
        u[kf] = ez;
        const int64_t nz = orient(u[0], u[1], u[2], u[3]) - d;
        const int64_t sg = o > 0 ? 1 : -1;
        const int64_t rows = (int64_t)S.y * S.z, budget = kHullScanWork / 32;
        int64_t work = 0;
        bool stop = false;                          // a far-side valid point, or out of budget
        for (int64_t row = lane; row < rows && !stop; row += 32) {
            const int64_t y = (int)row % S.y, z = (int)row / S.y;
            if (++work > budget) { stop = true; break; }
            int64_t t0, t1;
            if (!positive_range(sg * nx, sg * (ny * (y - cy) + nz * (z - cz) + d), -cx, (int64_t)S.x - 1 - cx, t0, t1))
                continue;
            for (int64_t t = t0; t <= t1; ++t) {
                if (++work > budget || valid[lattice_rank(S, t + cx, y, z)]) { stop = true; break; }
            }
        }
        if (__any_sync(kAll, stop)) return false;
        T[kf] = T[(kf + 1) & 3];
        return true;
    }
    return false;
}

// The walk continues from the tetrahedron T it is given (a feasible basis:
// q inside it), so a larger window resumes where a smaller one stopped.
__device__ __noinline__ int walk(int3 S, const uint8_t *__restrict__ valid, int64_t cx, int64_t cy, int64_t cz, int R,
                    LPt (&T)[4], double (&lam)[4]) {
    const int lane = threadIdx.x & 31;
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const LPt q0 = {0, 0, 0, -1};
    const int64_t x0 = max(cx - R, (int64_t)0), x1 = min(cx + R, (int64_t)S.x - 1);
    const int64_t y0 = max(cy - R, (int64_t)0), y1 = min(cy + R, (int64_t)S.y - 1);
    const int64_t z0 = max(cz - R, (int64_t)0), z1 = min(cz + R, (int64_t)S.z - 1);
    const int wx = (int)(x1 - x0 + 1), wy = (int)(y1 - y0 + 1), W = wx * wy * (int)(z1 - z0 + 1);
    for (int it = 0; it < kMaxPivots; ++it) {
        // entering point: the lowest-ranked valid window point inside the
        // circumsphere of T (each lane takes the first of its points in rank
        // order, the warp the least of those). A point clearly outside by
        // its FP32 distance to the centre (circumsphere_f) is skipped. T
        // holds q, so the centre lies within r of q, and near the sphere the
        // squared distance's rounding error stays below 2e-6 r^2: with the
        // margin 1e-4 r^2 + 1e-2 only points strictly outside are skipped;
        // every other point gets the exact predicate, so the choice is the
        // exact one.
        float fc[3], fr2e;
        circumsphere_f(T, fc, fr2e);
        const float fc0 = fc[0], fc1 = fc[1], fc2 = fc[2];
        const float fr2 = fr2e * (1.0f + 1e-4f) + 1e-2f;
        const bool deep = it < kDeepPivots;
        int64_t best = kNone;
        unsigned long long bkey = 0;
        for (WinIter w(wx, wy, lane); w.k < W; w.step()) {
            const int64_t x = x0 + w.x, y = y0 + w.y, z = z0 + w.z;
            const int64_t r = lattice_rank(S, x, y, z);
            if (!valid[r]) continue;
            const float dx = (float)(x - cx) - fc0, dy = (float)(y - cy) - fc1, dz = (float)(z - cz) - fc2;
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 > fr2) continue;
            if (T[0].rank == r || T[1].rank == r || T[2].rank == r || T[3].rank == r) continue;
            const LPt p = {x - cx, y - cy, z - cz, r};
            if (deep) {
                const unsigned long long key = depth_key(fr2e - d2, r);
                if (key > bkey && lifted_sign(T, p) < 0) bkey = key;
            } else if (lifted_sign(T, p) < 0) {
                best = r;
                break;
            }
        }
        if (deep) {
            bkey = warp_max_u64(bkey);
            best = bkey ? (int64_t)(0xffffffffu - (unsigned)(bkey & 0xffffffffu)) : kNone;
        } else {
            best = warp_min(best);
        }
        const int64_t o = orient(T[0], T[1], T[2], T[3]);
        if (best == kNone) {
            // optimal: q's barycentric coordinates in T
            int64_t ol[4];
            int nfar = 0, kf = -1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                LPt u[4] = {T[0], T[1], T[2], T[3]};
                u[k] = q0;
                ol[k] = orient(u[0], u[1], u[2], u[3]);
                lam[k] = (double)ol[k] / (double)o;
                if (T[k].rank >= P) { ++nfar; kf = k; }
            }
            // the circumsphere (FP64) must fit in the window: then no
            // lattice point outside the window is inside it
            if (nfar == 0) {
                double ctr[3], r2;
                circumsphere(T, ctr, r2);
                return sphere_fits(ctr, r2, S, cx, cy, cz, x0, x1, y0, y1, z0, z1) ? 1 : 0;
            }
            // a starting point with weight above 0: q is outside the hull
            // of the window's valid points; with weight 0: q is on a facet
            if (nfar > 1 || ol[kf] != 0) return 0;
            return across_facet(S, valid, cx, cy, cz, x0, x1, y0, y1, z0, z1, T, kf) ? 1 : 0;
        }
        int64_t bc[3];
        rank_coords(S, best, bc);
        const LPt e = {bc[0] - cx, bc[1] - cy, bc[2] - cz, best};
        // ratio test: leaving vertex k minimises lambda_k / d_k over d_k > 0,
        // with lambda_k = O_k(q) / O and d_k = O_k(e) / O (O_k: orientation
        // with vertex k replaced); ties go to the lowest rank
        int leave = -1;
        int64_t bq = 0, be = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            LPt u[4] = {T[0], T[1], T[2], T[3]};
            u[k] = e;
            const int64_t oe = orient(u[0], u[1], u[2], u[3]);   // same sign as o when d_k > 0
            if (!(o > 0 ? oe > 0 : oe < 0)) continue;
            u[k] = q0;
            const int64_t oq = orient(u[0], u[1], u[2], u[3]);
            // compare oq / oe against bq / be (both denominators of o's sign)
            bool better = leave < 0;
            if (!better) {
                // oe and be share o's sign, so oe * be > 0
                const i128 lhs = (i128)oq * be, rhs = (i128)bq * oe;
                better = lhs < rhs || (lhs == rhs && T[k].rank < T[leave].rank);
            }
            if (better) { leave = k; bq = oq; be = oe; }
        }
        if (leave < 0) return 0;   // cannot happen for a point inside the circumsphere
        T[leave] = e;
        positive_orientation(T);
    }
    return 0;
}

// ---- Faces: the same program in a face's two free coordinates ----------

struct LPt2 {
    int64_t u, v;      // free coordinates relative to the query point
    int64_t rank;
};

// Counter-clockwise orientation of (a, b, c): positive when counter-clockwise.
// Coordinates differ by less than 2^12 (as for LPt), so 64 bits are exact.
__device__ __forceinline__ int64_t orient2(const LPt2 &a, const LPt2 &b, const LPt2 &c) {
    return (b.u - a.u) * (c.v - a.v) - (b.v - a.v) * (c.u - a.u);
}

__device__ __noinline__ int perturbed_sign2(const LPt2 (&t)[3], const LPt2 &e);

// Sign of the 4 x 4 determinant with rows (u, v, w, 1) of t0, t1, t2, e under
// the perturbed lifting w = u^2 + v^2 + d_rank: positive when e is inside the
// circumcircle of the counter-clockwise triangle (t0, t1, t2). Translated so
// that e is the origin, the unperturbed part is the 3 x 3 determinant of the
// rows (p - e, |p - e|^2).
__device__ __noinline__ int lifted_sign2(const LPt2 (&t)[3], const LPt2 &e) {
    int64_t r[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        r[i][0] = t[i].u - e.u;
        r[i][1] = t[i].v - e.v;
        r[i][2] = r[i][0] * r[i][0] + r[i][1] * r[i][1];
    }
    const int64_t d0 = det3(r[0][0], r[0][1], r[0][2], r[1][0], r[1][1], r[1][2], r[2][0], r[2][1], r[2][2]);
    if (d0 != 0) return d0 > 0 ? 1 : -1;
    return perturbed_sign2(t, e);
}

// The sign when the unperturbed determinant is zero: the lifted entry of
// point k of (t0, t1, t2, e) has the cofactor (-1)^k orient2(the other three,
// in order); the lowest-ranked point with a non-zero cofactor decides.
__device__ __noinline__ int perturbed_sign2(const LPt2 (&t)[3], const LPt2 &e) {
    const LPt2 *p[4] = {&t[0], &t[1], &t[2], &e};
    bool used[4] = {false, false, false, false};
    for (int round = 0; round < 4; ++round) {
        int k = -1;
        for (int m = 0; m < 4; ++m)
            if (!used[m] && (k < 0 || p[m]->rank < p[k]->rank)) k = m;
        used[k] = true;
        const LPt2 *q[3];
        for (int m = 0, n = 0; m < 4; ++m)
            if (m != k) q[n++] = p[m];
        const int64_t o = orient2(*q[0], *q[1], *q[2]);
        if (o != 0) {
            const int64_t c = (k & 1) ? -o : o;
            return c > 0 ? 1 : -1;
        }
    }
    return 0;
}

// Circumcircle of T (centre and squared radius, FP64), for the filter.
__device__ __noinline__ void circumcircle(const LPt2 (&T)[3], double (&ctr)[2], double &r2) {
    const double bx = (double)(T[1].u - T[0].u), by = (double)(T[1].v - T[0].v);
    const double cx = (double)(T[2].u - T[0].u), cy = (double)(T[2].v - T[0].v);
    const double d = 2.0 * (bx * cy - by * cx);
    const double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    const double ux = (cy * b2 - by * c2) / d, uy = (bx * c2 - cx * b2) / d;
    ctr[0] = ux + (double)T[0].u;
    ctr[1] = uy + (double)T[0].v;
    r2 = ux * ux + uy * uy;
}

// The circumcircle of T for the face walk's filter, as circumsphere_f:
// exact 64-bit Cramer numerators, FP32 quotients.
__device__ __forceinline__ void circumcircle_f(const LPt2 (&T)[3], float (&c)[2], float &r2) {
    const int64_t bx = T[1].u - T[0].u, by = T[1].v - T[0].v, cx = T[2].u - T[0].u, cy = T[2].v - T[0].v;
    const int64_t b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    const float d = (float)(2 * (bx * cy - by * cx));
    const float ux = (float)(cy * b2 - by * c2) / d, uy = (float)(bx * c2 - cx * b2) / d;
    c[0] = ux + (float)T[0].u;
    c[1] = uy + (float)T[0].v;
    r2 = ux * ux + uy * uy;
}

// Sets T to three far starting points around q (counter-clockwise).
__device__ void start_triangle(int64_t P, LPt2 (&T)[3]) {
    const int64_t far[3][2] = {{kFar, 0}, {-kFar, kFar}, {-kFar, -kFar}};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T[k].u = far[k][0]; T[k].v = far[k][1];
        T[k].rank = P + k;
    }
    if (orient2(T[0], T[1], T[2]) < 0) { const LPt2 s = T[0]; T[0] = T[1]; T[1] = s; }
}

// The face version of sphere_fits: the circle centred at ctr (free
// coordinates relative to c) with squared radius r2 stays clear of the
// lattice lines just outside the window [u0, u1] x [v0, v1] of the face.
__device__ bool circle_fits(const double (&ctr)[2], double r2, int3 S, const int64_t (&c)[3], int a, int b,
                            int64_t u0, int64_t u1, int64_t v0, int64_t v1) {
    const int64_t ext[3] = {S.x, S.y, S.z};
    const double rad = sqrt(r2) * (1.0 + 1e-12) + 1e-9;
    const int ax[2] = {a, b};
    const int64_t lo[2] = {u0 - c[a], v0 - c[b]}, hi[2] = {u1 - c[a], v1 - c[b]};
    for (int m = 0; m < 2; ++m) {
        const int64_t cm = c[ax[m]];
        if (cm + lo[m] > 0 && ctr[m] - rad <= (double)lo[m] - 1.0) return false;
        if (cm + hi[m] < ext[ax[m]] - 1 && ctr[m] + rad >= (double)hi[m] + 1.0) return false;
    }
    return true;
}

// across_facet on a face: q lies on the edge F opposite the starting point
// T[kf] (weight exactly 0). Wrap across F to the valid window point D whose
// circle through F holds no other point on that side; accept when that
// triangle's circle holds no valid window point and fits in the window, or
// when no valid point of the face lies strictly on the far side of F (F is
// then on the hull of the face's points).
__device__ __noinline__ bool across_edge(int3 S, const uint8_t *__restrict__ valid, const int64_t (&c)[3], int a, int b,
                            int64_t u0, int64_t u1, int64_t v0, int64_t v1, LPt2 (&T)[3], int kf) {
    const int lane = threadIdx.x & 31;
    const int64_t ext[3] = {S.x, S.y, S.z};
    const LPt2 A = T[(kf + 1) % 3], B = T[(kf + 2) % 3];
    const int64_t sf = orient2(A, B, T[kf]);
    const int wu = (int)(u1 - u0 + 1), W = wu * (int)(v1 - v0 + 1);
    bool far_pt = false, have = false;
    LPt2 D = A;
    for (WinIter w(wu, 1 << 30, lane); w.k < W; w.step()) {
        int64_t pc[3] = {c[0], c[1], c[2]};
        pc[a] = u0 + w.x;
        pc[b] = v0 + w.y;
        const int64_t r = lattice_rank(S, pc[0], pc[1], pc[2]);
        if (!valid[r] || r == A.rank || r == B.rank) continue;
        const LPt2 p = {pc[a] - c[a], pc[b] - c[b], r};
        const int64_t so = orient2(A, B, p);
        if (so == 0) continue;
        if ((so > 0) == (sf > 0)) { far_pt = true; continue; }
        if (!have) { D = p; have = true; continue; }
        LPt2 t3[3] = {A, B, D};
        if (orient2(t3[0], t3[1], t3[2]) < 0) { const LPt2 sw = t3[0]; t3[0] = t3[1]; t3[1] = sw; }
        if (lifted_sign2(t3, p) > 0) D = p;
    }
    far_pt = __any_sync(kAll, far_pt);
    for (int off = 16; off > 0; off >>= 1) {
        LPt2 Do;
        Do.u = __shfl_xor_sync(kAll, (long long)D.u, off);
        Do.v = __shfl_xor_sync(kAll, (long long)D.v, off);
        Do.rank = __shfl_xor_sync(kAll, (long long)D.rank, off);
        const bool ho = __shfl_xor_sync(kAll, (int)have, off) != 0;
        if (!ho || Do.rank == D.rank) continue;
        if (!have) { D = Do; have = true; continue; }
        LPt2 t3[3] = {A, B, D};
        if (orient2(t3[0], t3[1], t3[2]) < 0) { const LPt2 sw = t3[0]; t3[0] = t3[1]; t3[1] = sw; }
        if (lifted_sign2(t3, Do) > 0) D = Do;
    }
    if (have) {
        LPt2 t3[3] = {A, B, D};
        if (orient2(t3[0], t3[1], t3[2]) < 0) { const LPt2 sw = t3[0]; t3[0] = t3[1]; t3[1] = sw; }
        bool inside = false;
        for (WinIter w(wu, 1 << 30, lane); w.k < W && !inside; w.step()) {
            int64_t pc[3] = {c[0], c[1], c[2]};
            pc[a] = u0 + w.x;
            pc[b] = v0 + w.y;
            const int64_t r = lattice_rank(S, pc[0], pc[1], pc[2]);
            if (!valid[r] || r == A.rank || r == B.rank || r == D.rank) continue;
            const LPt2 p = {pc[a] - c[a], pc[b] - c[b], r};
            inside = lifted_sign2(t3, p) > 0;
        }
        inside = __any_sync(kAll, inside);
        double ctr[2], r2;
        circumcircle(t3, ctr, r2);
        if (!inside && circle_fits(ctr, r2, S, c, a, b, u0, u1, v0, v1)) {
            T[kf] = D;
            return true;
        }
    }
    // no valid point of the face strictly on the far side of F, visiting
    // only the far-side interval of each row (orient2(A, B, p) is affine in
    // p), within kHullScanWork rows and points
    if (!far_pt) {
        const LPt2 o0 = {0, 0, -1}, eu = {1, 0, -1}, ev = {0, 1, -1};
        const int64_t d = orient2(A, B, o0);
        const int64_t nu = orient2(A, B, eu) - d, nv = orient2(A, B, ev) - d;
        const int64_t sg = sf > 0 ? 1 : -1;
        const int64_t budget = kHullScanWork / 32;
        int64_t work = 0;
        bool stop = false;
        for (int64_t vv = lane; vv < ext[b] && !stop; vv += 32) {
            if (++work > budget) { stop = true; break; }
            int64_t t0, t1;
            if (!positive_range(sg * nu, sg * (nv * (vv - c[b]) + d), -c[a], ext[a] - 1 - c[a], t0, t1)) continue;
            for (int64_t t = t0; t <= t1; ++t) {
                int64_t pc[3] = {c[0], c[1], c[2]};
                pc[a] = t + c[a];
                pc[b] = vv;
                if (++work > budget || valid[lattice_rank(S, pc[0], pc[1], pc[2])]) { stop = true; break; }
            }
        }
        if (__any_sync(kAll, stop)) return false;
        T[kf] = A;
        return true;
    }
    return false;
}

// The walk of `walk` on the face through c whose free axes are a < b: the
// window is the square of radius R around c on that face, its points in
// rank order (axis a fastest). Returns 1 with the triangle and q's
// barycentric coordinates, or 0.
__device__ __noinline__ int walk2(int3 S, const uint8_t *__restrict__ valid, const int64_t (&c)[3], int a, int b, int R,
                     LPt2 (&T)[3], double (&lam)[3]) {
    const int lane = threadIdx.x & 31;
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const int64_t ext[3] = {S.x, S.y, S.z};
    const LPt2 q0 = {0, 0, -1};
    const int64_t u0 = max(c[a] - R, (int64_t)0), u1 = min(c[a] + R, ext[a] - 1);
    const int64_t v0 = max(c[b] - R, (int64_t)0), v1 = min(c[b] + R, ext[b] - 1);
    const int wu = (int)(u1 - u0 + 1), W = wu * (int)(v1 - v0 + 1);
    for (int it = 0; it < kMaxPivots; ++it) {
        float fc[2], fr2e;
        circumcircle_f(T, fc, fr2e);
        const float fc0 = fc[0], fc1 = fc[1];
        const float fr2 = fr2e * (1.0f + 1e-4f) + 1e-2f;   // as in walk
        const bool deep = it < kDeepPivots;   // the pivot rule of walk
        int64_t best = kNone;
        unsigned long long bkey = 0;
        for (WinIter w(wu, 1 << 30, lane); w.k < W; w.step()) {
            int64_t pc[3] = {c[0], c[1], c[2]};
            pc[a] = u0 + w.x;
            pc[b] = v0 + w.y;
            const int64_t r = lattice_rank(S, pc[0], pc[1], pc[2]);
            if (!valid[r]) continue;
            const float du = (float)(pc[a] - c[a]) - fc0, dv = (float)(pc[b] - c[b]) - fc1;
            const float d2 = du * du + dv * dv;
            if (d2 > fr2) continue;
            if (T[0].rank == r || T[1].rank == r || T[2].rank == r) continue;
            const LPt2 cand = {pc[a] - c[a], pc[b] - c[b], r};
            if (deep) {
                const unsigned long long key = depth_key(fr2e - d2, r);
                if (key > bkey && lifted_sign2(T, cand) > 0) bkey = key;
            } else if (lifted_sign2(T, cand) > 0) {
                best = r;
                break;
            }
        }
        if (deep) {
            bkey = warp_max_u64(bkey);
            best = bkey ? (int64_t)(0xffffffffu - (unsigned)(bkey & 0xffffffffu)) : kNone;
        } else {
            best = warp_min(best);
        }
        const int64_t o = orient2(T[0], T[1], T[2]);   // > 0: T is kept counter-clockwise
        if (best == kNone) {
            int64_t ol[3];
            int nfar = 0, kf = -1;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                LPt2 u[3] = {T[0], T[1], T[2]};
                u[k] = q0;
                ol[k] = orient2(u[0], u[1], u[2]);
                lam[k] = (double)ol[k] / (double)o;
                if (T[k].rank >= P) { ++nfar; kf = k; }
            }
            if (nfar == 0) {
                double ctr[2], r2;
                circumcircle(T, ctr, r2);
                return circle_fits(ctr, r2, S, c, a, b, u0, u1, v0, v1) ? 1 : 0;
            }
            if (nfar > 1 || ol[kf] != 0) return 0;
            return across_edge(S, valid, c, a, b, u0, u1, v0, v1, T, kf) ? 1 : 0;
        }
        int64_t bc[3];
        rank_coords(S, best, bc);
        const LPt2 e = {bc[a] - c[a], bc[b] - c[b], best};
        int leave = -1;
        int64_t bq = 0, be = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            LPt2 u[3] = {T[0], T[1], T[2]};
            u[k] = e;
            const int64_t oe = orient2(u[0], u[1], u[2]);
            if (oe <= 0) continue;
            u[k] = q0;
            const int64_t oq = orient2(u[0], u[1], u[2]);
            bool better = leave < 0;
            if (!better) {
                const int64_t lhs = oq * be, rhs = bq * oe;   // below 2^50
                better = lhs < rhs || (lhs == rhs && T[k].rank < T[leave].rank);
            }
            if (better) { leave = k; bq = oq; be = oe; }
        }
        if (leave < 0) return 0;
        T[leave] = e;
        if (orient2(T[0], T[1], T[2]) < 0) { const LPt2 s = T[0]; T[0] = T[1]; T[1] = s; }
    }
    return 0;
}

// ---- Edges: nearest valid neighbours along the free axis a --------------
__device__ __noinline__ int edge_interp(int3 S, const uint8_t *__restrict__ valid, const int64_t (&c)[3], int a,
                           int64_t (&vtx)[4], double (&lam)[4]) {
    const int lane = threadIdx.x & 31;
    const int64_t ext[3] = {S.x, S.y, S.z};
    int64_t pc[3] = {c[0], c[1], c[2]};
    int64_t lo = -1, hi = kNone;
    for (int64_t t = c[a] - 1 - lane; t >= 0; t -= 32) {
        pc[a] = t;
        if (valid[lattice_rank(S, pc[0], pc[1], pc[2])]) { lo = t; break; }
    }
    for (int64_t t = c[a] + 1 + lane; t < ext[a]; t += 32) {
        pc[a] = t;
        if (valid[lattice_rank(S, pc[0], pc[1], pc[2])]) { hi = t; break; }
    }
    lo = warp_max(lo);
    hi = warp_min(hi);
    if (lo < 0 || hi == kNone) return 0;
    pc[a] = lo;
    vtx[0] = lattice_rank(S, pc[0], pc[1], pc[2]);
    pc[a] = hi;
    vtx[1] = lattice_rank(S, pc[0], pc[1], pc[2]);
    lam[0] = (double)(hi - c[a]) / (double)(hi - lo);
    lam[1] = (double)(c[a] - lo) / (double)(hi - lo);
    return 1;
}

// The missing entry p, solved by the whole warp: the barycentric
// interpolant over its Delaunay simplex (status 2), or missing (NaN,
// status 0); lane 0 writes it.
__device__ void solve_entry(int3 S, int64_t p, const float *__restrict__ ends, const uint8_t *__restrict__ valid,
                            float *__restrict__ out, uint8_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t P = (int64_t)S.x * S.y * S.z;
    int64_t c[3];
    rank_coords(S, p, c);
    const int64_t cx = c[0], cy = c[1], cz = c[2];
    const bool fixed[3] = {cx == 0 || cx == S.x - 1, cy == 0 || cy == S.y - 1, cz == 0 || cz == S.z - 1};
    const int nfix = (int)fixed[0] + (int)fixed[1] + (int)fixed[2];
    const bool flat = S.x == 1 || S.y == 1 || S.z == 1;
    int64_t vtx[4] = {-1, -1, -1, -1};
    double lam[4] = {0.0, 0.0, 0.0, 0.0};
    int nv = 0, ok = 0;
    if (flat || nfix == 3) {
        ok = 0;                                   // no tetrahedra, or a corner
    } else if (nfix == 0) {
        LPt T[4];
        start_tetrahedron(P, T);
        for (int R = 2; R <= kMaxWindow && !ok; ++R) ok = walk(S, valid, cx, cy, cz, R, T, lam);
        for (int k = 0; k < 4; ++k) vtx[k] = T[k].rank;
        nv = 4;
    } else if (nfix == 1) {
        const int a = fixed[0] ? 1 : 0, b = fixed[2] ? 1 : 2;
        LPt2 T2[3];
        double l2[3];
        start_triangle(P, T2);
        for (int R = 2; R <= kMaxWindow2 && !ok; ++R) ok = walk2(S, valid, c, a, b, R, T2, l2);
        for (int k = 0; k < 3; ++k) { vtx[k] = T2[k].rank; lam[k] = l2[k]; }
        nv = 3;
    } else {
        const int a = !fixed[0] ? 0 : (!fixed[1] ? 1 : 2);
        ok = edge_interp(S, valid, c, a, vtx, lam);
        nv = 2;
    }
    if (lane != 0) return;
    if (ok != 1) {
        const float nan = __int_as_float(0x7fc00000);
        out[3 * p] = nan; out[3 * p + 1] = nan; out[3 * p + 2] = nan;
        if (status) status[p] = 0;
        return;
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < nv; ++k) {
        const int64_t v = vtx[k];
        if (v < 0 || v >= P) {   // never: both walks reject starting points
            (void)BTO_IN_BOUNDS(false, nullptr);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] += lam[k] * (double)ends[3 * v + d];
    }
    out[3 * p] = (float)acc[0]; out[3 * p + 1] = (float)acc[1]; out[3 * p + 2] = (float)acc[2];
    if (status) status[p] = 2;
}

constexpr int kFillThreads = 128;

// Each warp takes chunks of 32 lattice points (grid-stride): valid entries
// are copied (status 1) by their lanes, and the warp then solves the
// chunk's missing entries one after another, all lanes on each.
__global__ void __launch_bounds__(kFillThreads) fill_delaunay_kernel(int3 S, const float *__restrict__ ends,
                                                                     const uint8_t *__restrict__ valid,
                                                                     float *__restrict__ out,
                                                                     uint8_t *__restrict__ status) {
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < P; base += nwarps * 32) {
        const int64_t p = base + lane;
        bool miss = false;
        if (p < P) {
            if (valid[p]) {
                out[3 * p] = ends[3 * p]; out[3 * p + 1] = ends[3 * p + 1]; out[3 * p + 2] = ends[3 * p + 2];
                if (status) status[p] = 1;
            } else {
                miss = true;
            }
        }
        unsigned m = __ballot_sync(kAll, miss);
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            solve_entry(S, base + bit, ends, valid, out, status);
        }
    }
}

}  // namespace

BTO_BOUNDS_ACCESSOR(bounds_failures_delaunay)

cudaError_t launch_fill_delaunay(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                 uint8_t *status, int grid, cudaStream_t s) {
    fill_delaunay_kernel<<<grid, kFillThreads, 0, s>>>(make_int3(S[0], S[1], S[2]), ends, valid, out, status);
    return cudaGetLastError();
}

}  // namespace bto
