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
// Each thread solves this program for one missing lattice point by the
// simplex method over the valid points of a window around it: the basis is
// a tetrahedron holding q; a point inside the tetrahedron's circumsphere
// (below the plane through its lifted vertices) has a negative reduced
// cost and enters; the ratio test picks the vertex that leaves so that q
// stays inside. It starts from four far points around q and stops when no
// window point lies inside the circumsphere. The result is the Delaunay
// tetrahedron of all valid points when its circumsphere fits in the window
// (no lattice point outside the window can then lie inside it); otherwise
// the window grows (radius 2 to 6 lattice units) and the walk restarts.
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

__device__ int perturbed_sign(const LPt (&t)[4], const LPt &e);

// Sign of the 5 x 5 determinant with rows (x, y, z, w, 1) of t0..t3, e
// under the perturbed lifting: negative when e is inside the circumsphere of
// the positively oriented tetrahedron (t0, t1, t2, t3).
__device__ int lifted_sign(const LPt (&t)[4], const LPt &e) {
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
constexpr int kMaxWindow = 6;      // largest window radius, lattice units

// Outcome of one walk in a window of radius R around the lattice point c:
// 1 and the tetrahedron with q's barycentric coordinates, or 0 (no result
// in this window: q outside the hull of its valid points, circumsphere
// larger than the window, or the pivot limit).
// Circumsphere of T (centre and squared radius, FP64), for the filter that
// spares most points the exact predicate.
__device__ void circumsphere(const LPt (&T)[4], double (&ctr)[3], double &r2) {
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

// The walk continues from the tetrahedron T it is given (a feasible basis:
// q inside it), so a larger window resumes where a smaller one stopped.
__device__ int walk(int3 S, const uint8_t *__restrict__ valid, int64_t cx, int64_t cy, int64_t cz, int R,
                    LPt (&T)[4], double (&lam)[4]) {
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const LPt q0 = {0, 0, 0, -1};
    const int64_t x0 = max(cx - R, (int64_t)0), x1 = min(cx + R, (int64_t)S.x - 1);
    const int64_t y0 = max(cy - R, (int64_t)0), y1 = min(cy + R, (int64_t)S.y - 1);
    const int64_t z0 = max(cz - R, (int64_t)0), z1 = min(cz + R, (int64_t)S.z - 1);
    for (int it = 0; it < kMaxPivots; ++it) {
        // entering point: the lowest-ranked valid window point inside the
        // circumsphere of T (points are visited in rank order). A point
        // clearly outside by the FP64 distance to the centre (margin far
        // above its rounding error) is skipped; every other point gets the
        // exact predicate, so the choice is the exact one.
        double ctr[3], r2;
        circumsphere(T, ctr, r2);
        const double tol = 1e-9 * (r2 + 1.0);
        LPt e;
        bool found = false;
        for (int64_t z = z0; z <= z1 && !found; ++z)
            for (int64_t y = y0; y <= y1 && !found; ++y)
                for (int64_t x = x0; x <= x1 && !found; ++x) {
                    if (!valid[lattice_rank(S, x, y, z)]) continue;
                    const double dx = (double)(x - cx) - ctr[0], dy = (double)(y - cy) - ctr[1],
                                 dz = (double)(z - cz) - ctr[2];
                    if (dx * dx + dy * dy + dz * dz > r2 + tol) continue;
                    const LPt c = {x - cx, y - cy, z - cz, lattice_rank(S, x, y, z)};
                    bool inT = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) inT |= T[k].rank == c.rank;
                    if (inT) continue;
                    if (lifted_sign(T, c) < 0) { e = c; found = true; }
                }
        const int64_t o = orient(T[0], T[1], T[2], T[3]);
        if (!found) {
            // optimal: q's barycentric coordinates in T; a starting point
            // may stay only with weight exactly 0 (q on the opposite face)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                LPt u[4] = {T[0], T[1], T[2], T[3]};
                u[k] = q0;
                const int64_t ok = orient(u[0], u[1], u[2], u[3]);
                if (T[k].rank >= P && ok != 0) return 0;
                lam[k] = (double)ok / (double)o;
            }
            // the circumsphere must fit in the window: then no lattice
            // point outside the window is inside it
            if (T[0].rank >= P || T[1].rank >= P || T[2].rank >= P || T[3].rank >= P) return 1;
            const double rad = sqrt(r2) * (1.0 + 1e-12) + 1e-9;
            const double lo[3] = {(double)(x0 - cx), (double)(y0 - cy), (double)(z0 - cz)};
            const double hi[3] = {(double)(x1 - cx), (double)(y1 - cy), (double)(z1 - cz)};
            const int64_t ext[3] = {S.x, S.y, S.z};
            const int64_t cc[3] = {cx, cy, cz};
            for (int m = 0; m < 3; ++m) {
                // a window edge on the lattice boundary needs no margin
                if (cc[m] + (int64_t)lo[m] > 0 && ctr[m] - rad <= lo[m] - 1.0) return 0;
                if (cc[m] + (int64_t)hi[m] < ext[m] - 1 && ctr[m] + rad >= hi[m] + 1.0) return 0;
            }
            return 1;
        }
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
        if (orient(T[0], T[1], T[2], T[3]) < 0) { const LPt s = T[0]; T[0] = T[1]; T[1] = s; }
    }
    return 0;
}

// One thread per lattice point: valid entries are copied (status 1),
// missing ones take the barycentric interpolant over their Delaunay
// tetrahedron (status 2) or stay missing (NaN, status 0).
__global__ void fill_delaunay_kernel(int3 S, const float *__restrict__ ends, const uint8_t *__restrict__ valid,
                                     float *__restrict__ out, uint8_t *__restrict__ status) {
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
        if (valid[p]) {
            out[3 * p] = ends[3 * p]; out[3 * p + 1] = ends[3 * p + 1]; out[3 * p + 2] = ends[3 * p + 2];
            if (status) status[p] = 1;
            continue;
        }
        const int64_t cx = p % S.x, cy = (p / S.x) % S.y, cz = p / ((int64_t)S.x * S.y);
        LPt T[4];
        double lam[4];
        int ok = 0;
        // entries on the lattice's boundary faces have neighbours on one side
        // only and stay missing
        const bool interior = cx > 0 && cy > 0 && cz > 0 && cx < S.x - 1 && cy < S.y - 1 && cz < S.z - 1;
        if (!interior) ok = -1;
        start_tetrahedron(P, T);
        for (int R = 2; R <= kMaxWindow && !ok; ++R) ok = walk(S, valid, cx, cy, cz, R, T, lam);
        if (ok != 1) {
            const float nan = __int_as_float(0x7fc00000);
            out[3 * p] = nan; out[3 * p + 1] = nan; out[3 * p + 2] = nan;
            if (status) status[p] = 0;
            continue;
        }
        double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t v = T[k].rank;
            if (v >= P) continue;   // a starting point with weight 0
            if (!BTO_IN_BOUNDS(v >= 0, nullptr)) continue;
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[d] += lam[k] * (double)ends[3 * v + d];
        }
        out[3 * p] = (float)acc[0]; out[3 * p + 1] = (float)acc[1]; out[3 * p + 2] = (float)acc[2];
        if (status) status[p] = 2;
    }
}

}  // namespace

BTO_BOUNDS_ACCESSOR(bounds_failures_delaunay)

cudaError_t launch_fill_delaunay(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                 uint8_t *status, int grid, cudaStream_t s) {
    fill_delaunay_kernel<<<grid, 128, 0, s>>>(make_int3(S[0], S[1], S[2]), ends, valid, out, status);
    return cudaGetLastError();
}

}  // namespace bto
