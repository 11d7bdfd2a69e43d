/*
 * bto_oracle.c -- plain FP64 CPU oracle for Boundary Termination Optimization
 * (BTO) Lagrangian flow-map extraction (Sane, Yenpure, Bujack, Larsen,
 * Moreland, Garth, Childs: "Scalable In Situ Lagrangian Flow Map Extraction:
 * Demonstrating the Viability of a Communication-Free Model").
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it. It shares no source, header, table or helper with the CUDA library, and
 * neither side includes or links the other.
 *
 * What it computes, in the paper's order (Sec. 3.1, "In Situ Extraction Using
 * BTO", and Sec. 2.3 on the Agranovsky et al. method it modifies):
 *   - particles are seeded on a uniform lattice at the start of an interval
 *     (Sec. 2.3: seeded along a uniform grid; a 1:X reduction places one
 *     particle per X grid points);
 *   - every cycle each particle still alive advances by one RK4 step through
 *     the velocity field of that cycle only (Sec. 3.1: RK4 advection;
 *     Sec. 2.2: only one time step is resident, and a particle advances by a
 *     single step before the field changes);
 *   - the velocity at a point is the trilinear interpolant of the 8 corner
 *     nodes of its cell: Eq. (1) applied per axis and per component
 *     (Sec. 3.3, Eq. linearInterpolation and the sentence after it);
 *   - a particle that reaches the block boundary during the interval is
 *     terminated and its trajectory discarded, i.e. flagged invalid
 *     (Sec. 3.1; Sec. 3.3 first paragraph after Eq. 1);
 *   - at the end of the interval the basis flows (seed, end, valid) are
 *     written (Sec. 2.3).
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes of the repository):
 *   R1 trilinear = tensor product of Eq. (1);
 *   R2 all four RK4 stages use the field of the current cycle;
 *   R3 the block is the CLOSED box [origin, origin + n*h]; the stage points
 *      p2, p3, p4 and the end point x' are tested in that order and the first
 *      one outside terminates the particle (a point outside cannot be sampled
 *      because the neighbour's data are not resident);
 *   R4 a terminated particle keeps its last in-block position (the position
 *      before the failing step) and records the cycle index of that step;
 *   R5 n cells per axis, n+1 nodes, seeds at node indices j*s for
 *      j = 0 .. ceil(n/s)-1 (upper faces belong to the neighbour);
 *   R6 the cell index is clamp(floor(xi), 0, n-1).
 *
 * Arithmetic is IEEE double; build with -ffp-contract=off so that x86 and
 * Arm hosts produce identical results.
 *
 * Field layout: float32, (n0+1)*(n1+1)*(n2+1) nodes, 3 components per node
 * (AoS), x index fastest. Positions are physical coordinates.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------------------
 * Seeds (Sec. 2.3 "seeded along a uniform grid"; reading R5).
 * Lattice counts S_a = ceil(n_a / s); canonical index p = jx + Sx*(jy + Sy*jz).
 * ------------------------------------------------------------------------- */
ORACLE_API int64_t bto_oracle_num_seeds(const int64_t n[3], int64_t s)
{
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) total *= (n[a] + s - 1) / s;
    return total;
}

ORACLE_API void bto_oracle_seeds(const int64_t n[3], const double origin[3],
                                 const double h[3], int64_t s,
                                 int64_t m, const int64_t *ids, double *out)
{
    int64_t S[3];
    for (int a = 0; a < 3; ++a) S[a] = (n[a] + s - 1) / s;
    for (int64_t q = 0; q < m; ++q) {
        int64_t p = ids ? ids[q] : q;
        int64_t j[3];
        j[0] = p % S[0];
        j[1] = (p / S[0]) % S[1];
        j[2] = p / (S[0] * S[1]);
        for (int a = 0; a < 3; ++a)
            out[3 * q + a] = origin[a] + (double)(j[a] * s) * h[a];
    }
}

/* ---------------------------------------------------------------------------
 * Velocity at a point: Eq. (1) per axis and component (reading R1, R6).
 * Eq. (1) with t = (x - x0)/(x1 - x0) gives the weights (1 - t) on f(x0) and
 * t on f(x1); the tensor product over the three axes weights corner
 * (i+a, j+b, k+c) by w_a(tx) * w_b(ty) * w_c(tz).
 * ------------------------------------------------------------------------- */
static void sample(const float *field, const int64_t n[3], const double origin[3],
                   const double h[3], const double q[3], double v[3])
{
    int64_t cell[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double xi = (q[a] - origin[a]) / h[a];
        int64_t i = (int64_t)floor(xi);
        if (i < 0) i = 0;
        if (i > n[a] - 1) i = n[a] - 1;
        cell[a] = i;
        t[a] = xi - (double)i;
    }
    const int64_t nx = n[0] + 1, ny = n[1] + 1;
    v[0] = v[1] = v[2] = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                double w = (a ? t[0] : 1.0 - t[0]) *
                           (b ? t[1] : 1.0 - t[1]) *
                           (c ? t[2] : 1.0 - t[2]);
                size_t node = (size_t)(cell[0] + a) +
                              (size_t)nx * ((size_t)(cell[1] + b) +
                                            (size_t)ny * (size_t)(cell[2] + c));
                const float *f = field + 3 * node;
                v[0] += w * (double)f[0];
                v[1] += w * (double)f[1];
                v[2] += w * (double)f[2];
            }
}

ORACLE_API void bto_oracle_sample(const float *field, const int64_t n[3],
                                  const double origin[3], const double h[3],
                                  int64_t m, const double *q, double *v)
{
    for (int64_t i = 0; i < m; ++i) sample(field, n, origin, h, q + 3 * i, v + 3 * i);
}

/* Signed distance, in cells, from q to the nearest face of the closed box:
 * min over axes of min(xi, n - xi). Negative outside. Reading R3: the point
 * is inside iff every xi lies in [0, n]. */
static double margin_cells(const int64_t n[3], const double origin[3],
                           const double h[3], const double q[3], int *inside)
{
    double m = INFINITY;
    int in = 1;
    for (int a = 0; a < 3; ++a) {
        double xi = (q[a] - origin[a]) / h[a];
        if (!(xi >= 0.0 && xi <= (double)n[a])) in = 0;
        double d = xi < (double)n[a] - xi ? xi : (double)n[a] - xi;
        if (d < m) m = d;
    }
    *inside = in;
    return m;
}

/* ---------------------------------------------------------------------------
 * One cycle (Sec. 3.1, readings R2-R4): every live particle takes one RK4
 * step through `field`.
 *   k1 = v(x)
 *   p2 = x + dt/2 k1   -> tested, k2 = v(p2)
 *   p3 = x + dt/2 k2   -> tested, k3 = v(p3)
 *   p4 = x + dt   k3   -> tested, k4 = v(p4)
 *   x' = x + dt/6 (k1 + 2 k2 + 2 k3 + k4) -> tested
 * On the first failing test: exit_cycle = cycle, x unchanged, and (when the
 * arrays are given) exit_pos / exit_time receive the clipped exit location.
 * min_margin[p] keeps the smallest |margin| (cells) over the tested points,
 * which the parity check uses for its near-face exemption.
 * x: m*3 doubles (in/out); exit_cycle: m ints, -1 while alive (in/out);
 * min_margin: m doubles (in/out), start at +inf.
 * exit_pos: m*3 doubles or NULL; exit_time: m doubles or NULL (outputs).
 * ------------------------------------------------------------------------- */
/* Termination location (storing it is the paper's future work, Sec. 6;
 * reading of this library): the chord from the last in-block position x to
 * the first tested point q found outside is clipped to the closed box,
 * t = largest value in [0, 1] with x + t (q - x) inside; the exit time is
 * cycle + t * f, f = 1/2 when q was p2 or p3, 1 for p4 or the end point. A q
 * with a NaN component gives no direction: location x, t = 0. */
static void clip_exit(const int64_t n[3], const double origin[3], const double h[3],
                      const double x[3], const double q[3], double f, int32_t cycle,
                      double *pos, double *time)
{
    if (isnan(q[0]) || isnan(q[1]) || isnan(q[2])) {
        for (int a = 0; a < 3; ++a) pos[a] = x[a];
        *time = (double)cycle;
        return;
    }
    double t = 1.0;
    for (int a = 0; a < 3; ++a) {
        double xi = (x[a] - origin[a]) / h[a], qi = (q[a] - origin[a]) / h[a];
        if (qi > (double)n[a]) { double ta = ((double)n[a] - xi) / (qi - xi); if (ta < t) t = ta; }
        if (qi < 0.0) { double ta = (0.0 - xi) / (qi - xi); if (ta < t) t = ta; }
    }
    if (t < 0.0) t = 0.0;
    for (int a = 0; a < 3; ++a) {
        double lo = origin[a], hi = origin[a] + (double)n[a] * h[a];
        double v = x[a] + t * (q[a] - x[a]);
        pos[a] = v < lo ? lo : (v > hi ? hi : v);
    }
    *time = (double)cycle + t * f;
}

ORACLE_API void bto_oracle_cycle(const float *field, const int64_t n[3],
                                 const double origin[3], const double h[3],
                                 double dt, int32_t cycle, int64_t m,
                                 double *x, int32_t *exit_cycle,
                                 double *min_margin, double *exit_pos, double *exit_time,
                                 int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t p = 0; p < m; ++p) {
        if (exit_cycle[p] >= 0) continue;
        double *xp = x + 3 * p;
        double k1[3], k2[3], k3[3], k4[3], q[3];
        double mm = min_margin[p];
        double f = 0.0;
        int in;
        double d;

        sample(field, n, origin, h, xp, k1);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + 0.5 * dt * k1[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { f = 0.5; goto terminated; }
        sample(field, n, origin, h, q, k2);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + 0.5 * dt * k2[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { f = 0.5; goto terminated; }
        sample(field, n, origin, h, q, k3);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + dt * k3[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { f = 1.0; goto terminated; }
        sample(field, n, origin, h, q, k4);

        for (int a = 0; a < 3; ++a)
            q[a] = xp[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { f = 1.0; goto terminated; }
        min_margin[p] = mm;
        for (int a = 0; a < 3; ++a) xp[a] = q[a];
        continue;
    terminated:
        min_margin[p] = mm;
        exit_cycle[p] = cycle;
        if (exit_pos && exit_time) clip_exit(n, origin, h, xp, q, f, cycle, exit_pos + 3 * p, exit_time + p);
    }
}

/* ---------------------------------------------------------------------------
 * Discrete adjoint of one cycle (reverse mode through the steps of
 * bto_oracle_cycle), for the gradient of a loss on end positions with
 * respect to seeds and node velocities. Termination is a discrete decision:
 * a particle whose step of this cycle was taken (alive[p] = 1) passes its
 * gradient back through that step; the others are left unchanged.
 *
 * Velocity and its derivative at q: with t = (q - origin)/h - i per axis,
 * v = sum_corners w(t) F_corner and dv/dq_b = sum_corners (dw/dt_b) F / h_b,
 * where w = w_a(tx) w_b(ty) w_c(tz) (Eq. 1 per axis) and dw_a/dt = +1 for
 * the upper corner, -1 for the lower.
 *
 * Reverse of  x' = x + dt/6 (k1 + 2 k2 + 2 k3 + k4),
 *             k1 = v(x), k2 = v(x + dt/2 k1), k3 = v(x + dt/2 k2),
 *             k4 = v(x + dt k3),
 * given lam = dL/dx':  g1 = dt/6 lam, g2 = g3 = dt/3 lam, g4 = dt/6 lam,
 * then for stage 4, 3, 2: qbar = (dv/dq)^T g_s; lam_x += qbar; the stage
 * before receives (dt or dt/2) qbar; stage 1 adds (dv/dx)^T g1 to lam_x.
 * Each stage also adds w(q) g_s to the gradient of its 8 corner nodes.
 *   x      m*3 positions at the START of the cycle
 *   alive  m flags: 1 = the step of this cycle was taken
 *   lam    m*3, in: dL/dx after the cycle, out: dL/dx before it
 *   gF     NULL or nodes*3 doubles, accumulated (+=)
 * ------------------------------------------------------------------------- */
static void sample_jac(const float *field, const int64_t n[3], const double origin[3],
                       const double h[3], const double q[3], double v[3], double J[3][3],
                       size_t nodes_out[8], double w_out[8])
{
    int64_t cell[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double xi = (q[a] - origin[a]) / h[a];
        int64_t i = (int64_t)floor(xi);
        if (i < 0) i = 0;
        if (i > n[a] - 1) i = n[a] - 1;
        cell[a] = i;
        t[a] = xi - (double)i;
    }
    const int64_t nx = n[0] + 1, ny = n[1] + 1;
    for (int a = 0; a < 3; ++a) {
        v[a] = 0.0;
        J[a][0] = J[a][1] = J[a][2] = 0.0;
    }
    int k = 0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a, ++k) {
                double wx = a ? t[0] : 1.0 - t[0], dwx = a ? 1.0 : -1.0;
                double wy = b ? t[1] : 1.0 - t[1], dwy = b ? 1.0 : -1.0;
                double wz = c ? t[2] : 1.0 - t[2], dwz = c ? 1.0 : -1.0;
                double w = wx * wy * wz;
                double dw[3] = {dwx * wy * wz / h[0], wx * dwy * wz / h[1], wx * wy * dwz / h[2]};
                size_t node = (size_t)(cell[0] + a) +
                              (size_t)nx * ((size_t)(cell[1] + b) + (size_t)ny * (size_t)(cell[2] + c));
                const float *f = field + 3 * node;
                for (int comp = 0; comp < 3; ++comp) {
                    v[comp] += w * (double)f[comp];
                    for (int d = 0; d < 3; ++d) J[comp][d] += dw[d] * (double)f[comp];
                }
                nodes_out[k] = node;
                w_out[k] = w;
            }
}

static void scatter(double *gF, const size_t nodes[8], const double w[8], const double g[3])
{
    if (!gF) return;
    for (int k = 0; k < 8; ++k)
        for (int comp = 0; comp < 3; ++comp) {
#ifdef _OPENMP
#pragma omp atomic
#endif
            gF[3 * nodes[k] + comp] += w[k] * g[comp];
        }
}

ORACLE_API void bto_oracle_adjoint_cycle(const float *field, const int64_t n[3],
                                         const double origin[3], const double h[3],
                                         double dt, int64_t m, const double *x,
                                         const uint8_t *alive, double *lam, double *gF,
                                         int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int64_t p = 0; p < m; ++p) {
        if (!alive[p]) continue;
        const double *xp = x + 3 * p;
        double k1[3], k2[3], k3[3], k4[3], q2[3], q3[3], q4[3];
        double J1[3][3], J2[3][3], J3[3][3], J4[3][3];
        size_t n1[8], n2[8], n3[8], n4[8];
        double w1[8], w2[8], w3[8], w4[8];
        /* forward stages (same steps as bto_oracle_cycle) */
        sample_jac(field, n, origin, h, xp, k1, J1, n1, w1);
        for (int a = 0; a < 3; ++a) q2[a] = xp[a] + 0.5 * dt * k1[a];
        sample_jac(field, n, origin, h, q2, k2, J2, n2, w2);
        for (int a = 0; a < 3; ++a) q3[a] = xp[a] + 0.5 * dt * k2[a];
        sample_jac(field, n, origin, h, q3, k3, J3, n3, w3);
        for (int a = 0; a < 3; ++a) q4[a] = xp[a] + dt * k3[a];
        sample_jac(field, n, origin, h, q4, k4, J4, n4, w4);
        /* reverse */
        double *lp = lam + 3 * p;
        double g1[3], g2[3], g3[3], g4[3], lx[3], qb[3];
        for (int a = 0; a < 3; ++a) {
            g1[a] = dt / 6.0 * lp[a];
            g2[a] = dt / 3.0 * lp[a];
            g3[a] = dt / 3.0 * lp[a];
            g4[a] = dt / 6.0 * lp[a];
            lx[a] = lp[a];
        }
        /* stage 4: k4 = v(q4), q4 = x + dt k3 */
        for (int d = 0; d < 3; ++d) qb[d] = J4[0][d] * g4[0] + J4[1][d] * g4[1] + J4[2][d] * g4[2];
        scatter(gF, n4, w4, g4);
        for (int a = 0; a < 3; ++a) { lx[a] += qb[a]; g3[a] += dt * qb[a]; }
        /* stage 3: k3 = v(q3), q3 = x + dt/2 k2 */
        for (int d = 0; d < 3; ++d) qb[d] = J3[0][d] * g3[0] + J3[1][d] * g3[1] + J3[2][d] * g3[2];
        scatter(gF, n3, w3, g3);
        for (int a = 0; a < 3; ++a) { lx[a] += qb[a]; g2[a] += 0.5 * dt * qb[a]; }
        /* stage 2: k2 = v(q2), q2 = x + dt/2 k1 */
        for (int d = 0; d < 3; ++d) qb[d] = J2[0][d] * g2[0] + J2[1][d] * g2[1] + J2[2][d] * g2[2];
        scatter(gF, n2, w2, g2);
        for (int a = 0; a < 3; ++a) { lx[a] += qb[a]; g1[a] += 0.5 * dt * qb[a]; }
        /* stage 1: k1 = v(x) */
        for (int d = 0; d < 3; ++d) qb[d] = J1[0][d] * g1[0] + J1[1][d] * g1[1] + J1[2][d] * g1[2];
        scatter(gF, n1, w1, g1);
        for (int a = 0; a < 3; ++a) lp[a] = lx[a] + qb[a];
    }
}

ORACLE_API int32_t bto_oracle_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Post hoc reconstruction over a Delaunay triangulation (Sec. 3.2): the
 * start locations of the valid basis flows are triangulated, and a point of
 * the domain takes the barycentric interpolant of the end positions at the
 * vertices of the tetrahedron that holds it.
 *
 * Points are seed-lattice indices j (integers); the triangulation is built
 * by the Bowyer-Watson algorithm (Bowyer 1981; Watson 1981): points are
 * inserted one at a time; the tetrahedra whose circumsphere holds the new
 * point are removed, and the new point is joined to the faces of the cavity
 * they leave. A large enclosing tetrahedron of four extra points starts the
 * triangulation and its tetrahedra are dropped at the end.
 *
 * Predicates are exact (integer arithmetic in 128 bits). The paper does not
 * say how its triangulation chooses among the Delaunay triangulations of
 * cospherical points (lattice cells are cospherical in eights). Reading:
 * the triangulation is the lower convex hull of the points lifted to
 * w(j) = |j|^2 + d_r(j), where d_0 >> d_1 >> ... > 0 are infinitesimal and
 * r(j) is the point's rank (canonical lattice id, x fastest; the enclosing
 * points rank last). A point e is inside the circumsphere of the tetrahedron
 * (a, b, c, d) when the sign of the 5x5 determinant of the rows
 * (x, y, z, w, 1) says so; when the unperturbed determinant is zero, the
 * term of the lowest-ranked point whose cofactor is not zero decides.
 * --------------------------------------------------------------------------- */
typedef __int128 i128;

typedef struct {
    int64_t x[3];
    int64_t rank;
} dpt;

static i128 det3_128(i128 a0, i128 a1, i128 a2, i128 b0, i128 b1, i128 b2, i128 c0, i128 c1, i128 c2)
{
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
}

/* orientation of (a, b, c, d): det of the rows b - a, c - a, d - a */
static i128 orient3(const dpt *a, const dpt *b, const dpt *c, const dpt *d)
{
    return det3_128(b->x[0] - a->x[0], b->x[1] - a->x[1], b->x[2] - a->x[2],
                    c->x[0] - a->x[0], c->x[1] - a->x[1], c->x[2] - a->x[2],
                    d->x[0] - a->x[0], d->x[1] - a->x[1], d->x[2] - a->x[2]);
}

/* 4x4 determinant by expansion along the last column */
static i128 det4_128(const i128 m[4][4])
{
    i128 r = 0;
    for (int i = 0; i < 4; ++i) {
        i128 s[3][3];
        for (int k = 0, rr = 0; k < 4; ++k) {
            if (k == i) continue;
            for (int c = 0; c < 3; ++c) s[rr][c] = m[k][c];
            ++rr;
        }
        const i128 minor = det3_128(s[0][0], s[0][1], s[0][2], s[1][0], s[1][1], s[1][2], s[2][0], s[2][1], s[2][2]);
        r += ((i + 3) % 2 ? -1 : 1) * m[i][3] * minor;
    }
    return r;
}

/* The 5x5 determinant of the rows (x, y, z, w, 1) of p[0..4] with the lifted
 * weights w = |x|^2 + d_rank: its sign, the infinitesimals resolving a zero. */
static int lifted_sign(const dpt *const p[5])
{
    /* unperturbed part, translated so that p[4] is the origin (the last
     * column then leaves the 4x4 determinant of the first four rows) */
    i128 m[4][4];
    for (int i = 0; i < 4; ++i) {
        i128 s = 0;
        for (int a = 0; a < 3; ++a) {
            m[i][a] = (i128)(p[i]->x[a] - p[4]->x[a]);
            s += m[i][a] * m[i][a];
        }
        m[i][3] = s;
    }
    const i128 d0 = det4_128(m);
    if (d0 != 0) return d0 > 0 ? 1 : -1;
    /* d_r term of row i: (-1)^(i + 3) times the determinant of the rows
     * (x, y, z, 1) of the other four points (0-based rows, w in column 3) */
    int order[5] = {0, 1, 2, 3, 4};
    for (int i = 1; i < 5; ++i)
        for (int k = i; k > 0 && p[order[k]]->rank < p[order[k - 1]]->rank; --k) {
            const int t = order[k]; order[k] = order[k - 1]; order[k - 1] = t;
        }
    for (int oi = 0; oi < 5; ++oi) {
        const int i = order[oi];
        const dpt *q[4];
        for (int k = 0, r = 0; k < 5; ++k)
            if (k != i) q[r++] = p[k];
        /* det of rows (x, y, z, 1) = -orient3(q0, q1, q2, q3) */
        const i128 o = -orient3(q[0], q[1], q[2], q[3]);
        if (o != 0) {
            const i128 c = ((i + 3) % 2 ? -o : o);
            return c > 0 ? 1 : -1;
        }
    }
    return 0;
}

/* e strictly inside the circumsphere of the positively oriented (a, b, c, d) */
static int in_sphere(const dpt *a, const dpt *b, const dpt *c, const dpt *d, const dpt *e)
{
    const dpt *p[5] = {a, b, c, d, e};
    return lifted_sign(p) < 0;
}

typedef struct {
    int32_t v[4];
} dtet;

typedef struct {
    int32_t v[3];     /* sorted vertex ids */
    int32_t o[3];     /* the face's vertices in the order of its tetrahedron's listing */
    int32_t count;
} dface;

static int face_cmp(const void *pa, const void *pb)
{
    const dface *a = (const dface *)pa, *b = (const dface *)pb;
    for (int k = 0; k < 3; ++k)
        if (a->v[k] != b->v[k]) return a->v[k] < b->v[k] ? -1 : 1;
    return 0;
}

/* Delaunay triangulation of the valid points of the lattice S (x fastest).
 * Writes at most cap tetrahedra as canonical lattice ids (each positively
 * oriented) and returns their number; -1: cap too small or allocation
 * failed; -2: a degenerate cavity (never expected with exact predicates). */
ORACLE_API int64_t bto_oracle_delaunay(const int64_t S[3], const uint8_t *valid, int64_t cap, int32_t *tets)
{
    const int64_t P = S[0] * S[1] * S[2];
    int64_t n = 0;
    for (int64_t i = 0; i < P; ++i) n += valid[i] != 0;
    dpt *pts = (dpt *)malloc(sizeof(dpt) * (size_t)(n + 4));
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 4));
    if (!pts || !ids) { free(pts); free(ids); return -1; }
    int64_t k = 0;
    for (int64_t i = 0; i < P; ++i) {
        if (!valid[i]) continue;
        pts[k].x[0] = i % S[0];
        pts[k].x[1] = (i / S[0]) % S[1];
        pts[k].x[2] = i / (S[0] * S[1]);
        pts[k].rank = i;
        ids[k] = i;
        ++k;
    }
    /* enclosing tetrahedron: vertices 2^20 away from the lattice's centre */
    const int64_t B = (int64_t)1 << 20;
    const int64_t cx = S[0] / 2, cy = S[1] / 2, cz = S[2] / 2;
    const int64_t dir[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
    for (int q = 0; q < 4; ++q) {
        pts[n + q].x[0] = cx + 3 * B * dir[q][0];
        pts[n + q].x[1] = cy + 3 * B * dir[q][1];
        pts[n + q].x[2] = cz + 3 * B * dir[q][2];
        pts[n + q].rank = P + q;
        ids[n + q] = -1;
    }
    int64_t tcap = 64 + 8 * (n + 4), nt = 0;
    dtet *T = (dtet *)malloc(sizeof(dtet) * (size_t)tcap);
    uint8_t *alive = (uint8_t *)malloc((size_t)tcap);
    if (!T || !alive) { free(pts); free(ids); free(T); free(alive); return -1; }
    {
        dtet t0 = {{(int32_t)n, (int32_t)(n + 1), (int32_t)(n + 2), (int32_t)(n + 3)}};
        if (orient3(&pts[n], &pts[n + 1], &pts[n + 2], &pts[n + 3]) < 0) {
            const int32_t s = t0.v[0]; t0.v[0] = t0.v[1]; t0.v[1] = s;
        }
        T[0] = t0;
        alive[0] = 1;
        nt = 1;
    }
    int64_t status = 0;
    dface *faces = NULL;
    int64_t fcap = 0;
    for (int64_t ip = 0; ip < n && status == 0; ++ip) {
        const dpt *e = &pts[ip];
        /* the cavity: every tetrahedron whose circumsphere holds the point */
        int64_t nf = 0;
        for (int64_t t = 0; t < nt; ++t) {
            if (!alive[t]) continue;
            const dtet *tt = &T[t];
            if (!in_sphere(&pts[tt->v[0]], &pts[tt->v[1]], &pts[tt->v[2]], &pts[tt->v[3]], e)) continue;
            alive[t] = 0;
            if (nf + 4 > fcap) {
                fcap = 2 * (nf + 4) + 64;
                dface *nfaces = (dface *)realloc(faces, sizeof(dface) * (size_t)fcap);
                if (!nfaces) { status = -1; break; }
                faces = nfaces;
            }
            static const int fv[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
            for (int f = 0; f < 4; ++f) {
                dface *F = &faces[nf++];
                for (int m = 0; m < 3; ++m) F->o[m] = F->v[m] = tt->v[fv[f][m]];
                /* sort v */
                for (int a = 1; a < 3; ++a)
                    for (int b = a; b > 0 && F->v[b] < F->v[b - 1]; --b) {
                        const int32_t s = F->v[b]; F->v[b] = F->v[b - 1]; F->v[b - 1] = s;
                    }
                F->count = 1;
            }
        }
        if (status) break;
        /* faces met twice are inside the cavity; the others bound it */
        qsort(faces, (size_t)nf, sizeof(dface), face_cmp);
        for (int64_t f = 0; f < nf;) {
            int64_t g = f + 1;
            while (g < nf && face_cmp(&faces[f], &faces[g]) == 0) ++g;
            if (g - f == 1) {
                dtet nt4 = {{faces[f].o[0], faces[f].o[1], faces[f].o[2], (int32_t)ip}};
                const i128 o = orient3(&pts[nt4.v[0]], &pts[nt4.v[1]], &pts[nt4.v[2]], &pts[nt4.v[3]]);
                if (o == 0) { status = -2; break; }
                if (o < 0) { const int32_t s = nt4.v[0]; nt4.v[0] = nt4.v[1]; nt4.v[1] = s; }
                if (nt == tcap) {
                    tcap *= 2;
                    dtet *T2 = (dtet *)realloc(T, sizeof(dtet) * (size_t)tcap);
                    uint8_t *a2 = (uint8_t *)realloc(alive, (size_t)tcap);
                    if (T2) T = T2;
                    if (a2) alive = a2;
                    if (!T2 || !a2) { status = -1; break; }
                }
                T[nt] = nt4;
                alive[nt] = 1;
                ++nt;
            }
            f = g;
        }
        /* compact the list now and then */
        if (status == 0 && nt > 4 * (n + 4) + 1024) {
            int64_t w = 0;
            for (int64_t t = 0; t < nt; ++t)
                if (alive[t]) { T[w] = T[t]; alive[w] = 1; ++w; }
            nt = w;
        }
    }
    int64_t out = 0;
    if (status == 0) {
        for (int64_t t = 0; t < nt; ++t) {
            if (!alive[t]) continue;
            if (T[t].v[0] >= n || T[t].v[1] >= n || T[t].v[2] >= n || T[t].v[3] >= n) continue;
            if (out >= cap) { status = -1; break; }
            for (int m = 0; m < 4; ++m) tets[4 * out + m] = (int32_t)ids[T[t].v[m]];
            ++out;
        }
    }
    free(faces); free(T); free(alive); free(pts); free(ids);
    return status ? status : out;
}
