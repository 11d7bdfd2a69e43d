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
