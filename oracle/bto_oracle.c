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
 * On the first failing test: exit_cycle = cycle, x unchanged.
 * min_margin[p] keeps the smallest |margin| (cells) over the tested points,
 * which the parity check uses for its near-face exemption.
 * x: m*3 doubles (in/out); exit_cycle: m ints, -1 while alive (in/out);
 * min_margin: m doubles (in/out), start at +inf.
 * ------------------------------------------------------------------------- */
ORACLE_API void bto_oracle_cycle(const float *field, const int64_t n[3],
                                 const double origin[3], const double h[3],
                                 double dt, int32_t cycle, int64_t m,
                                 double *x, int32_t *exit_cycle,
                                 double *min_margin, int32_t nthreads)
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
        int in;
        double d;

        sample(field, n, origin, h, xp, k1);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + 0.5 * dt * k1[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { exit_cycle[p] = cycle; min_margin[p] = mm; continue; }
        sample(field, n, origin, h, q, k2);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + 0.5 * dt * k2[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { exit_cycle[p] = cycle; min_margin[p] = mm; continue; }
        sample(field, n, origin, h, q, k3);

        for (int a = 0; a < 3; ++a) q[a] = xp[a] + dt * k3[a];
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        if (!in) { exit_cycle[p] = cycle; min_margin[p] = mm; continue; }
        sample(field, n, origin, h, q, k4);

        for (int a = 0; a < 3; ++a)
            q[a] = xp[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        d = margin_cells(n, origin, h, q, &in);
        if (fabs(d) < mm) mm = fabs(d);
        min_margin[p] = mm;
        if (!in) { exit_cycle[p] = cycle; continue; }
        for (int a = 0; a < 3; ++a) xp[a] = q[a];
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
