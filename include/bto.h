/*
 * bto.h -- C ABI of libbto: GB300 (sm_103a) Boundary Termination Optimization
 * (BTO) Lagrangian flow-map extraction.
 *
 * The method (Sane et al., "Scalable In Situ Lagrangian Flow Map Extraction:
 * Demonstrating the Viability of a Communication-Free Model"):
 *   - Sec. 2.3: particles are seeded along a uniform grid at the start of an
 *     interval; an interval is a fixed number of cycles after which the end
 *     positions are saved and the particles reset onto the grid; a 1:X data
 *     reduction places one particle per X grid points.
 *   - Sec. 3.1: each cycle advances every particle by one RK4 step through
 *     the velocity field of that cycle; a particle that would need another
 *     block's data is terminated and its trajectory discarded; particle
 *     management keeps terminated particles off the GPU threads.
 *   - Sec. 3.3, Eq. (1): the velocity between nodes is the linear
 *     interpolant per axis and per component (trilinear in 3D).
 *
 * Conventions of this library (the paper is silent on them):
 *   - A block has n[a] CELLS per axis and (n[a]+1) velocity NODES per axis at
 *     origin[a] + i*spacing[a], i = 0..n[a]. Neighbouring blocks share their
 *     face node layer.
 *   - The block is the CLOSED box [origin, origin + n*spacing]. Each RK4 stage
 *     point (p2, p3, p4) and the end point are tested in that order; the first
 *     one outside terminates the particle, which keeps its position from
 *     before that step and records the cycle index.
 *   - Seeds sit at node indices j*s (j = 0..ceil(n/s)-1 per axis); the seed
 *     with lattice index (jx, jy, jz) has canonical id
 *     p = jx + Sx*(jy + Sy*jz), S = ceil(n/s). Outputs are in canonical order.
 *   - Cycles are numbered 0..interval_cycles-1 within each interval.
 *
 * Memory and streams: all pointers named d_* are DEVICE pointers of the
 * current CUDA device; all others are host pointers. Every call that takes a
 * stream enqueues its work on that stream and returns without waiting for it
 * (no host synchronisation on the per-cycle path). The caller keeps d_field
 * and output buffers valid until that stream work has completed. The library
 * owns the context and all particle state; it never retains caller pointers
 * beyond the stream work of the call that received them (except the field
 * table given to bto_launch_interval_graph, see there).
 *
 * Errors: argument checks are synchronous and return BTO_ERR_INVALID_ARG
 * without launching anything; calls out of order return BTO_ERR_STATE without
 * launching anything; a failed launch returns BTO_ERR_CUDA. Device-side
 * errors are sticky and reported by bto_last_error().
 */
#ifndef BTO_H
#define BTO_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BTO_API __attribute__((visibility("default")))
#else
#define BTO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *bto_stream;

typedef struct bto_ctx bto_ctx;

typedef enum {
    BTO_OK = 0,
    BTO_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or value */
    BTO_ERR_STATE = 2,       /* call out of order (see bto_advect_cycle) */
    BTO_ERR_CUDA = 3,        /* a CUDA call or launch failed */
    BTO_ERR_OOM = 4,         /* device or host allocation failed */
    BTO_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    BTO_ERR_UNSUPPORTED = 6, /* valid request in a configuration the library does not support */
    BTO_ERR_BOUNDS = 7       /* a bounds check failed (bounds-checked builds only) */
} bto_status;

/* Field layouts accepted by bto_advect_cycle.
 * F3_AOS: float32 x,y,z per node, 12 bytes per node, x index fastest
 *         (node (i,j,k) at element i + (n0+1)*(j + (n1+1)*k)).
 * F4_AOS: float32 x,y,z,pad per node, 16 bytes per node, same order;
 *         the pad value is ignored; d_field must be 16-byte aligned. */
typedef enum { BTO_FIELD_F3_AOS = 0, BTO_FIELD_F4_AOS = 1 } bto_field_layout;

/* Create a context for one block (Sec. 2.3 problem statement: a block of a
 * uniform grid, a seeding density and an interval length).
 *   extent_cells[3]  cells per axis, each >= 1; nodes per block <= 2^29
 *   origin[3]        physical position of node (0,0,0), finite
 *   spacing[3]       physical cell size per axis, finite and > 0
 *   seed_stride      s >= 1: one seed per s^3 grid points (1:s^3 reduction)
 *   interval_cycles  L >= 1 cycles per interval
 *   out              receives the context; unchanged on error
 * Allocates the particle state on the current device and seeds the first
 * interval (synchronously). Returns BTO_ERR_OOM if the device memory is not
 * available. */
BTO_API bto_status bto_create(const int32_t extent_cells[3], const float origin[3],
                      const float spacing[3], int32_t seed_stride,
                      int32_t interval_cycles, bto_ctx **out);

/* Create one context for nb independent blocks of possibly different shapes
 * that advance together, one persistent launch per cycle (the paper's
 * per-rank blocks, Sec. 3.1, emulated on one device). Arrays have nb entries
 * (extents, origins and spacings: nb*3 values, block-major). Seeds of block b
 * occupy canonical ids offsets[b] .. offsets[b+1]-1 (bto_batch_offsets). */
BTO_API bto_status bto_batch_create(int32_t nb, const int32_t *extents,
                            const float *origins, const float *spacings,
                            const int32_t *strides, int32_t interval_cycles,
                            bto_ctx **out);

/* Select the layout of the fields passed to the advect calls (default
 * BTO_FIELD_F3_AOS). Only between intervals (cycle 0), else BTO_ERR_STATE. */
BTO_API bto_status bto_set_field_layout(bto_ctx *ctx, bto_field_layout layout);

/* Field ingest (enable = 1): with F3_AOS fields, each cycle first repacks
 * every block's field into a 16-byte-per-node buffer owned by the context
 * (two buffers, block b+1 repacked on an internal stream while block b is
 * advected on the caller's stream) and the advection gathers one 16-byte
 * load per node from it. Results are identical with and without ingest.
 * Allocates 2 x (largest block's nodes) x 16 bytes on first use. Only at
 * cycle 0 and with the F3_AOS layout, else BTO_ERR_STATE; not available
 * with bto_launch_interval_graph (BTO_ERR_UNSUPPORTED). enable = 0 goes
 * back to gathering from the caller's F3 field directly (the default). */
BTO_API bto_status bto_set_ingest(bto_ctx *ctx, int32_t enable);

/* Total number of seeds P of the context (all blocks), or -1 for NULL. */
BTO_API int64_t bto_num_seeds(const bto_ctx *ctx);

/* Number of blocks of the context, or -1 for NULL. */
BTO_API int32_t bto_num_blocks(const bto_ctx *ctx);

/* offsets[nb+1] (host): first canonical id of each block, offsets[nb] = P. */
BTO_API bto_status bto_batch_offsets(const bto_ctx *ctx, int64_t *offsets);

/* One cycle of a single-block context (Sec. 3.1): every live particle takes
 * one RK4 step through d_field with step dt (any finite value; negative
 * integrates backward, 0 is a no-op step). Particles whose stage or end point
 * leaves the block are terminated and removed from the active set.
 *   d_field  device pointer to the block's nodes in the selected layout
 * BTO_ERR_STATE if interval_cycles cycles were already advanced since the
 * last bto_end_interval, or if ctx holds more than one block.
 * The cycle's kernel (here and in bto_batch_advect_cycle) is launched with
 * programmatic stream serialisation: its launch may overlap the tail of the
 * kernel before it on the stream, and it reads nothing before that kernel
 * has completed. It lets the next kernel launch early in turn: a kernel the
 * caller launches next on the stream with programmatic serialisation must
 * wait on its grid dependency (griddepcontrol.wait) before it touches memory
 * the cycle reads or writes (the context's outputs, or d_field, for
 * instance when it writes the next cycle's field in place); ordinary
 * launches, copies and events wait for completion as usual. */
BTO_API bto_status bto_advect_cycle(bto_ctx *ctx, const void *d_field, float dt,
                            bto_stream stream);

/* One cycle of a batched context.
 *   d_fields  DEVICE array of nb device pointers, entry b = field of block b
 * The pointer array is read by the kernel on the stream. */
BTO_API bto_status bto_batch_advect_cycle(bto_ctx *ctx, const void *const *d_fields,
                                  float dt, bto_stream stream);

/* End the interval (Sec. 2.3): write the basis flows in canonical order and
 * reseed every block on its lattice.
 *   d_seeds       P*3 floats: seed position (physical)
 *   d_ends        P*3 floats: end position (physical); for a terminated
 *                 particle, its last position inside the block
 *   d_valid       P bytes: 1 = stayed in its block for the whole interval
 *   d_exit_cycle  P int32 or NULL: cycle of termination, -1 if valid
 * Every entry of every non-NULL buffer is written exactly once.
 * BTO_ERR_STATE unless exactly interval_cycles cycles were advanced. */
BTO_API bto_status bto_end_interval(bto_ctx *ctx, float *d_seeds, float *d_ends,
                            uint8_t *d_valid, int32_t *d_exit_cycle,
                            bto_stream stream);

/* bto_end_interval plus the termination locations (storing them is the
 * paper's stated future work, Sec. 6; a reading of this library):
 *   d_exit_pos   P*3 floats or NULL: for a terminated particle, the point
 *                where the chord from its last in-block position to the
 *                first tested point found outside (p2, p3, p4 or end
 *                point) leaves the closed block; NaN for valid particles
 *   d_exit_time  P floats or NULL: the matching time in cycles from the
 *                start of the interval, c + t * f, with c the exit cycle,
 *                t in [0, 1] the clipped fraction of the chord and f = 1/2
 *                for p2/p3, 1 for p4 and the end point; NaN if valid
 * Other arguments, errors and the reseed as in bto_end_interval. */
BTO_API bto_status bto_end_interval_ex(bto_ctx *ctx, float *d_seeds, float *d_ends,
                                       uint8_t *d_valid, int32_t *d_exit_cycle,
                                       float *d_exit_pos, float *d_exit_time, bto_stream stream);

/* Capture the cycles of one interval of a context into a CUDA graph and
 * launch it on `stream`; later intervals relaunch the cached graph.
 *   d_field_table  DEVICE array of interval_cycles*nb device pointers,
 *                  entry c*nb + b = field of block b in cycle c; it must
 *                  stay valid (and its entries point at the fields) for as
 *                  long as the graph is relaunched
 *   dt             step of every cycle
 * Equivalent to interval_cycles advect calls, but one graph launch.
 * Must be called at cycle 0; leaves the context at cycle interval_cycles. */
BTO_API bto_status bto_launch_interval_graph(bto_ctx *ctx, const void *const *d_field_table,
                                     float dt, bto_stream stream);

/* Launch shape of the advection kernel: threads per CTA (128 or 256),
 * particles per thread (1, 2 or 4; a warp owns 32*ppt list slots), CTAs per
 * SM (0 = as many as fit) and reg_cap (1 = registers capped at 80 per
 * thread so that 768 threads fit on an SM; 0 = no cap). Results do not
 * depend on the shape. Only at cycle 0 (between intervals), else
 * BTO_ERR_STATE; changing particles_per_thread reseeds the interval
 * (synchronously). */
BTO_API bto_status bto_set_launch(bto_ctx *ctx, int32_t threads_per_cta,
                                  int32_t particles_per_thread, int32_t ctas_per_sm,
                                  int32_t reg_cap);

/* Report the launch shape in use (host ints: threads, ppt, ctas_per_sm,
 * reg_cap, grid size). */
BTO_API bto_status bto_get_launch(const bto_ctx *ctx, int32_t out[5]);

/* Autotuner: times every compiled launch shape of the advection kernel
 * (threads 128/256 x particles per thread 1/2/4 x reg_cap 0/1) on this
 * context's own blocks, and keeps the fastest. Each trial reseeds the
 * interval, runs `cycles` cycles (1..interval_cycles) on the fields of
 * d_field_table (DEVICE array of at least cycles*nb field pointers, entry
 * c*nb + b for block b in cycle c, as for bto_launch_interval_graph) with
 * step dt, and is timed with CUDA events on `stream`; the interval is
 * reseeded at the end. Synchronises the stream (a set-up call). Only at
 * cycle 0, else BTO_ERR_STATE. Outputs (host, optional): best[5] as
 * bto_get_launch, ms[12] the mean time per cycle of each shape in the order
 * above (threads slowest, reg_cap fastest). Results do not depend on the
 * shape, only the speed does. */
BTO_API bto_status bto_autotune(bto_ctx *ctx, const void *const *d_field_table, int32_t cycles,
                                float dt, bto_stream stream, int32_t best[5], float ms[12]);

/* Tiled advection (kernel K3t): the same cycle (Sec. 3.1, Eq. 1; results
 * identical to the untiled kernel), organised around the field. Each
 * block's cells are cut into tiles of tile_cells[0] x [1] x [2] cells
 * (powers of two, 2..128 each; ragged at the upper faces). A persistent CTA
 * stages, a few tiles ahead, each tile's nodes plus one cell of halo and the
 * tile's particle records into shared memory with bulk asynchronous copies,
 * advects the particles whose cell lies in the tile, and writes every
 * survivor to the bucket of its new tile. Cells outside the staged box are
 * gathered from global memory, so any speed is handled.
 *   tile_cells       host int32[3]; NULL or {0,0,0} switches tiling off
 *   threads_per_cta  128 or 256
 * Allocates the buckets (about 2.3 x 16 bytes per particle, twice) on the
 * first call; reseeds the interval (synchronously). Only at cycle 0, else
 * BTO_ERR_STATE; BTO_ERR_STATE also with H1 ingest on; BTO_ERR_UNSUPPORTED
 * when the staging buffers do not fit in shared memory or a tile has more
 * than 4 * threads_per_cta - 2 staged node rows, (ty + 3) * (tz + 3). The
 * autotuner times untiled shapes only (BTO_ERR_STATE while tiling is on). */
BTO_API bto_status bto_set_tiling(bto_ctx *ctx, const int32_t tile_cells[3], int32_t threads_per_cta);

/* Test hook for the bounded-wait error path of the tiled kernel: in the
 * next `cycles` tiled cycles, CTA 0 announces on its staging barrier 16
 * bytes more than its copies deliver, so its wait gives up after about two
 * seconds. The CTA then waits (bounded) for its copies in flight, leaves its
 * tiles empty and consistent (their particles are lost) and returns; the
 * other CTAs are unaffected. bto_last_error reports BTO_ERR_TIMEOUT; the
 * context stays usable and the next interval is reseeded as usual. Nothing
 * faults: every wait ends by its bound. BTO_ERR_STATE unless tiling is on. */
BTO_API bto_status bto_test_wait_timeout(bto_ctx *ctx, int32_t cycles);

/* Tiling in use (host ints: tile cells x, y, z, threads per CTA, grid,
 * tiles, staging buffers per CTA, 1 if the particle records are staged with
 * the nodes; all 0 when off). */
BTO_API bto_status bto_get_tiling(const bto_ctx *ctx, int32_t out[8]);

/* Diagnostics (not for the per-cycle path): copy the active particle list as
 * it stands before the next cycle.
 *   d_out  P*4 floats (device); for block b, rows offsets[b] ..
 *          offsets[b] + live[b] - 1 hold (xi_x, xi_y, xi_z, id bits) of its live
 *          particles, xi = (x - origin) / spacing in block-local cell units and
 *          id = canonical id within the block (int32 bits); other rows are
 *          unspecified; with tiling on, the order inside a block is
 *          unspecified too
 *   live   nb int32 (host): live particles per block
 * Waits for `stream`. */
BTO_API bto_status bto_copy_active(bto_ctx *ctx, float *d_out, int32_t *live,
                                   bto_stream stream);

/* Sticky error of earlier asynchronous work of this context (a launch
 * failure, or BTO_ERR_TIMEOUT when a bounded device wait of the tiled
 * kernel gave up); waits for the context's last stream work; clears the
 * sticky state. */
BTO_API bto_status bto_last_error(bto_ctx *ctx);

/* ---- Post hoc reconstruction (Sec. 3.2, Sec. 3.3 Eq. 2) -----------------
 *
 * Lattice stand-in for the paper's Delaunay + barycentric reconstruction:
 * basis flows on a lattice in canonical order (index jx + Sx*(jy + Sy*jz)),
 * for instance the union of the blocks' seed lattices of a decomposed
 * domain. A missing entry (valid = 0) takes, along the axis whose nearest
 * valid neighbours on both sides are closest (a + b smallest; ties x, then
 * y, then z), the linear interpolant (Eq. 1) of their end positions:
 * end(J) = (b end(J - a) + a end(J + b)) / (a + b). Eq. (2) shows that
 * interpolating through such a filled value equals interpolating from the
 * two neighbours. Entries with no such axis stay missing (NaN).
 *   lattice[3]  Sx, Sy, Sz >= 1 (host)
 *   d_ends      P*3 floats; entries with valid = 0 are ignored
 *   d_valid     P bytes
 *   d_out       P*3 floats written (must not overlap d_ends)
 *   d_status    P bytes or NULL: 1 = valid, 2 = filled, 0 = still missing */
BTO_API bto_status bto_fill_lattice(const int32_t lattice[3], const float *d_ends,
                                    const uint8_t *d_valid, float *d_out, uint8_t *d_status,
                                    bto_stream stream);

/* Reconstruction over a Delaunay triangulation (Sec. 3.2: a Delaunay
 * triangulation over the start locations of the valid basis flows of the
 * own and adjacent blocks, then barycentric interpolation). Same lattice,
 * arguments and outputs as bto_fill_lattice: a missing entry takes the
 * barycentric interpolant of the end positions at the vertices of the
 * Delaunay tetrahedron of the valid lattice points that holds its own
 * lattice point. Ties among cospherical lattice points are broken by
 * infinitesimal lifted weights ordered by canonical lattice id. Each
 * missing entry is solved over the valid points within 2 to 8 lattice
 * units of it, 2 to 12 on a boundary face (the smallest window that
 * holds its simplex's circumsphere). An entry on a boundary face of the
 * lattice lies on the hull of the valid points and takes the interpolant
 * over the face's triangle (the tetrahedra meet the face in the Delaunay
 * triangulation of the face's own points); one on a boundary edge takes
 * the linear interpolant of its nearest valid neighbours along the edge. A
 * corner, an entry outside the hull of the valid points, one whose
 * tetrahedron (triangle) needs a larger window, and every missing entry of
 * a lattice one point thick along some axis stay missing (NaN, status 0). */
BTO_API bto_status bto_fill_delaunay(const int32_t lattice[3], const float *d_ends,
                                     const uint8_t *d_valid, float *d_out, uint8_t *d_status,
                                     bto_stream stream);

/* Pathline stitching (Sec. 3.2): new particles follow the basis flows of
 * successive intervals. In interval k a particle's next position is the
 * trilinear interpolant (Eq. 1 per axis; bto_stitch_pathlines_ex also
 * offers the paper's barycentric interpolation) of the end positions of the
 * 8 basis flows of its seed-lattice cell. Outside the lattice, or in a cell with a
 * missing (NaN) basis flow, the particle stops and its later positions are
 * NaN.
 *   lattice[3], origin[3], spacing[3]  seed lattice (host): point j at
 *                origin + j * spacing, j = 0..lattice-1 per axis
 *   d_ends_table DEVICE array of `intervals` device pointers, each P*3 floats
 *                of lattice end positions in canonical order (bto_fill_lattice
 *                output)
 *   d_start      nq*3 floats, start positions (physical)
 *   d_path       (intervals+1)*nq*3 floats written: positions at the start
 *                and at the end of every interval */
BTO_API bto_status bto_stitch_pathlines(const int32_t lattice[3], const float origin[3],
                                        const float spacing[3], int32_t intervals,
                                        const float *const *d_ends_table, int64_t nq,
                                        const float *d_start, float *d_path, bto_stream stream);

/* Interpolation of the basis flows in bto_stitch_pathlines_ex. */
typedef enum {
    BTO_STITCH_TRILINEAR = 0,   /* the 8 corners of the lattice cell (Eq. 1 per axis) */
    BTO_STITCH_BARYCENTRIC = 1  /* barycentric coordinates in a tetrahedron of the cell */
} bto_stitch_scheme;

/* bto_stitch_pathlines with a choice of interpolant (Sec. 3.2: the paper
 * follows a Delaunay neighbourhood of basis flows with barycentric
 * coordinates). On a complete seed lattice the 8 corners of a cell lie on
 * one sphere, so any face-conforming split of the cells into tetrahedra is
 * a Delaunay triangulation of the start points; BTO_STITCH_BARYCENTRIC
 * takes the Kuhn split, the 6 tetrahedra around the cell's main diagonal.
 * For fractional cell coordinates t sorted in decreasing order,
 * t_a >= t_b >= t_c (ties keep the axis order x, y, z), the tetrahedron is
 * corner 0, corner 0 + e_a, corner 0 + e_a + e_b, corner 0 + (1, 1, 1),
 * with weights 1 - t_a, t_a - t_b, t_b - t_c, t_c. A particle stops (NaN)
 * outside the lattice or when a vertex of its tetrahedron is missing; for
 * BTO_STITCH_TRILINEAR, when any corner of its cell is missing.
 *   scheme       a bto_stitch_scheme value; anything else is
 *                BTO_ERR_INVALID_ARG
 *   other arguments as in bto_stitch_pathlines */
BTO_API bto_status bto_stitch_pathlines_ex(const int32_t lattice[3], const float origin[3],
                                           const float spacing[3], int32_t intervals,
                                           const float *const *d_ends_table, int64_t nq,
                                           const float *d_start, float *d_path, int32_t scheme,
                                           bto_stream stream);

/* ---- Adjoint: gradients of a loss on end positions ----------------------
 *
 * The basis flow of a particle is a function of its start position and of
 * every cycle's node velocities (Sec. 3.1 advection, Eq. 1 sampling). A tape
 * runs one interval of one block from caller-given start positions, keeps
 * positions every checkpoint_every cycles, and then returns vector-Jacobian
 * products of the end positions: with respect to the start positions (the
 * flow-map Jacobian, from which FTLE) and to the node velocities. Segments
 * between checkpoints are recomputed during the backward sweep.
 * A terminated particle's end is its last in-block position; its gradient
 * flows back through the cycles before its exit cycle only (termination
 * itself is a discrete decision with no gradient). Particles occupy fixed
 * slots (no compaction); start positions outside the block never move.
 * Only the F3_AOS field layout is accepted. */
typedef struct bto_tape bto_tape;

/* extent_cells, origin, spacing as in bto_create; num_particles >= 1;
 * cycles >= 1; checkpoint_every >= 1 (clamped to cycles). Allocates
 * (cycles/checkpoint_every + 2 + checkpoint_every) * num_particles * 16 B. */
BTO_API bto_status bto_tape_create(const int32_t extent_cells[3], const float origin[3],
                                   const float spacing[3], int64_t num_particles,
                                   int32_t cycles, int32_t checkpoint_every, bto_tape **out);

/* Particles of the tape, or -1 for NULL. */
BTO_API int64_t bto_tape_num_particles(const bto_tape *tape);

/* Forward interval.
 *   d_seeds        P*3 floats, start positions (physical)
 *   d_field_table  DEVICE array of `cycles` device pointers (F3_AOS fields);
 *                  the table and the fields must stay valid until the last
 *                  backward/jacobian call of this forward has completed
 *   d_ends, d_valid, d_exit_cycle (nullable): as in bto_end_interval */
BTO_API bto_status bto_tape_forward(bto_tape *tape, const float *d_seeds,
                                    const void *const *d_field_table, float dt, float *d_ends,
                                    uint8_t *d_valid, int32_t *d_exit_cycle, bto_stream stream);

/* Reverse sweep of the last forward.
 *   d_grad_ends          P*3 floats: dL/d(end position)
 *   d_grad_seeds         P*3 floats written: dL/d(start position)
 *   d_grad_field_table   NULL, or DEVICE array of `cycles` device pointers to
 *                        F3-shaped float buffers that receive (+=) dL/d(node
 *                        velocity) of each cycle (scatter-add with atomics)
 * BTO_ERR_STATE without a forward. */
BTO_API bto_status bto_tape_backward(bto_tape *tape, const float *d_grad_ends,
                                     float *d_grad_seeds, float *const *d_grad_field_table,
                                     bto_stream stream);

/* Flow-map Jacobian of the last forward: d_jac (P*9 floats, row-major per
 * particle) receives J[a][b] = d end_a / d start_b (three reverse sweeps). */
BTO_API bto_status bto_tape_jacobian(bto_tape *tape, float *d_jac, bto_stream stream);

/* FTLE from a Jacobian: d_ftle[p] = ln(sqrt(lambda_max(J^T J))) / |cycles*dt|
 * for particles valid over the interval, NaN for terminated ones. */
BTO_API bto_status bto_tape_ftle(bto_tape *tape, const float *d_jac, float *d_ftle,
                                 bto_stream stream);

/* Wait for outstanding work, then free the tape. NULL is a no-op. */
BTO_API void bto_tape_destroy(bto_tape *tape);

/* ---- Allocation-free interval (no counterpart in the paper) -------------
 *
 * For callers that cannot let a library allocate device memory: for example an
 * in situ simulation that gives all device memory to its own pool allocator at
 * start-up and forbids allocations by analysis libraries while it runs, which
 * rules out bto_create (it allocates the particle state). This call runs one
 * whole interval of one block (seed, interval_cycles RK4 cycles with
 * termination, basis-flow output: the same kernels as the context calls)
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * The particle state lives in a fixed array of BTO_NOALLOC_SCRATCH_BYTES in
 * the library's device image. The CUDA runtime loads that image on a device
 * lazily (its default module loading): the first call on each device, made
 * with that device current, loads it, which reserves the array's
 * BTO_NOALLOC_SCRATCH_BYTES of device memory there, looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it. That first call is
 * therefore itself a device allocation by the runtime: make it once at
 * start-up, before handing device memory to a pool allocator and before any
 * stream capture; later calls on that device allocate nothing. The array
 * stays reserved until the process exits. All calls on a device share it,
 * and it keeps the last call's contents (each call rewrites what it reads
 * first), so calls whose GPU work overlaps (different streams, or several
 * host threads) race with each other and give wrong results: order them on
 * one stream.
 *
 *   extent_cells, origin, spacing, seed_stride, interval_cycles
 *                  as in bto_create; at most BTO_NOALLOC_MAX_SEEDS seeds
 *                  (more returns BTO_ERR_UNSUPPORTED, nothing launched)
 *   d_field_table  DEVICE array of interval_cycles device pointers: entry c
 *                  is the F3_AOS field of cycle c
 *   dt             step of every cycle (finite)
 *   d_seeds, d_ends, d_valid, d_exit_cycle
 *                  outputs as in bto_end_interval (d_exit_cycle may be NULL)
 *   stream         all work is enqueued on it; the call does not wait
 * Seeds are processed in canonical lattice order (not brick order); the
 * outputs are identical to the context calls'. */
#define BTO_NOALLOC_MAX_SEEDS 65536
#define BTO_NOALLOC_SCRATCH_BYTES 2375936
BTO_API bto_status bto_interval_noalloc(const int32_t extent_cells[3], const float origin[3],
                                        const float spacing[3], int32_t seed_stride,
                                        int32_t interval_cycles,
                                        const void *const *d_field_table, float dt,
                                        float *d_seeds, float *d_ends, uint8_t *d_valid,
                                        int32_t *d_exit_cycle, bto_stream stream);

/* ---- Device allocator hook (no counterpart in the paper) ----------------
 *
 * For callers whose own pool allocator owns the device memory: once a hook is
 * installed, every device allocation the library makes for a context or a
 * tape (bto_create, bto_batch_create, bto_set_tiling, bto_set_ingest,
 * bto_copy_active, bto_tape_create) calls alloc(bytes, user) instead of
 * cudaMalloc, and frees with free_fn(ptr, user) instead of cudaFree.
 *   alloc     returns a device pointer to at least `bytes` bytes, 256-byte
 *             aligned, on the current device; or NULL: the calling function
 *             then frees what it had allocated through free_fn and returns
 *             BTO_ERR_OOM. A misaligned pointer is freed again and the call
 *             returns BTO_ERR_CUDA.
 *   free_fn   releases a pointer alloc returned.
 * Both NULL restores cudaMalloc / cudaFree; one NULL: BTO_ERR_INVALID_ARG.
 * Process-wide; a context or tape keeps the hook that was installed when it
 * was created and frees through it, so the hook's memory must outlive it.
 * Allocations by the CUDA runtime itself (module loading, streams, graphs)
 * do not go through the hook. */
typedef void *(*bto_alloc_fn)(size_t bytes, void *user);
typedef void (*bto_free_fn)(void *ptr, void *user);
BTO_API bto_status bto_set_device_allocator(bto_alloc_fn alloc, bto_free_fn free_fn, void *user);

/* ---- Bounds-checked builds (no counterpart in the paper) ----------------
 *
 * Compiled with BTO_CHECK_BOUNDS defined (build.build(check_bounds=True)),
 * the kernels test every field-node index of a global gather, every group
 * count and particle id of the particle list, every destination tile of the
 * tiled path and every lattice index of the post hoc kernels before using
 * it. A failed test skips the access (a node or lattice index is replaced by
 * 0, a write is dropped), adds one to a failure counter and, for the kernels
 * of a context, sets the context's error word, which bto_last_error returns
 * as BTO_ERR_BOUNDS. No check traps. Product builds compile the tests out.
 *
 * bto_check_bounds_build: 1 for a bounds-checked build, 0 otherwise.
 * bto_bounds_failures:    failed checks since load (or the last reset) in
 *                         *count (0 in product builds); reset != 0 clears
 *                         the counters. Synchronous: waits for the device. */
BTO_API int32_t bto_check_bounds_build(void);
BTO_API bto_status bto_bounds_failures(uint64_t *count, int32_t reset);

/* Static string for a status code. */
BTO_API const char *bto_status_string(bto_status status);

/* Wait for outstanding work of the context, then free it. NULL is a no-op. */
BTO_API void bto_destroy(bto_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BTO_H */
