// Internal declarations shared by the host API (bto_api.cu) and the kernels
// (bto_kernels.cu) of libbto. Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bto {

// Where the library's device memory comes from: the caller's allocator
// installed with bto_set_device_allocator, else cudaMalloc / cudaFree.
// Contexts and tapes keep the allocator that was current when they were
// created and free through it.
struct DevAlloc {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *user = nullptr;
    template <class T>
    cudaError_t get(T **p, size_t bytes) const {
        if (!alloc) return cudaMalloc(reinterpret_cast<void **>(p), bytes);
        if (bytes == 0) {   // as cudaMalloc: nothing to allocate, a null pointer
            *p = nullptr;
            return cudaSuccess;
        }
        void *q = alloc(bytes, user);
        if (q && (reinterpret_cast<uintptr_t>(q) & 255u)) {   // the contract asks for 256-byte alignment
            release(q, user);
            *p = nullptr;
            return cudaErrorInvalidValue;
        }
        *p = static_cast<T *>(q);
        return q ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    void put(void *p) const {
        if (!p) return;
        if (alloc) release(p, user);
        else cudaFree(p);
    }
};

// The process-wide allocator (bto_api.cu).
DevAlloc current_allocator();

// Values of a context's device error word.
constexpr int32_t kErrTimeout = 1;   // a bounded wait gave up
constexpr int32_t kErrBounds = 2;    // a bounds check failed (bounds-checked builds)

// Bounds-checked builds (-DBTO_CHECK_BOUNDS): BTO_IN_BOUNDS(cond, err)
// tests cond before an access; when it fails, the access is skipped, the
// translation unit's failure counter is incremented and, when err is not
// null, the context's error word is set to kErrBounds. Product builds
// compile the test out (it is always true). No check traps.
#ifdef BTO_CHECK_BOUNDS
static __device__ unsigned long long g_bto_bounds_failures;
__device__ __forceinline__ bool in_bounds_check(bool ok, int32_t *err) {
    if (!ok) {
        atomicAdd(&g_bto_bounds_failures, 1ull);
        if (err) atomicExch(err, kErrBounds);
    }
    return ok;
}
#define BTO_IN_BOUNDS(cond, err) ::bto::in_bounds_check((cond), (err))
#define BTO_BOUNDS_ACCESSOR(name)                                                                 \
    unsigned long long name(bool reset) {                                                         \
        unsigned long long v = 0;                                                                 \
        if (cudaMemcpyFromSymbol(&v, g_bto_bounds_failures, sizeof(v)) != cudaSuccess) return ~0ull; \
        if (reset) {                                                                              \
            const unsigned long long z = 0;                                                       \
            if (cudaMemcpyToSymbol(g_bto_bounds_failures, &z, sizeof(z)) != cudaSuccess) return ~0ull; \
        }                                                                                         \
        return v;                                                                                 \
    }
#else
#define BTO_IN_BOUNDS(cond, err) true
#define BTO_BOUNDS_ACCESSOR(name) \
    unsigned long long name(bool) { return 0; }
#endif
// Failure counters of the kernels' translation units (bounds-checked
// builds; 0 otherwise; ~0 when the counter cannot be read).
unsigned long long bounds_failures_kernels(bool reset);
unsigned long long bounds_failures_tiled(bool reset);
unsigned long long bounds_failures_posthoc(bool reset);
unsigned long long bounds_failures_delaunay(bool reset);

// One block of the uniform grid, as the kernels see it. Positions inside the
// library are block-local CELL coordinates xi = (x - origin) / h, so node i
// sits at xi = i and the block is the closed box [0, n].
struct BlockDev {
    int32_t n[3];       // cells per axis
    int32_t nn[3];      // nodes per axis (n + 1)
    int32_t S[3];       // seed lattice size per axis, ceil(n / stride)
    int32_t stride;     // seed stride in cells
    float inv_h[3];     // 1 / spacing
    float origin[3];    // physical position of node (0,0,0)
    float h[3];         // spacing
    int32_t pad_;
    int64_t base;       // first canonical id of the block
    int64_t slot_base;  // first slot of the block's list region (multiple of kRegionAlign)
    int64_t nseeds;     // seeds of the block
};

// Every block's list region starts at a multiple of kRegionAlign slots, so a
// particle group (32 * particles-per-thread slots, a divisor of kRegionAlign)
// never straddles two blocks. gblock[] maps each 32-slot unit to its block.
constexpr int kRegionAlign = 128;
constexpr int kUnit = 32;

// Particle state of the untiled path, updated in place every cycle. The
// slots come in units of 32 (kUnit); unit u holds, at rec + 128 u, the x
// coordinates of its 32 slots, then their y, their z (cell units) and their
// block-local canonical ids (int bits), so that a warp reads or writes one
// field of 32 slots as one 128-byte line. The list is cut into groups of
// G = 32 * ppt slots; group g holds its gcnt[g] live particles in its first
// slots, in brick order of their seeds. Positions are read and written
// every cycle; ids move only when a group loses a particle.
struct PartList {
    float *rec;
    int32_t *gcnt;
};

// Field f (0: x, 1: y, 2: z, 3: id bits) of slot i.
__host__ __device__ __forceinline__ int64_t part_at(int64_t i, int f) {
    return ((i >> 5) << 7) + 32 * f + (i & 31);
}

// Arguments of one advection cycle (kernel K3: RK4 + termination + compaction).
struct AdvectArgs {
    const BlockDev *blocks;      // [nb] device
    const int32_t *gblock;       // [slots / 32] block of each 32-slot unit
    int32_t nb;
    int32_t cycle;               // cycle index within the interval
    const void *field;           // single field pointer (nb == 1 calls), or NULL
    const void *const *fields;   // device array [nb] used when field == NULL
    PartList p;                  // particle state (groups from 0 to ngroups - 1)
    int64_t ngroups;
    float4 *term;                // [P] termination record per canonical id
    float4 *clip;                // [P] first outside point (xi) and its RK4 stage, or NULL
    int32_t *err;                // context error word (bounds-checked builds)
    float dt;
};

enum { LAYOUT_F3 = 0, LAYOUT_F4 = 1 };

// Tiled advection (kernel K3t). Each block's cells are cut into tiles of
// tx * ty * tz cells (powers of two; ragged at the upper faces). The live
// particles whose cell lies in tile t at the start of a cycle sit in two
// regions of the list: the front region [fbase, fbase + capf), holding the
// particles that stayed in t during the last cycle (or its seeds), and the
// move-in region [mbase + t * cm, + cm), holding those that came from other
// tiles. Records that find their region full go to an overflow region
// shared by all blocks, [obase, obase + ocap).
struct TileDev {
    int32_t b;          // block
    int32_t capf;       // front-region capacity (multiple of 32)
    int64_t fbase;      // first slot of the front region (multiple of 32)
    int32_t lo[3];      // staged node box: first node per axis (first cell - 1, clamped)
    int32_t hi[3];      // last node per axis (last cell + 2, clamped to n)
    float tlo[3];       // first cell of the tile per axis
    float thi[3];       // first cell after the tile; +inf on the block's last tile of the axis
};

struct BlockTiles {
    int32_t first;      // index of the block's first tile
    int32_t nt[3];      // tiles per axis (x fastest)
};

// Counts of a tiled list, as the interval-end and diagnostic kernels read
// them: per tile its front count and move-in count, and the overflow count.
struct TileCounts {
    const int32_t *front;
    const int32_t *movein;
    const int32_t *ocnt;
    int64_t mbase;       // first slot of the move-in regions
    int64_t obase;       // first slot of the overflow region
    int64_t ocap;        // overflow capacity
    int32_t cm;          // move-in capacity per tile
};

// Arguments of one tiled cycle. Front counts are written (plain stores) for
// every tile every cycle and ping-pong; move-in counts are atomic and rotate
// over three arrays (cycle c reads one, appends to the next and clears the
// third), as do the overflow counts. List records are (xi, global id bits).
// Tile extents are powers of two (tsh = log2).
struct TiledArgs {
    const BlockDev *blocks;
    const BlockTiles *btiles;
    const TileDev *tiles;
    int32_t ntiles;
    int32_t nb;
    const void *field;           // single field pointer (nb == 1 calls), or NULL
    const void *const *fields;   // device array [nb] used when field == NULL
    const float4 *in;
    float4 *out;
    const int32_t *front_in;
    int32_t *front_out;
    const int32_t *movein_in;
    int32_t *movein_out;
    int32_t *movein_zero;
    const int32_t *ocnt_in;      // overflow counts (one int each)
    int32_t *ocnt_out;
    int32_t *ocnt_zero;
    int64_t mbase;               // first slot of the move-in regions
    int64_t obase;               // first slot of the overflow region
    int64_t ocap;                // its capacity (all particles)
    int32_t cm;                  // move-in capacity per tile
    float4 *term;
    float4 *clip;
    int32_t *err;                // set to 1 when a bounded wait gives up
    int32_t cycle;
    float dt;
    int32_t tsh[3];              // log2 of the tile extent per axis
    int32_t pitch;               // floats per staged node row
    int32_t box_floats;          // floats of a staged box
    int32_t buf_floats;          // floats per staging buffer (a tile's box)
    int32_t nbuf;                // staging buffers (2..6)
    int32_t inject_stall;        // test hook: CTA 0's first staged tile never completes
};

// Kernel launchers (bto_kernels.cu). Each returns cudaGetLastError().
cudaError_t launch_advect(const AdvectArgs &a, int layout, int nt, int ppt, bool cap, int grid,
                          size_t dyn_smem, cudaStream_t s);
cudaError_t advect_occupancy(int layout, int nt, int ppt, bool cap, bool batched, size_t dyn_smem,
                             int *ctas_per_sm);
// Tiled advection (bto_tiled.cu).
// Staged box of one tile (bytes); pitch and box_floats as in TiledArgs.
size_t tiled_box_bytes(int layout, const int32_t tdim[3], int32_t *pitch, int32_t *box_floats);
// Dynamic shared memory of a CTA with nbuf staging buffers of buffer_bytes.
size_t tiled_smem_bytes(size_t buffer_bytes, int nbuf);
// nt = threads per CTA (128, 256 or 512); ctas_per_sm = resident CTAs at smem.
cudaError_t tiled_prepare(int layout, int nt, size_t smem, int *ctas_per_sm);
// Largest number of box buffers a CTA of the tiled kernel can hold.
int tiled_max_buffers();
cudaError_t launch_advect_tiled(const TiledArgs &a, int layout, int nt, int grid, size_t smem,
                                cudaStream_t s);
cudaError_t launch_seed_tiled(const BlockDev *blocks, int32_t nb, const int32_t *tseed,
                              const int64_t *tslot, int64_t P, float4 *act, int grid, cudaStream_t s);
cudaError_t launch_write_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                    float *ends, uint8_t *valid, int32_t *exit_cycle, int grid,
                                    cudaStream_t s);
cudaError_t launch_gather_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                     const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                     int64_t *cursor, float4 *out, int grid, cudaStream_t s);
cudaError_t launch_count_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                    int64_t *per_block, int grid, cudaStream_t s);

cudaError_t launch_seed(const BlockDev *blocks, const int32_t *gblock, const int32_t *perm,
                        int64_t slots, int group, PartList p, int grid, cudaStream_t s);
cudaError_t launch_write_live(const BlockDev *blocks, const int32_t *gblock, PartList p, int64_t slots,
                              int group, float *ends, uint8_t *valid, int32_t *exit_cycle, int grid,
                              cudaStream_t s, int32_t *err = nullptr);
cudaError_t launch_gather_live(PartList p, const int64_t *dst, int64_t slots, int group, float4 *out,
                               int grid, cudaStream_t s);
cudaError_t launch_ingest(const void *field, const void *const *fields, int b, int64_t nodes, float4 *out,
                          int grid, cudaStream_t s);
cudaError_t launch_stitch(const int32_t S[3], const float origin[3], const float spacing[3], int32_t intervals,
                          const float *const *ends_table, int64_t nq, const float *start, float *path, int grid,
                          cudaStream_t s, bool barycentric);
cudaError_t launch_fill_delaunay(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                 uint8_t *status, int grid, cudaStream_t s);
cudaError_t launch_fill_lattice(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                uint8_t *status, int grid, cudaStream_t s);
cudaError_t launch_write_term(const BlockDev *blocks, int32_t nb, int64_t P, float4 *term,
                              float *seeds, float *ends, uint8_t *valid, int32_t *exit_cycle,
                              int grid, cudaStream_t s, const float4 *clip = nullptr,
                              float *exit_pos = nullptr, float *exit_time = nullptr);

}  // namespace bto
