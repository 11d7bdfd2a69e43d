// libbto host side: the C ABI declared in include/bto.h.
//
// A context owns, on one device:
//   blocks   [nb] BlockDev          geometry of each block
//   perm     [P] int32              lattice point of each rank in brick order, per block
//   gblock   [slots/32] int32       block of each 32-slot unit of the lists
//   pstate   [4 slots] float        particle list, updated in place every cycle:
//                                   units of 32 slots holding 32 x, 32 y, 32 z
//                                   (cell units), 32 block-local ids
//   gcnt     [slots/group] int32    live particles per group (in place)
//   term     [P] float4             termination record per canonical id: xi, cycle
// Each block's list region is its seed count rounded up to 128 slots. No
// host synchronisation happens on the per-cycle path.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bto.h"
#include "bto_internal.h"

using bto::BlockDev;

struct bto_ctx {
    bto::DevAlloc mem;        // device allocator captured at creation
    int device = 0;
    int sm_count = 0;
    int32_t nb = 0;
    int64_t P = 0;
    int64_t slots = 0;        // list slots (regions rounded up to kRegionAlign)
    int32_t L = 0;            // cycles per interval
    int32_t cycle = 0;        // cycles advanced in the current interval
    int layout = bto::LAYOUT_F3;
    int nt = 128, ppt = 2, ctas_per_sm = 0, grid = 0;
    bool cap = false;         // cap registers at 80 (768 threads per SM)
    size_t dyn_smem = 0;
    std::vector<BlockDev> blocks_h;
    BlockDev *blocks = nullptr;
    int32_t *perm = nullptr;
    int32_t *gblock = nullptr;
    float *pstate = nullptr;      // [4 * slots]: the particle list, units of 32 slots (x, y, z, id)
    int32_t *gcnt = nullptr;      // [slots / 32] live particles per group
    float4 *term = nullptr;
    float4 *clip = nullptr;        // [P] first outside point (xi) and stage per canonical id
    int64_t *diag_dst = nullptr;   // bto_copy_active scratch
    bto_status sticky = BTO_OK;
    // cached interval graph
    cudaGraphExec_t gexec = nullptr;
    const void *const *gtable = nullptr;
    float gdt = 0.f;
    int gshape[5] = {0, 0, 0, 0, 0};
    int gtiling = -1;
    cudaStream_t capture_stream = nullptr;
    // H1 ingest (F3 fields repacked to F4 per block, two buffers in flight)
    bool ingest = false;
    float4 *f4buf[2] = {nullptr, nullptr};
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ing_done[2] = {nullptr, nullptr}, adv_done[2] = {nullptr, nullptr};
    // tiled advection (K3t): per-tile front and move-in regions, overflow region, rotating counts
    bool tiled = false;
    int32_t tdim[3] = {0, 0, 0};
    int tnt = 128, tgrid = 0, tocc = 0;
    size_t tsmem = 0;
    int32_t tpitch = 0, tbox = 0, tbuf = 0, tnbuf = 2, tcap_max = 0, tcm = 0;
    int32_t ntiles = 0;
    int64_t mbase = 0, obase = 0, tslots = 0;
    int tiling_gen = 0;
    bto::TileDev *tiles = nullptr;
    bto::BlockTiles *btiles = nullptr;
    int32_t *unit_tile = nullptr;   // [mbase/32] tile of each 32-slot unit of the front regions
    int32_t *tseed = nullptr;       // [P] global id of the i-th seed
    int64_t *tslot = nullptr;       // [P] its slot
    int32_t *tcnt0 = nullptr;       // [ntiles] seeds per tile
    int32_t *tfront[2] = {nullptr, nullptr};
    int32_t *tmv[3] = {nullptr, nullptr, nullptr};
    int32_t *ocnt = nullptr;        // [3] overflow counts
    float4 *tact[2] = {nullptr, nullptr};
    int32_t *derr = nullptr;        // device error flag (bounded waits)
    int32_t inject_stall = 0;       // test hook: tiled cycles left whose first wait is made to run out
};

namespace {

std::mutex g_alloc_mu;
bto::DevAlloc g_alloc;

}  // namespace

bto::DevAlloc bto::current_allocator() {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

namespace {

bto_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return BTO_OK;
    return e == cudaErrorMemoryAllocation ? BTO_ERR_OOM : BTO_ERR_CUDA;
}

#define BTO_TRY(expr)                                     \
    do {                                                  \
        bto_status st__ = (expr);                         \
        if (st__ != BTO_OK) return st__;                  \
    } while (0)

#define BTO_CUDA(expr)                                    \
    do {                                                  \
        cudaError_t e__ = (expr);                         \
        if (e__ != cudaSuccess) {                         \
            (void)cudaGetLastError();                     \
            return cuda_status(e__);                      \
        }                                                 \
    } while (0)

// Bits of a Morton code: every third bit, starting at bit 0.
uint32_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// Canonical lattice ids in Morton order of (jx, jy, jz).
void morton_order(const int32_t S[3], int32_t *out) {
    const int32_t m = std::max(S[0], std::max(S[1], S[2]));
    int bits = 0;
    while ((1 << bits) < m) ++bits;
    const uint64_t ncode = 1ull << (3 * bits);
    int64_t k = 0;
    for (uint64_t code = 0; code < ncode; ++code) {
        const uint32_t x = compact3(code), y = compact3(code >> 1), z = compact3(code >> 2);
        if ((int32_t)x < S[0] && (int32_t)y < S[1] && (int32_t)z < S[2])
            out[k++] = (int32_t)x + S[0] * ((int32_t)y + S[1] * (int32_t)z);
    }
}

// Canonical lattice ids in brick order: the lattice is cut into bricks of
// bx x by x bz seeds (32 seeds: bx = min(32, Sx rounded up to a power of
// two), then by, then bz), the bricks are taken in Morton order and the
// seeds of a brick x fastest. A warp then holds one run of 32 seeds along x
// where the block is that wide, so each of its corner loads touches the
// node rows of a few cell rows instead of the eight rows of a 4 x 4 x 2
// Morton cube: about 13% more particle-steps per second on 128^3 blocks at
// seed stride 2 and 12% on the uneven batched blocks, measured against
// plain Morton order (bricks 32 x 1 x 1, 16 x 2 x 1, 8 x 4 x 1, 8 x 2 x 2,
// 64 x 1 x 1 and 32 x 2 x 1 were measured; long x runs win).
void brick_order(const int32_t S[3], int32_t *out) {
    auto pow2 = [](int32_t v) { int32_t r = 1; while (r < v) r <<= 1; return r; };
    const int32_t bx = std::min(32, pow2(S[0]));
    const int32_t by = std::min(32 / bx, pow2(S[1]));
    const int32_t bz = std::max(1, 32 / (bx * by));
    const int32_t B[3] = {(S[0] + bx - 1) / bx, (S[1] + by - 1) / by, (S[2] + bz - 1) / bz};
    std::vector<int32_t> bricks((size_t)B[0] * B[1] * B[2]);
    morton_order(B, bricks.data());
    int64_t k = 0;
    for (const int32_t q : bricks) {
        const int32_t qx = q % B[0], qy = (q / B[0]) % B[1], qz = q / (B[0] * B[1]);
        for (int32_t z = qz * bz; z < std::min(S[2], (qz + 1) * bz); ++z)
            for (int32_t y = qy * by; y < std::min(S[1], (qy + 1) * by); ++y)
                for (int32_t x = qx * bx; x < std::min(S[0], (qx + 1) * bx); ++x)
                    out[k++] = x + S[0] * (y + S[1] * z);
    }
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

void free_tiling(bto_ctx *c) {
    c->mem.put(c->tiles);
    c->mem.put(c->btiles);
    c->mem.put(c->unit_tile);
    c->mem.put(c->tseed);
    c->mem.put(c->tslot);
    c->mem.put(c->tcnt0);
    for (int k = 0; k < 2; ++k) c->mem.put(c->tfront[k]);
    for (int k = 0; k < 3; ++k) c->mem.put(c->tmv[k]);
    c->mem.put(c->ocnt);
    c->mem.put(c->tact[0]);
    c->mem.put(c->tact[1]);
    c->tiles = nullptr;
    c->btiles = nullptr;
    c->unit_tile = nullptr;
    c->tseed = nullptr;
    c->tslot = nullptr;
    c->tcnt0 = nullptr;
    for (int k = 0; k < 2; ++k) c->tfront[k] = nullptr;
    for (int k = 0; k < 3; ++k) c->tmv[k] = nullptr;
    c->ocnt = nullptr;
    c->tact[0] = c->tact[1] = nullptr;
    c->tiled = false;
    c->ntiles = 0;
}

void free_ctx(bto_ctx *c) {
    if (!c) return;
    free_tiling(c);
    c->mem.put(c->derr);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->mem.put(c->blocks);
    c->mem.put(c->perm);
    c->mem.put(c->gblock);
    c->mem.put(c->pstate);
    c->mem.put(c->gcnt);
    c->mem.put(c->term);
    c->mem.put(c->clip);
    c->mem.put(c->diag_dst);
    c->mem.put(c->f4buf[0]);
    c->mem.put(c->f4buf[1]);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    for (int k = 0; k < 2; ++k) {
        if (c->ing_done[k]) cudaEventDestroy(c->ing_done[k]);
        if (c->adv_done[k]) cudaEventDestroy(c->adv_done[k]);
    }
    delete c;
}

int group_size(const bto_ctx *c) { return 32 * c->ppt; }

// The particle list from slot `first` on (a block's region for per-block
// launches).
bto::PartList part_list(const bto_ctx *c, int64_t first = 0) {
    bto::PartList p;
    p.rec = c->pstate + 4 * first;   // first is a multiple of 32
    p.gcnt = c->gcnt + first / group_size(c);
    return p;
}

bto_status configure_launch(bto_ctx *c) {
    const bool batched = c->nb > 1;
    c->dyn_smem = 0;
    int occ = 0;
    BTO_CUDA(bto::advect_occupancy(c->layout, c->nt, c->ppt, c->cap, batched, c->dyn_smem, &occ));
    if (occ < 1) return BTO_ERR_UNSUPPORTED;
    const int per_sm = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, occ) : occ;
    // Enough CTAs to fill every SM, never more warps than there are groups.
    const int64_t groups = c->slots / group_size(c);
    const int64_t warps_per_cta = c->nt / 32;
    const int64_t need = (groups + warps_per_cta - 1) / warps_per_cta;
    c->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sm_count * per_sm, need));
    return BTO_OK;
}

void drop_graph(bto_ctx *c) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
}

int aux_grid(const bto_ctx *c) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((c->slots + 255) / 256, (int64_t)c->sm_count * 8));
}

// Counts of the tiled list at the start of cycle c.
bto::TileCounts tile_counts(const bto_ctx *c, int cyc) {
    return bto::TileCounts{c->tfront[cyc & 1], c->tmv[cyc % 3], c->ocnt + cyc % 3, c->mbase, c->obase, c->P, c->tcm};
}

int tiled_aux_grid(const bto_ctx *c) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((c->tslots + 255) / 256, (int64_t)c->sm_count * 8));
}

bto_status seed(bto_ctx *c, cudaStream_t s) {
    if (c->tiled) {
        BTO_CUDA(bto::launch_seed_tiled(c->blocks, c->nb, c->tseed, c->tslot, c->P, c->tact[0], aux_grid(c), s));
        const size_t tb = sizeof(int32_t) * (size_t)c->ntiles;
        BTO_CUDA(cudaMemcpyAsync(c->tfront[0], c->tcnt0, tb, cudaMemcpyDeviceToDevice, s));
        for (int k = 0; k < 3; ++k) BTO_CUDA(cudaMemsetAsync(c->tmv[k], 0, tb, s));
        BTO_CUDA(cudaMemsetAsync(c->ocnt, 0, sizeof(int32_t) * 3, s));
        c->cycle = 0;
        return BTO_OK;
    }
    BTO_CUDA(bto::launch_seed(c->blocks, c->gblock, c->perm, c->slots, group_size(c), part_list(c),
                              aux_grid(c), s));
    c->cycle = 0;
    return BTO_OK;
}

// Launch configuration of the tiled kernel for the current layout: one
// CTA of 16 warps per SM (two of 8, four of 4), each with as many box
// buffers (2..6) as fit in its share of the SM's shared memory.
bto_status configure_tiled(bto_ctx *c) {
    const size_t box = bto::tiled_box_bytes(c->layout, c->tdim, &c->tpitch, &c->tbox);
    int optin = 0, per_sm = 0;
    BTO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    BTO_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
    const int want_ctas = std::max(1, 512 / c->tnt);
    const size_t room = std::min<size_t>((size_t)optin, (size_t)per_sm / want_ctas - 1024);
    c->tbuf = (int32_t)(box / 4);
    int nbuf = bto::tiled_max_buffers();
    while (nbuf > 2 && bto::tiled_smem_bytes(box, nbuf) > room) --nbuf;
    const size_t smem = bto::tiled_smem_bytes(box, nbuf);
    if (smem > (size_t)optin) return BTO_ERR_UNSUPPORTED;
    int occ = 0;
    BTO_CUDA(bto::tiled_prepare(c->layout, c->tnt, smem, &occ));
    if (occ < 1) return BTO_ERR_UNSUPPORTED;
    c->tsmem = smem;
    c->tnbuf = nbuf;
    c->tocc = occ;
    c->tgrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sm_count * occ, c->ntiles));
    return BTO_OK;
}

// Tiles of every block, the seeds' front regions (the seeds of a tile in
// brick order of the block's lattice) and the device arrays of the tiled
// path. Front capacity: the tile's seeds plus a quarter (at least 32),
// rounded up to 32; move-in capacity: the same margin for the tile with the
// most seeds, for every tile.
bto_status build_tiling(bto_ctx *c, const int32_t td[3], int nt) {
    std::vector<bto::TileDev> tiles;
    std::vector<bto::BlockTiles> bt((size_t)c->nb);
    for (int32_t b = 0; b < c->nb; ++b) {
        const BlockDev &B = c->blocks_h[(size_t)b];
        int32_t ntl[3];
        for (int a = 0; a < 3; ++a) ntl[a] = (B.n[a] + td[a] - 1) / td[a];
        if ((int64_t)tiles.size() + (int64_t)ntl[0] * ntl[1] * ntl[2] > (1ll << 26)) return BTO_ERR_UNSUPPORTED;
        bt[(size_t)b].first = (int32_t)tiles.size();
        for (int a = 0; a < 3; ++a) bt[(size_t)b].nt[a] = ntl[a];
        for (int32_t z = 0; z < ntl[2]; ++z)
            for (int32_t y = 0; y < ntl[1]; ++y)
                for (int32_t x = 0; x < ntl[0]; ++x) {
                    bto::TileDev T{};
                    T.b = b;
                    const int32_t k[3] = {x, y, z};
                    for (int a = 0; a < 3; ++a) {
                        const int32_t c0 = k[a] * td[a], tn = std::min(td[a], B.n[a] - c0);
                        T.lo[a] = std::max(c0 - 1, 0);
                        T.hi[a] = std::min(c0 + tn + 1, B.n[a]);
                        T.tlo[a] = (float)c0;
                        T.thi[a] = k[a] + 1 < ntl[a] ? (float)(c0 + tn) : INFINITY;
                    }
                    tiles.push_back(T);
                }
    }
    const int64_t ntiles = (int64_t)tiles.size();
    std::vector<int32_t> count((size_t)ntiles, 0);
    std::vector<int32_t> tile_of((size_t)c->P);
    std::vector<int32_t> order;
    for (int32_t b = 0; b < c->nb; ++b) {
        const BlockDev &B = c->blocks_h[(size_t)b];
        order.resize((size_t)B.nseeds);
        brick_order(B.S, order.data());
        const bto::BlockTiles &T = bt[(size_t)b];
        for (int64_t m = 0; m < B.nseeds; ++m) {
            const int32_t p = order[(size_t)m];
            const int32_t j[3] = {p % B.S[0], (p / B.S[0]) % B.S[1], p / (B.S[0] * B.S[1])};
            int32_t k[3];
            for (int a = 0; a < 3; ++a) k[a] = std::min(j[a] * B.stride, B.n[a] - 1) / td[a];
            const int32_t t = T.first + k[0] + T.nt[0] * (k[1] + T.nt[1] * k[2]);
            tile_of[(size_t)(B.base + m)] = t;
            ++count[(size_t)t];
        }
    }
    auto margin = [](int64_t n) { return (n + std::max<int64_t>(n / 4, 32) + 31) / 32 * 32; };
    int64_t base = 0, seeds_max = 0;
    int32_t cap_max = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t capf = margin(count[(size_t)t]);
        tiles[(size_t)t].capf = (int32_t)capf;
        tiles[(size_t)t].fbase = base;
        base += capf;
        cap_max = std::max(cap_max, (int32_t)capf);
        seeds_max = std::max<int64_t>(seeds_max, count[(size_t)t]);
    }
    const int64_t cm = margin(seeds_max) - seeds_max;
    const int64_t mbase = base, obase = mbase + ntiles * cm, tslots = obase + c->P;
    std::vector<int32_t> unit_tile((size_t)(mbase / bto::kUnit));
    for (int64_t t = 0; t < ntiles; ++t)
        for (int64_t u = tiles[(size_t)t].fbase / bto::kUnit; u < (tiles[(size_t)t].fbase + tiles[(size_t)t].capf) / bto::kUnit; ++u)
            unit_tile[(size_t)u] = (int32_t)t;
    std::vector<int32_t> fill((size_t)ntiles, 0);
    std::vector<int32_t> tseed((size_t)c->P);
    std::vector<int64_t> tslot((size_t)c->P);
    for (int32_t b = 0; b < c->nb; ++b) {
        const BlockDev &B = c->blocks_h[(size_t)b];
        order.resize((size_t)B.nseeds);
        brick_order(B.S, order.data());
        for (int64_t m = 0; m < B.nseeds; ++m) {
            const int64_t i = B.base + m;
            const int32_t t = tile_of[(size_t)i];
            tseed[(size_t)i] = (int32_t)(B.base + order[(size_t)m]);
            tslot[(size_t)i] = tiles[(size_t)t].fbase + fill[(size_t)t]++;
        }
    }

    free_tiling(c);
    c->ntiles = (int32_t)ntiles;
    c->mbase = mbase;
    c->obase = obase;
    c->tslots = tslots;
    cudaError_t e = c->mem.get(&c->tiles, sizeof(bto::TileDev) * (size_t)ntiles);
    if (e == cudaSuccess) e = c->mem.get(&c->btiles, sizeof(bto::BlockTiles) * (size_t)c->nb);
    if (e == cudaSuccess) e = c->mem.get(&c->unit_tile, sizeof(int32_t) * std::max<size_t>(1, unit_tile.size()));
    if (e == cudaSuccess) e = c->mem.get(&c->tseed, sizeof(int32_t) * (size_t)c->P);
    if (e == cudaSuccess) e = c->mem.get(&c->tslot, sizeof(int64_t) * (size_t)c->P);
    const size_t tb = sizeof(int32_t) * (size_t)ntiles;
    if (e == cudaSuccess) e = c->mem.get(&c->tcnt0, tb);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = c->mem.get(&c->tfront[k], tb);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = c->mem.get(&c->tmv[k], tb);
    if (e == cudaSuccess) e = c->mem.get(&c->ocnt, sizeof(int32_t) * 4);
    if (e == cudaSuccess) e = c->mem.get(&c->tact[0], sizeof(float4) * (size_t)tslots);
    if (e == cudaSuccess) e = c->mem.get(&c->tact[1], sizeof(float4) * (size_t)tslots);
    if (e == cudaSuccess) e = cudaMemcpy(c->tiles, tiles.data(), sizeof(bto::TileDev) * (size_t)ntiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->btiles, bt.data(), sizeof(bto::BlockTiles) * (size_t)c->nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !unit_tile.empty())
        e = cudaMemcpy(c->unit_tile, unit_tile.data(), sizeof(int32_t) * unit_tile.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->tseed, tseed.data(), sizeof(int32_t) * (size_t)c->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->tslot, tslot.data(), sizeof(int64_t) * (size_t)c->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->tcnt0, count.data(), tb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { (void)cudaGetLastError(); free_tiling(c); return cuda_status(e); }
    for (int a = 0; a < 3; ++a) c->tdim[a] = td[a];
    c->tnt = nt;
    c->tcap_max = cap_max;
    c->tcm = (int32_t)cm;
    c->tiled = true;
    bto_status st = configure_tiled(c);
    if (st != BTO_OK) { free_tiling(c); return st; }
    return BTO_OK;
}

bto_status create_impl(int32_t nb, const int32_t *extents, const float *origins,
                       const float *spacings, const int32_t *strides, int32_t L, bto_ctx **out) {
    if (!out || !extents || !origins || !spacings || !strides) return BTO_ERR_INVALID_ARG;
    if (nb < 1 || nb > 8192 || L < 1) return BTO_ERR_INVALID_ARG;
    std::vector<BlockDev> bl((size_t)nb);
    int64_t P = 0;
    for (int32_t b = 0; b < nb; ++b) {
        BlockDev &B = bl[(size_t)b];
        std::memset(&B, 0, sizeof(B));
        int64_t nodes = 1;
        const int32_t s = strides[b];
        if (s < 1) return BTO_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a) {
            const int32_t n = extents[3 * b + a];
            const float o = origins[3 * b + a], h = spacings[3 * b + a];
            if (n < 1 || !std::isfinite(o) || !finite_pos(h)) return BTO_ERR_INVALID_ARG;
            // cell coordinates must stay exact integers at every node
            if (n > (1 << 23)) return BTO_ERR_INVALID_ARG;
            B.n[a] = n;
            B.nn[a] = n + 1;
            B.S[a] = (n + s - 1) / s;
            B.inv_h[a] = 1.0f / h;
            B.origin[a] = o;
            B.h[a] = h;
            nodes *= (int64_t)(n + 1);
        }
        if (nodes > (1ll << 29)) return BTO_ERR_INVALID_ARG;
        B.stride = s;
        B.nseeds = (int64_t)B.S[0] * B.S[1] * B.S[2];
        if (B.nseeds > (1ll << 30)) return BTO_ERR_INVALID_ARG;
        B.base = P;
        P += B.nseeds;
    }
    if (P > (1ll << 31) - 1) return BTO_ERR_INVALID_ARG;
    int64_t slots = 0;
    for (int32_t b = 0; b < nb; ++b) {
        bl[(size_t)b].slot_base = slots;
        slots += (bl[(size_t)b].nseeds + bto::kRegionAlign - 1) / bto::kRegionAlign * bto::kRegionAlign;
    }
    std::vector<int32_t> gblock((size_t)(slots / bto::kUnit));
    for (int32_t b = 0; b < nb; ++b) {
        const int64_t end = b + 1 < nb ? bl[(size_t)b + 1].slot_base : slots;
        for (int64_t u = bl[(size_t)b].slot_base / bto::kUnit; u < end / bto::kUnit; ++u) gblock[(size_t)u] = b;
    }

    bto_ctx *c = new (std::nothrow) bto_ctx();
    if (!c) return BTO_ERR_OOM;
    c->mem = bto::current_allocator();
    c->nb = nb;
    c->P = P;
    c->slots = slots;
    c->L = L;
    c->blocks_h = bl;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) { (void)cudaGetLastError(); free_ctx(c); return cuda_status(e); }

    std::vector<int32_t> perm((size_t)P);
    for (int32_t b = 0; b < nb; ++b) brick_order(bl[(size_t)b].S, perm.data() + bl[(size_t)b].base);

    const size_t units = (size_t)(slots / bto::kUnit);
    e = c->mem.get(&c->blocks, sizeof(BlockDev) * (size_t)nb);
    if (e == cudaSuccess) e = c->mem.get(&c->perm, sizeof(int32_t) * (size_t)P);
    if (e == cudaSuccess) e = c->mem.get(&c->gblock, sizeof(int32_t) * units);
    if (e == cudaSuccess) e = c->mem.get(&c->pstate, 4 * sizeof(float) * (size_t)slots);
    if (e == cudaSuccess) e = c->mem.get(&c->gcnt, sizeof(int32_t) * units);
    if (e == cudaSuccess) e = c->mem.get(&c->term, sizeof(float4) * (size_t)P);
    if (e == cudaSuccess) e = c->mem.get(&c->clip, sizeof(float4) * (size_t)P);
    if (e == cudaSuccess) e = c->mem.get(&c->derr, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->derr, 0, sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->blocks, bl.data(), sizeof(BlockDev) * (size_t)nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->perm, perm.data(), sizeof(int32_t) * (size_t)P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->gblock, gblock.data(), sizeof(int32_t) * units, cudaMemcpyHostToDevice);
    // term records start as "not terminated" (w = -1: all bits set)
    if (e == cudaSuccess) e = cudaMemset(c->term, 0xff, sizeof(float4) * (size_t)P);
    if (e == cudaSuccess) e = cudaMemset(c->gcnt, 0, sizeof(int32_t) * units);
    if (e != cudaSuccess) { (void)cudaGetLastError(); free_ctx(c); return cuda_status(e); }

    bto_status st = configure_launch(c);
    if (st == BTO_OK) st = seed(c, 0);
    if (st == BTO_OK) st = cuda_status(cudaDeviceSynchronize());
    if (st != BTO_OK) { (void)cudaGetLastError(); free_ctx(c); return st; }
    *out = c;
    return BTO_OK;
}

// One cycle with H1 ingest: block by block, the F3 field is repacked into
// an F4 buffer on a side stream while the previous block is advected on the
// caller's stream from the other buffer (events order the two).
bto_status advect_ingest(bto_ctx *c, const void *field, const void *const *fields, float dt,
                         cudaStream_t s) {
    const int cyc = c->cycle;
    const int G = group_size(c);
    const int aux = (int)std::max<int64_t>(1, (int64_t)c->sm_count * 4);
    BTO_CUDA(cudaEventRecord(c->ev_start, s));
    BTO_CUDA(cudaStreamWaitEvent(c->side, c->ev_start, 0));
    for (int32_t b = 0; b < c->nb; ++b) {
        const BlockDev &B = c->blocks_h[(size_t)b];
        const int64_t nodes = (int64_t)B.nn[0] * B.nn[1] * B.nn[2];
        const int k = b & 1;
        if (b >= 2) BTO_CUDA(cudaStreamWaitEvent(c->side, c->adv_done[k], 0));
        BTO_CUDA(bto::launch_ingest(field, fields, b, nodes, c->f4buf[k], aux, c->side));
        BTO_CUDA(cudaEventRecord(c->ing_done[k], c->side));
        BTO_CUDA(cudaStreamWaitEvent(s, c->ing_done[k], 0));
        const int64_t region = (b + 1 < c->nb ? c->blocks_h[(size_t)b + 1].slot_base : c->slots) - B.slot_base;
        bto::AdvectArgs a{};
        a.blocks = c->blocks + b;
        a.gblock = c->gblock;
        a.nb = 1;
        a.cycle = cyc;
        a.field = c->f4buf[k];
        a.fields = nullptr;
        a.p = part_list(c, B.slot_base);
        a.err = c->derr;
        a.ngroups = region / G;
        a.term = c->term;
        a.clip = c->clip;
        a.dt = dt;
        const int64_t need = (a.ngroups + c->nt / 32 - 1) / (c->nt / 32);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(c->grid, need));
        cudaError_t e = bto::launch_advect(a, bto::LAYOUT_F4, c->nt, c->ppt, c->cap, grid, 0, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            c->sticky = cuda_status(e);
            return c->sticky;
        }
        BTO_CUDA(cudaEventRecord(c->adv_done[k], s));
    }
    c->cycle = cyc + 1;
    return BTO_OK;
}

bto_status advect_impl(bto_ctx *c, const void *field, const void *const *fields, float dt,
                       cudaStream_t s) {
    if (!std::isfinite(dt)) return BTO_ERR_INVALID_ARG;
    if (c->cycle >= c->L) return BTO_ERR_STATE;
    if (c->ingest) return advect_ingest(c, field, fields, dt, s);
    const int cyc = c->cycle;
    if (c->tiled) {
        bto::TiledArgs a{};
        a.blocks = c->blocks;
        a.btiles = c->btiles;
        a.tiles = c->tiles;
        a.ntiles = c->ntiles;
        a.nb = c->nb;
        a.field = field;
        a.fields = fields;
        a.in = c->tact[cyc & 1];
        a.out = c->tact[(cyc + 1) & 1];
        a.front_in = c->tfront[cyc & 1];
        a.front_out = c->tfront[(cyc + 1) & 1];
        a.movein_in = c->tmv[cyc % 3];
        a.movein_out = c->tmv[(cyc + 1) % 3];
        a.movein_zero = c->tmv[(cyc + 2) % 3];
        a.ocnt_in = c->ocnt + cyc % 3;
        a.ocnt_out = c->ocnt + (cyc + 1) % 3;
        a.ocnt_zero = c->ocnt + (cyc + 2) % 3;
        a.mbase = c->mbase;
        a.obase = c->obase;
        a.ocap = c->P;
        a.cm = c->tcm;
        a.term = c->term;
        a.clip = c->clip;
        a.err = c->derr;
        a.cycle = cyc;
        a.dt = dt;
        for (int k = 0; k < 3; ++k) {
            int sh = 0;
            while ((1 << sh) < c->tdim[k]) ++sh;
            a.tsh[k] = sh;
        }
        a.pitch = c->tpitch;
        a.box_floats = c->tbox;
        a.buf_floats = c->tbuf;
        a.nbuf = c->tnbuf;
        a.inject_stall = c->inject_stall > 0 ? 1 : 0;
        if (c->inject_stall > 0) --c->inject_stall;
        cudaError_t e = bto::launch_advect_tiled(a, c->layout, c->tnt, c->tgrid, c->tsmem, s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            c->sticky = cuda_status(e);
            return c->sticky;
        }
        c->cycle = cyc + 1;
        return BTO_OK;
    }
    bto::AdvectArgs a{};
    a.blocks = c->blocks;
    a.gblock = c->gblock;
    a.nb = c->nb;
    a.cycle = cyc;
    a.field = field;
    a.fields = fields;
    a.p = part_list(c);
    a.err = c->derr;
    a.ngroups = c->slots / group_size(c);
    a.term = c->term;
    a.clip = c->clip;
    a.dt = dt;
    cudaError_t e = bto::launch_advect(a, c->layout, c->nt, c->ppt, c->cap, c->grid, c->dyn_smem, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        c->sticky = cuda_status(e);
        return c->sticky;
    }
    c->cycle = cyc + 1;
    return BTO_OK;
}

}  // namespace

extern "C" {

bto_status bto_create(const int32_t extent_cells[3], const float origin[3], const float spacing[3],
                      int32_t seed_stride, int32_t interval_cycles, bto_ctx **out) {
    if (!extent_cells || !origin || !spacing) return BTO_ERR_INVALID_ARG;
    return create_impl(1, extent_cells, origin, spacing, &seed_stride, interval_cycles, out);
}

bto_status bto_batch_create(int32_t nb, const int32_t *extents, const float *origins,
                            const float *spacings, const int32_t *strides,
                            int32_t interval_cycles, bto_ctx **out) {
    return create_impl(nb, extents, origins, spacings, strides, interval_cycles, out);
}

bto_status bto_set_field_layout(bto_ctx *ctx, bto_field_layout layout) {
    if (!ctx) return BTO_ERR_INVALID_ARG;
    if (layout != BTO_FIELD_F3_AOS && layout != BTO_FIELD_F4_AOS) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0) return BTO_ERR_STATE;
    if (ctx->ingest && layout != BTO_FIELD_F3_AOS) return BTO_ERR_STATE;
    const int old = ctx->layout;
    ctx->layout = layout == BTO_FIELD_F4_AOS ? bto::LAYOUT_F4 : bto::LAYOUT_F3;
    bto_status st = configure_launch(ctx);
    if (st == BTO_OK && ctx->tiled) st = configure_tiled(ctx);
    if (st != BTO_OK) {
        ctx->layout = old;
        configure_launch(ctx);
        if (ctx->tiled) configure_tiled(ctx);
        return st;
    }
    drop_graph(ctx);
    return BTO_OK;
}

bto_status bto_set_ingest(bto_ctx *ctx, int32_t enable) {
    if (!ctx || (enable != 0 && enable != 1)) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0) return BTO_ERR_STATE;
    if (enable && (ctx->layout != bto::LAYOUT_F3 || ctx->tiled)) return BTO_ERR_STATE;
    if (enable && !ctx->f4buf[0]) {
        int64_t maxn = 0;
        for (const BlockDev &B : ctx->blocks_h)
            maxn = std::max<int64_t>(maxn, (int64_t)B.nn[0] * B.nn[1] * B.nn[2]);
        BTO_CUDA(ctx->mem.get(&ctx->f4buf[0], sizeof(float4) * (size_t)maxn));
        BTO_CUDA(ctx->mem.get(&ctx->f4buf[1], sizeof(float4) * (size_t)maxn));
        BTO_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
        BTO_CUDA(cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
        for (int k = 0; k < 2; ++k) {
            BTO_CUDA(cudaEventCreateWithFlags(&ctx->ing_done[k], cudaEventDisableTiming));
            BTO_CUDA(cudaEventCreateWithFlags(&ctx->adv_done[k], cudaEventDisableTiming));
        }
    }
    ctx->ingest = enable != 0;
    drop_graph(ctx);
    return BTO_OK;
}

int64_t bto_num_seeds(const bto_ctx *ctx) { return ctx ? ctx->P : -1; }

int32_t bto_num_blocks(const bto_ctx *ctx) { return ctx ? ctx->nb : -1; }

bto_status bto_batch_offsets(const bto_ctx *ctx, int64_t *offsets) {
    if (!ctx || !offsets) return BTO_ERR_INVALID_ARG;
    for (int32_t b = 0; b < ctx->nb; ++b) offsets[b] = ctx->blocks_h[(size_t)b].base;
    offsets[ctx->nb] = ctx->P;
    return BTO_OK;
}

bto_status bto_advect_cycle(bto_ctx *ctx, const void *d_field, float dt, bto_stream stream) {
    if (!ctx || !d_field) return BTO_ERR_INVALID_ARG;
    if (ctx->nb != 1) return BTO_ERR_STATE;
    const uintptr_t align = ctx->layout == bto::LAYOUT_F4 ? 16 : 4;
    if (reinterpret_cast<uintptr_t>(d_field) % align) return BTO_ERR_INVALID_ARG;
    return advect_impl(ctx, d_field, nullptr, dt, (cudaStream_t)stream);
}

bto_status bto_batch_advect_cycle(bto_ctx *ctx, const void *const *d_fields, float dt,
                                  bto_stream stream) {
    if (!ctx || !d_fields) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_fields) % alignof(void *)) return BTO_ERR_INVALID_ARG;
    return advect_impl(ctx, nullptr, d_fields, dt, (cudaStream_t)stream);
}

bto_status bto_launch_interval_graph(bto_ctx *ctx, const void *const *d_field_table, float dt,
                                     bto_stream stream) {
    if (!ctx || !d_field_table || !std::isfinite(dt)) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_field_table) % alignof(void *)) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0) return BTO_ERR_STATE;
    if (ctx->ingest) return BTO_ERR_UNSUPPORTED;
    const bool same = ctx->gexec && ctx->gtable == d_field_table && ctx->gdt == dt &&
                      ctx->gshape[0] == ctx->layout && ctx->gshape[1] == ctx->nt &&
                      ctx->gshape[2] == ctx->ppt && ctx->gshape[3] == ctx->grid &&
                      ctx->gshape[4] == (ctx->cap ? 1 : 0) && ctx->gtiling == ctx->tiling_gen;
    if (!same) {
        drop_graph(ctx);
        if (!ctx->capture_stream)
            BTO_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        BTO_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        bto_status st = BTO_OK;
        for (int32_t c = 0; c < ctx->L && st == BTO_OK; ++c)
            st = advect_impl(ctx, nullptr, d_field_table + (size_t)c * ctx->nb, dt,
                             ctx->capture_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
        ctx->cycle = 0;
        if (st != BTO_OK) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            ctx->gexec = nullptr;
            return cuda_status(e);
        }
        ctx->gtable = d_field_table;
        ctx->gdt = dt;
        ctx->gshape[0] = ctx->layout;
        ctx->gshape[1] = ctx->nt;
        ctx->gshape[2] = ctx->ppt;
        ctx->gshape[3] = ctx->grid;
        ctx->gshape[4] = ctx->cap ? 1 : 0;
        ctx->gtiling = ctx->tiling_gen;
    }
    BTO_CUDA(cudaGraphLaunch(ctx->gexec, (cudaStream_t)stream));
    ctx->cycle = ctx->L;
    return BTO_OK;
}

bto_status bto_end_interval_ex(bto_ctx *ctx, float *d_seeds, float *d_ends, uint8_t *d_valid,
                               int32_t *d_exit_cycle, float *d_exit_pos, float *d_exit_time,
                               bto_stream stream) {
    if (!ctx || !d_seeds || !d_ends || !d_valid) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_seeds) % 4 || reinterpret_cast<uintptr_t>(d_ends) % 4 ||
        reinterpret_cast<uintptr_t>(d_exit_cycle) % 4 || reinterpret_cast<uintptr_t>(d_exit_pos) % 4 ||
        reinterpret_cast<uintptr_t>(d_exit_time) % 4)
        return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != ctx->L) return BTO_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = ctx->L;
    const int grid = aux_grid(ctx);
    if (ctx->tiled)
        BTO_CUDA(bto::launch_write_live_tiled(ctx->blocks, ctx->nb, ctx->tiles, ctx->unit_tile, ctx->tact[L & 1],
                                              tile_counts(ctx, L), d_ends, d_valid, d_exit_cycle,
                                              tiled_aux_grid(ctx), s));
    else
        BTO_CUDA(bto::launch_write_live(ctx->blocks, ctx->gblock, part_list(ctx),
                                        ctx->slots, group_size(ctx), d_ends, d_valid, d_exit_cycle,
                                        grid, s, ctx->derr));
    BTO_CUDA(bto::launch_write_term(ctx->blocks, ctx->nb, ctx->P, ctx->term, d_seeds, d_ends,
                                    d_valid, d_exit_cycle, grid, s, ctx->clip, d_exit_pos, d_exit_time));
    return seed(ctx, s);
}

bto_status bto_end_interval(bto_ctx *ctx, float *d_seeds, float *d_ends, uint8_t *d_valid,
                            int32_t *d_exit_cycle, bto_stream stream) {
    return bto_end_interval_ex(ctx, d_seeds, d_ends, d_valid, d_exit_cycle, nullptr, nullptr, stream);
}

bto_status bto_set_launch(bto_ctx *ctx, int32_t threads_per_cta, int32_t particles_per_thread,
                          int32_t ctas_per_sm, int32_t reg_cap) {
    if (!ctx) return BTO_ERR_INVALID_ARG;
    if (threads_per_cta != 128 && threads_per_cta != 256) return BTO_ERR_INVALID_ARG;
    if (particles_per_thread != 1 && particles_per_thread != 2 && particles_per_thread != 4)
        return BTO_ERR_INVALID_ARG;
    if (ctas_per_sm < 0 || ctas_per_sm > 64) return BTO_ERR_INVALID_ARG;
    if (reg_cap != 0 && reg_cap != 1) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0) return BTO_ERR_STATE;
    const int o[4] = {ctx->nt, ctx->ppt, ctx->ctas_per_sm, ctx->cap ? 1 : 0};
    ctx->nt = threads_per_cta;
    ctx->ppt = particles_per_thread;
    ctx->ctas_per_sm = ctas_per_sm;
    ctx->cap = reg_cap != 0;
    bto_status st = configure_launch(ctx);
    if (st != BTO_OK) {
        ctx->nt = o[0]; ctx->ppt = o[1]; ctx->ctas_per_sm = o[2]; ctx->cap = o[3] != 0;
        configure_launch(ctx);
        return st;
    }
    drop_graph(ctx);
    if (o[1] != ctx->ppt) {
        // group counts depend on the group size: seed the interval afresh
        BTO_CUDA(cudaDeviceSynchronize());
        BTO_TRY(seed(ctx, 0));
        BTO_CUDA(cudaDeviceSynchronize());
    }
    return BTO_OK;
}

bto_status bto_set_tiling(bto_ctx *ctx, const int32_t tile_cells[3], int32_t threads_per_cta) {
    if (!ctx) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0) return BTO_ERR_STATE;
    if (!tile_cells || (tile_cells[0] == 0 && tile_cells[1] == 0 && tile_cells[2] == 0)) {
        if (ctx->tiled) {
            BTO_CUDA(cudaDeviceSynchronize());
            free_tiling(ctx);
            ++ctx->tiling_gen;
            drop_graph(ctx);
            BTO_TRY(seed(ctx, 0));
            BTO_CUDA(cudaDeviceSynchronize());
        }
        return BTO_OK;
    }
    for (int a = 0; a < 3; ++a)
        if (tile_cells[a] < 2 || tile_cells[a] > 128 || (tile_cells[a] & (tile_cells[a] - 1)))
            return BTO_ERR_INVALID_ARG;
    if (threads_per_cta != 128 && threads_per_cta != 256 && threads_per_cta != 512) return BTO_ERR_INVALID_ARG;
    if (ctx->ingest) return BTO_ERR_STATE;
    // each lane stages at most four rows of a tile's box
    if ((int64_t)(tile_cells[1] + 3) * (tile_cells[2] + 3) > 4 * (int64_t)threads_per_cta)
        return BTO_ERR_UNSUPPORTED;
    int32_t pitch = 0, box = 0;
    int optin = 0;
    BTO_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    if (bto::tiled_smem_bytes(bto::tiled_box_bytes(ctx->layout, tile_cells, &pitch, &box), 2) > (size_t)optin)
        return BTO_ERR_UNSUPPORTED;
    BTO_CUDA(cudaDeviceSynchronize());
    BTO_TRY(build_tiling(ctx, tile_cells, threads_per_cta));
    ++ctx->tiling_gen;
    drop_graph(ctx);
    BTO_TRY(seed(ctx, 0));
    BTO_CUDA(cudaDeviceSynchronize());
    return BTO_OK;
}

bto_status bto_test_wait_timeout(bto_ctx *ctx, int32_t cycles) {
    if (!ctx || cycles < 0) return BTO_ERR_INVALID_ARG;
    if (!ctx->tiled) return BTO_ERR_STATE;
    ctx->inject_stall = cycles;
    drop_graph(ctx);
    return BTO_OK;
}

bto_status bto_get_tiling(const bto_ctx *ctx, int32_t out[8]) {
    if (!ctx || !out) return BTO_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) out[a] = ctx->tiled ? ctx->tdim[a] : 0;
    out[3] = ctx->tiled ? ctx->tnt : 0;
    out[4] = ctx->tiled ? ctx->tgrid : 0;
    out[5] = ctx->tiled ? ctx->ntiles : 0;
    out[6] = ctx->tiled ? ctx->tnbuf : 0;
    out[7] = ctx->tiled ? 1 : 0;   // particle records are staged with the box
    return BTO_OK;
}

bto_status bto_get_launch(const bto_ctx *ctx, int32_t out[5]) {
    if (!ctx || !out) return BTO_ERR_INVALID_ARG;
    out[0] = ctx->nt;
    out[1] = ctx->ppt;
    out[2] = ctx->ctas_per_sm;
    out[3] = ctx->cap ? 1 : 0;
    out[4] = ctx->grid;
    return BTO_OK;
}

bto_status bto_autotune(bto_ctx *ctx, const void *const *d_field_table, int32_t cycles, float dt,
                        bto_stream stream, int32_t best[5], float ms[12]) {
    if (!ctx || !d_field_table || !std::isfinite(dt)) return BTO_ERR_INVALID_ARG;
    if (cycles < 1 || cycles > ctx->L) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_field_table) % alignof(void *)) return BTO_ERR_INVALID_ARG;
    if (ctx->cycle != 0 || ctx->tiled) return BTO_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int shapes[12][3] = {{128, 1, 0}, {128, 1, 1}, {128, 2, 0}, {128, 2, 1}, {128, 4, 0}, {128, 4, 1},
                               {256, 1, 0}, {256, 1, 1}, {256, 2, 0}, {256, 2, 1}, {256, 4, 0}, {256, 4, 1}};
    const int keep[4] = {ctx->nt, ctx->ppt, ctx->ctas_per_sm, ctx->cap ? 1 : 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BTO_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); (void)cudaGetLastError(); return cuda_status(ce); }
    float best_ms = 0.f;
    int best_k = -1;
    bto_status st = BTO_OK;
    for (int k = 0; k < 12 && st == BTO_OK; ++k) {
        ctx->nt = shapes[k][0];
        ctx->ppt = shapes[k][1];
        ctx->ctas_per_sm = 0;
        ctx->cap = shapes[k][2] != 0;
        st = configure_launch(ctx);
        if (st == BTO_OK) st = seed(ctx, s);
        if (st != BTO_OK) break;
        ce = cudaEventRecord(e0, s);
        for (int32_t c = 0; c < cycles && st == BTO_OK && ce == cudaSuccess; ++c)
            st = advect_impl(ctx, nullptr, d_field_table + (size_t)c * ctx->nb, dt, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float t = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
        if (ce != cudaSuccess) { st = cuda_status(ce); (void)cudaGetLastError(); break; }
        t /= (float)cycles;
        if (ms) ms[k] = t;
        if (best_k < 0 || t < best_ms) { best_ms = t; best_k = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == BTO_OK && best_k >= 0) {
        ctx->nt = shapes[best_k][0];
        ctx->ppt = shapes[best_k][1];
        ctx->ctas_per_sm = 0;
        ctx->cap = shapes[best_k][2] != 0;
    } else {
        ctx->nt = keep[0]; ctx->ppt = keep[1]; ctx->ctas_per_sm = keep[2]; ctx->cap = keep[3] != 0;
    }
    const bto_status st2 = configure_launch(ctx);
    drop_graph(ctx);
    const bto_status st3 = seed(ctx, s);
    BTO_CUDA(cudaStreamSynchronize(s));
    if (st != BTO_OK) return st;
    if (st2 != BTO_OK) return st2;
    if (st3 != BTO_OK) return st3;
    if (best) return bto_get_launch(ctx, best);
    return BTO_OK;
}

bto_status bto_copy_active(bto_ctx *ctx, float *d_out, int32_t *live, bto_stream stream) {
    if (!ctx || !d_out || !live) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_out) % 16) return BTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int cyc = ctx->cycle;
    if (ctx->tiled) {
        // per-block counts, then each block's particles from its offset on
        if (!ctx->diag_dst) BTO_CUDA(ctx->mem.get(&ctx->diag_dst, sizeof(int64_t) * (size_t)std::max<int64_t>(ctx->nb, ctx->slots / 32)));
        BTO_CUDA(cudaMemsetAsync(ctx->diag_dst, 0, sizeof(int64_t) * (size_t)ctx->nb, s));
        BTO_CUDA(bto::launch_count_live_tiled(ctx->blocks, ctx->nb, ctx->tiles, ctx->unit_tile, ctx->tact[cyc & 1],
                                              tile_counts(ctx, cyc), ctx->diag_dst, tiled_aux_grid(ctx), s));
        std::vector<int64_t> cnt((size_t)ctx->nb), start((size_t)ctx->nb);
        BTO_CUDA(cudaMemcpyAsync(cnt.data(), ctx->diag_dst, sizeof(int64_t) * (size_t)ctx->nb, cudaMemcpyDeviceToHost, s));
        BTO_CUDA(cudaStreamSynchronize(s));
        for (int32_t b = 0; b < ctx->nb; ++b) {
            start[(size_t)b] = ctx->blocks_h[(size_t)b].base;
            live[b] = (int32_t)cnt[(size_t)b];
        }
        BTO_CUDA(cudaMemcpyAsync(ctx->diag_dst, start.data(), sizeof(int64_t) * (size_t)ctx->nb, cudaMemcpyHostToDevice, s));
        BTO_CUDA(bto::launch_gather_live_tiled(ctx->blocks, ctx->nb, ctx->tiles, ctx->unit_tile, ctx->tact[cyc & 1],
                                               tile_counts(ctx, cyc), ctx->diag_dst, reinterpret_cast<float4 *>(d_out),
                                               tiled_aux_grid(ctx), s));
        BTO_CUDA(cudaStreamSynchronize(s));
        return BTO_OK;
    }
    const int G = group_size(ctx);
    const int64_t ng = ctx->slots / G;
    std::vector<int32_t> cnt((size_t)ng);
    std::vector<int64_t> dst((size_t)ng);
    BTO_CUDA(cudaMemcpyAsync(cnt.data(), ctx->gcnt, sizeof(int32_t) * (size_t)ng,
                             cudaMemcpyDeviceToHost, s));
    BTO_CUDA(cudaStreamSynchronize(s));
    for (int32_t b = 0; b < ctx->nb; ++b) {
        const BlockDev &B = ctx->blocks_h[(size_t)b];
        const int64_t g0 = B.slot_base / G;
        const int64_t g1 = b + 1 < ctx->nb ? ctx->blocks_h[(size_t)b + 1].slot_base / G : ng;
        int64_t run = B.base;
        for (int64_t g = g0; g < g1; ++g) {
            dst[(size_t)g] = run;
            run += cnt[(size_t)g];
        }
        live[b] = (int32_t)(run - B.base);
    }
    if (!ctx->diag_dst) BTO_CUDA(ctx->mem.get(&ctx->diag_dst, sizeof(int64_t) * (size_t)(ctx->slots / 32)));
    BTO_CUDA(cudaMemcpyAsync(ctx->diag_dst, dst.data(), sizeof(int64_t) * (size_t)ng,
                             cudaMemcpyHostToDevice, s));
    BTO_CUDA(bto::launch_gather_live(part_list(ctx), ctx->diag_dst, ctx->slots,
                                     G, reinterpret_cast<float4 *>(d_out), aux_grid(ctx), s));
    BTO_CUDA(cudaStreamSynchronize(s));
    return BTO_OK;
}

bto_status bto_last_error(bto_ctx *ctx) {
    if (!ctx) return BTO_ERR_INVALID_ARG;
    bto_status st = ctx->sticky;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (st == BTO_OK && e != cudaSuccess) st = cuda_status(e);
    int32_t flag = 0;
    if (e == cudaSuccess && ctx->derr) {
        e = cudaMemcpy(&flag, ctx->derr, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && flag) e = cudaMemset(ctx->derr, 0, sizeof(int32_t));
        if (st == BTO_OK && e != cudaSuccess) st = cuda_status(e);
        if (st == BTO_OK && flag) st = flag == bto::kErrBounds ? BTO_ERR_BOUNDS : BTO_ERR_TIMEOUT;
    }
    ctx->sticky = BTO_OK;
    return st;
}

bto_status bto_fill_lattice(const int32_t lattice[3], const float *d_ends, const uint8_t *d_valid,
                            float *d_out, uint8_t *d_status, bto_stream stream) {
    if (!lattice || !d_ends || !d_valid || !d_out) return BTO_ERR_INVALID_ARG;
    if (lattice[0] < 1 || lattice[1] < 1 || lattice[2] < 1) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_ends) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4)
        return BTO_ERR_INVALID_ARG;
    const int64_t P = (int64_t)lattice[0] * lattice[1] * lattice[2];
    if (P > (1ll << 31) - 1) return BTO_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    BTO_CUDA(cudaGetDevice(&dev));
    BTO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, (int64_t)sms * 8));
    BTO_CUDA(bto::launch_fill_lattice(lattice, d_ends, d_valid, d_out, d_status, grid, (cudaStream_t)stream));
    return BTO_OK;
}

bto_status bto_fill_delaunay(const int32_t lattice[3], const float *d_ends, const uint8_t *d_valid, float *d_out,
                             uint8_t *d_status, bto_stream stream) {
    if (!lattice || !d_ends || !d_valid || !d_out) return BTO_ERR_INVALID_ARG;
    if (lattice[0] < 1 || lattice[1] < 1 || lattice[2] < 1) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_ends) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4)
        return BTO_ERR_INVALID_ARG;
    const int64_t P = (int64_t)lattice[0] * lattice[1] * lattice[2];
    if (P > (1ll << 31) - 1) return BTO_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    BTO_CUDA(cudaGetDevice(&dev));
    BTO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((P + 127) / 128, (int64_t)sms * 16));
    BTO_CUDA(bto::launch_fill_delaunay(lattice, d_ends, d_valid, d_out, d_status, grid, (cudaStream_t)stream));
    return BTO_OK;
}

bto_status bto_stitch_pathlines(const int32_t lattice[3], const float origin[3], const float spacing[3],
                                int32_t intervals, const float *const *d_ends_table, int64_t nq,
                                const float *d_start, float *d_path, bto_stream stream) {
    return bto_stitch_pathlines_ex(lattice, origin, spacing, intervals, d_ends_table, nq, d_start, d_path,
                                   BTO_STITCH_TRILINEAR, stream);
}

bto_status bto_stitch_pathlines_ex(const int32_t lattice[3], const float origin[3], const float spacing[3],
                                   int32_t intervals, const float *const *d_ends_table, int64_t nq,
                                   const float *d_start, float *d_path, int32_t scheme, bto_stream stream) {
    if (scheme != BTO_STITCH_TRILINEAR && scheme != BTO_STITCH_BARYCENTRIC) return BTO_ERR_INVALID_ARG;
    if (!lattice || !origin || !spacing || !d_ends_table || !d_start || !d_path) return BTO_ERR_INVALID_ARG;
    if (intervals < 1 || nq < 1) return BTO_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (lattice[a] < 1 || !std::isfinite(origin[a]) || !finite_pos(spacing[a])) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_ends_table) % alignof(void *) || reinterpret_cast<uintptr_t>(d_start) % 4 ||
        reinterpret_cast<uintptr_t>(d_path) % 4)
        return BTO_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    BTO_CUDA(cudaGetDevice(&dev));
    BTO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nq + 255) / 256, (int64_t)sms * 8));
    BTO_CUDA(bto::launch_stitch(lattice, origin, spacing, intervals, d_ends_table, nq, d_start, d_path, grid,
                                (cudaStream_t)stream, scheme == BTO_STITCH_BARYCENTRIC));
    return BTO_OK;
}

bto_status bto_set_device_allocator(bto_alloc_fn alloc, bto_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return BTO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = free_fn;
    g_alloc.user = alloc ? user : nullptr;
    return BTO_OK;
}

int32_t bto_check_bounds_build(void) {
#ifdef BTO_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

bto_status bto_bounds_failures(uint64_t *count, int32_t reset) {
    if (!count) return BTO_ERR_INVALID_ARG;
    const unsigned long long parts[4] = {bto::bounds_failures_kernels(reset != 0), bto::bounds_failures_tiled(reset != 0),
                                         bto::bounds_failures_posthoc(reset != 0),
                                         bto::bounds_failures_delaunay(reset != 0)};
    uint64_t total = 0;
    for (const unsigned long long v : parts) {
        if (v == ~0ull) {
            (void)cudaGetLastError();
            return BTO_ERR_CUDA;
        }
        total += v;
    }
    *count = total;
    return BTO_OK;
}

const char *bto_status_string(bto_status s) {
    switch (s) {
        case BTO_OK: return "ok";
        case BTO_ERR_INVALID_ARG: return "invalid argument";
        case BTO_ERR_STATE: return "call out of order for the interval state";
        case BTO_ERR_CUDA: return "CUDA error";
        case BTO_ERR_OOM: return "out of memory";
        case BTO_ERR_TIMEOUT: return "bounded device wait timed out";
        case BTO_ERR_UNSUPPORTED: return "unsupported configuration";
        case BTO_ERR_BOUNDS: return "bounds check failed (bounds-checked build)";
    }
    return "unknown status";
}

void bto_destroy(bto_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

}  // extern "C"
