// K3t: tiled advection cycle for sm_103a.
//
// Same step as K3 (one RK4 step per live particle with trilinear sampling,
// Sec. 3.1 and Eq. 1; closed-box termination of every stage and end point,
// Sec. 3.1 and Sec. 3.3; terminated particles leave the live set, Sec. 3.1's
// particle management), organised around the field instead of the particles:
//
//  * each block's cells are cut into tiles; the live particles whose cell
//    lies in a tile at the start of a cycle sit in that tile's two list
//    regions: its front region (the survivors that stayed in the tile) and
//    its move-in region (the survivors that came from other tiles);
//  * a persistent CTA takes the tiles t = blockIdx.x, + gridDim.x, ... One
//    producer warp stages, with bulk asynchronous copies (cp.async.bulk,
//    completion counted in bytes on an mbarrier), the nodes of a tile plus
//    one cell of halo on every side and the tile's particle records into
//    one buffer of a ring of shared-memory buffers, while the consumer
//    warps advect the tiles staged before it. Full and empty mbarriers hand
//    the buffers back and forth; there is no CTA-wide barrier in the loop;
//  * the corners of a cell are read from shared memory; a cell outside the
//    staged box (a particle faster than one cell per step, or one in the
//    overflow region) is gathered from global memory, so results do not
//    depend on the tiling;
//  * a survivor still in its tile is written to the tile's next front
//    region (position from a shared-memory counter); one that moved to
//    another tile is appended to that tile's next move-in region (one
//    global atomic on the destination's counter); a full region sends it
//    to the overflow region, which the CTAs advect after the tiles.
//
// Staged rows: the F3 node row [x0, x1] of (y, z) is copied as the 16-byte
// aligned span that contains it; its first node then sits d = (field_word +
// 3 * node) mod 4 floats into the row's buffer. Reading the 16-byte chunks
// that hold field bytes never leaves the field's pages.
//
// Every wait is bounded: a wait that gives up after about two seconds of SM
// clock raises the context's error word and the CTA's abort flag, after
// which the CTA stops, waits (again bounded) for its copies in flight and
// leaves the tiles it has not finished empty and consistent.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"
#include "bto_device.cuh"

namespace bto {
namespace {

using namespace dev;

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// One bounded try: the thread may be suspended up to about a millisecond
// while the phase is incomplete.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return done != 0;
}

// About two seconds of SM clock.
constexpr long long kWaitCycles = 1ll << 32;

// Bounded wait for a phase inside the tile loop: gives up when the CTA's
// abort flag is up, or after kWaitCycles, in which case it raises both the
// abort flag and the context's error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int32_t *err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Bounded wait used after an abort, for copies still in flight: it ignores
// the abort flag, so it waits up to the full bound for a phase that can
// still complete.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return;
}

__device__ __forceinline__ int find_block(const BlockDev *__restrict__ blocks, int nb, int64_t i) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].base <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ const void *block_field(const TiledArgs &a, int b) {
    return a.field ? a.field : a.fields[b];
}

// Cell source over a staged box, with the global gather as fallback.
template <int LAYOUT>
struct BoxSrc {
    const float *sm;
    const void *field;
    uint32_t nnx, nnxy;
    int lox, loy, loz;
    uint32_t cx, cy, cz;   // cells of the box per axis (staged nodes - 1)
    int my, pitch;         // rows per z plane, floats per row
    uint32_t d0, dy, dz;   // F3 row misalignment: (d0 + j dy + k dz) mod 4 floats
    uint32_t nodes;        // nodes of the block (bounds-checked builds)
    int32_t *err;          // context error word (bounds-checked builds)

    __device__ __forceinline__ void load(int ix, int iy, int iz, uint32_t node, PCell &C) const {
        const uint32_t xo = (uint32_t)(ix - lox), j = (uint32_t)(iy - loy), k = (uint32_t)(iz - loz);
        if (xo < cx && j < cy && k < cz) {
            const int r = (int)j + my * (int)k;
            float e[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = r + (q & 1) + ((q & 2) ? my : 0);
                if (LAYOUT == LAYOUT_F4) {
                    const float4 *p = reinterpret_cast<const float4 *>(sm + row * pitch) + xo;
                    const float4 a0 = p[0], a1 = p[1];
                    e[q][0] = a0.x; e[q][1] = a0.y; e[q][2] = a0.z;
                    e[q][3] = a1.x; e[q][4] = a1.y; e[q][5] = a1.z;
                } else {
                    const uint32_t d = (d0 + (j + (q & 1)) * dy + (k + (q >> 1)) * dz) & 3u;
                    const float *p = sm + row * pitch + d + 3 * xo;
#pragma unroll
                    for (int m = 0; m < 6; ++m) e[q][m] = p[m];
                }
            }
            pcell_set(C, e[0], e[1], e[2], e[3]);
        } else {
            load_pcell_global<LAYOUT>(field, nnx, nnxy, node, C, nodes, err);
        }
    }
};

// A non-empty tile of the CTA's sequence t = blockIdx.x + k * gridDim.x.
struct TileView {
    int t;        // tile
    int nf, nm;   // records in its front part and in its move-in part
};

// A warp's walk over the CTA's tiles, skipping the empty ones. The lanes
// hold the counts of a window of 32 consecutive tiles of the sequence;
// `left` marks the non-empty ones not yet returned. Every warp of the CTA
// walks the same sequence and sees the same tiles.
struct TileWalk {
    int k0;          // sequence index of the window's first tile
    unsigned left;   // non-empty tiles of the window not yet returned
    int nf, nm;      // counts of this lane's tile of the window
};

__device__ __forceinline__ void walk_load(const TiledArgs &a, TileWalk &w, bool write_empty) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x + (w.k0 + lane) * (int)gridDim.x;
    w.nf = 0;
    w.nm = 0;
    if (t < a.ntiles) {
        w.nf = min(max(__ldcg(a.front_in + t), 0), __ldg(&a.tiles[t].capf));
        w.nm = min(max(__ldcg(a.movein_in + t), 0), a.cm);
        // an empty tile holds no survivor at the end of the cycle either
        if (write_empty && w.nf + w.nm == 0) a.front_out[t] = 0;
    }
    w.left = __ballot_sync(kFull, w.nf + w.nm > 0);
}

__device__ __forceinline__ void walk_init(const TiledArgs &a, TileWalk &w, bool write_empty) {
    w.k0 = 0;
    walk_load(a, w, write_empty);
}

// Next non-empty tile of the walk; false at the end of the sequence.
__device__ __forceinline__ bool walk_next(const TiledArgs &a, TileWalk &w, TileView &v, bool write_empty) {
    const int G = gridDim.x;
    while (w.left == 0) {
        w.k0 += 32;
        if (blockIdx.x + w.k0 * G >= a.ntiles) return false;
        walk_load(a, w, write_empty);
    }
    const int p = __ffs(w.left) - 1;
    w.left &= w.left - 1;
    v.t = blockIdx.x + (w.k0 + p) * G;
    v.nf = __shfl_sync(kFull, w.nf, p);
    v.nm = __shfl_sync(kFull, w.nm, p);
    return true;
}

// This warp's share of the copies of tile v into buffer dst: the box rows
// r with r mod nwarps == warp, one per lane. Every lane arrives once on the
// full barrier, announcing the bytes of its own copies first.
template <int LAYOUT>
__device__ __forceinline__ void stage_share(const TiledArgs &a, const TileView &v, float *dst, uint32_t bar,
                                            int warp, int nwarps, bool stall) {
    const int lane = threadIdx.x & 31;
    const TileDev &T = a.tiles[v.t];
    const BlockDev &B = a.blocks[T.b];
    const uint64_t nnx = (uint64_t)B.nn[0], nnxy = (uint64_t)B.nn[0] * (uint64_t)B.nn[1];
    const int m0 = T.hi[0] - T.lo[0] + 1, m1 = T.hi[1] - T.lo[1] + 1, m2 = T.hi[2] - T.lo[2] + 1;
    const uint64_t esz = LAYOUT == LAYOUT_F4 ? 16 : 12;
    const uint64_t n0 = (uint64_t)T.lo[0] + nnx * (uint64_t)T.lo[1] + nnxy * (uint64_t)T.lo[2];
    const uintptr_t fbase = reinterpret_cast<uintptr_t>(a.field ? a.field : a.fields[T.b]) + esz * n0;
    const int rows = m1 * m2;
    uint32_t bytes = 0;
    uintptr_t src[4];
    uint32_t sdst[4], n[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = warp + nwarps * (lane + 32 * q);
        n[q] = 0;
        if (r < rows) {
            const int k = r / m1, j = r - k * m1;
            const uintptr_t lo = fbase + esz * (nnx * (uint64_t)j + nnxy * (uint64_t)k);
            src[q] = lo & ~(uintptr_t)15;
            sdst[q] = smem_u32(dst + (size_t)r * a.pitch);
            n[q] = (uint32_t)(((lo + esz * (uint64_t)m0 + 15) & ~(uintptr_t)15) - src[q]);
            bytes += n[q];
        }
    }
    // test hook: announce 16 bytes that no copy delivers, so that the
    // bounded wait on this buffer runs out (bto_test_wait_timeout)
    if (stall && warp == 0 && lane == 0) bytes += 16;
    mbar_arrive_expect(bar, bytes);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (n[q]) bulk_g2s(sdst[q], reinterpret_cast<const void *>(src[q]), n[q], bar);
}

__device__ __forceinline__ void record_term(const TiledArgs &a, const float4 &r, int failed, float3 q) {
    const int64_t gid = __float_as_int(r.w);
    __stcs(a.term + gid, make_float4(r.x, r.y, r.z, __int_as_float(a.cycle)));
    if (a.clip) __stcs(a.clip + gid, make_float4(q.x, q.y, q.z, __int_as_float(failed)));
}

__device__ __forceinline__ void append_overflow(const TiledArgs &a, const float4 &r) {
    const int o = atomicAdd(a.ocnt_out, 1);
    if ((int64_t)o < a.ocap) __stcs(a.out + a.obase + o, r);
}

// A survivor that left its tile: appended to the move-in region of the
// tile of its new cell (same block), or to the overflow region.
__device__ __forceinline__ void append_mover(const TiledArgs &a, const BlockTiles &bt, const Geo &g,
                                             const float4 &r) {
    int ix, iy, iz;
    float f;
    cell_coord(r.x, g.cmx, ix, f);
    cell_coord(r.y, g.cmy, iy, f);
    cell_coord(r.z, g.cmz, iz, f);
    const int dest = bt.first + (ix >> a.tsh[0]) + bt.nt[0] * ((iy >> a.tsh[1]) + bt.nt[1] * (iz >> a.tsh[2]));
    if (!BTO_IN_BOUNDS(dest >= 0 && dest < a.ntiles, a.err)) return;
    const int q = atomicAdd(a.movein_out + dest, 1);
    if (q < a.cm) __stcs(a.out + a.mbase + (int64_t)dest * a.cm + q, r);
    else append_overflow(a, r);
}

// Overflow particles: gathered from global memory (block from the id); every
// survivor is a mover. Warp w of the grid takes particles w*32 + lane, ...
template <int LAYOUT>
__device__ void advect_overflow(const TiledArgs &a, int nwarps_cta) {
    const int64_t n = min(max((int64_t)__ldcg(a.ocnt_in), (int64_t)0), a.ocap);
    const int64_t w = (int64_t)blockIdx.x * nwarps_cta + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * nwarps_cta * 32;
    for (int64_t i = w * 32 + (threadIdx.x & 31); i < n; i += stride) {
        float4 r = __ldcs(a.in + a.obase + i);
        const int b = a.nb == 1 ? 0 : find_block(a.blocks, a.nb, __float_as_int(r.w));
        const BlockDev &B = a.blocks[b];
        const Geo g = load_geo(B);
        const float3 s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
        float3 x = make_float3(r.x, r.y, r.z), q;
        const int failed = rk4_step<LAYOUT>(x, block_field(a, b), g, s, q, a.err);
        if (failed == 0) {
            r.x = x.x; r.y = x.y; r.z = x.z;
            append_mover(a, a.btiles[b], g, r);
        } else {
            record_term(a, r, failed, q);
        }
    }
}

// Shared memory of a CTA after its nbuf box buffers of buf_floats floats:
// barriers, per-buffer survivor counters and tiles, the abort flag.
constexpr int kMaxBufs = 6;
struct SmemTail {
    unsigned long long full[kMaxBufs];
    unsigned long long empty[kMaxBufs];
    int scount[kMaxBufs];
    int tile[kMaxBufs];
    int abort_flag;
};

// Every warp of the CTA walks the CTA's tiles in the same order, issues its
// share of the copies of the tile nbuf - 1 ahead, and advects its share of
// the particles of the current tile. Buffer of the j-th tile: j mod nbuf;
// its full and empty phases have parity (j / nbuf) & 1. Warp 0 also writes
// each tile's front count once every warp has finished the tile.
template <int LAYOUT, int NW, int MINB>
__global__ void __launch_bounds__(32 * NW, MINB) advect_tiled_kernel(const TiledArgs a) {
    // Programmatic dependent launch: nothing is read or written before the
    // previous cycle's grid has completed and its writes are visible.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(128) float tsm[];
    SmemTail *tail = reinterpret_cast<SmemTail *>(tsm + (size_t)a.nbuf * a.buf_floats);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NB = a.nbuf;
    volatile int *abort_flag = &tail->abort_flag;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NB; ++k) {
            mbar_init(smem_u32(&tail->full[k]), 32 * NW);
            mbar_init(smem_u32(&tail->empty[k]), NW);
            tail->scount[k] = 0;
        }
        tail->abort_flag = 0;
        mbar_fence_init();
    }
    // move-in and overflow counts of the cycle after next start at zero
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < a.ntiles; t += gridDim.x * blockDim.x) a.movein_zero[t] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.ocnt_zero = 0;
    __syncthreads();

    const bool w0 = warp == 0;
    bool stall = a.inject_stall && blockIdx.x == 0;
    TileWalk sw, pw;
    walk_init(a, sw, w0);
    walk_init(a, pw, false);
    int staged = 0;
    for (; staged < NB - 1; ++staged) {
        TileView v;
        if (!walk_next(a, sw, v, w0)) break;
        if (w0 && lane == 0) tail->tile[staged] = v.t;
        stage_share<LAYOUT>(a, v, tsm + (size_t)staged * a.buf_floats, smem_u32(&tail->full[staged]), warp, NW, stall);
        stall = false;
    }
    bool more = staged == NB - 1;   // the staging walk may hold more tiles

    int cur_b = -1;
    Geo g{};
    float3 s = make_float3(0.f, 0.f, 0.f);
    BlockTiles bt{};
    BoxSrc<LAYOUT> src;
    src.pitch = a.pitch;
    const unsigned lt = (1u << lane) - 1u;
    int fin = 0;          // tiles whose front count warp 0 has written
    int off = 0;          // chunks of 32 particles handed out so far, mod NW
    int j = 0;
    bool ok = true;
    for (;; ++j) {
        TileView v;
        if (!walk_next(a, pw, v, false)) break;
        const int b = j % NB;
        if (!mbar_wait(smem_u32(&tail->full[b]), (uint32_t)(j / NB) & 1u, abort_flag, a.err)) { ok = false; break; }
        const TileDev &T = a.tiles[v.t];
        const int tb = T.b;
        if (tb != cur_b) {
            cur_b = tb;
            const BlockDev &B = a.blocks[cur_b];
            g = load_geo(B);
            s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
            bt = a.btiles[cur_b];
            src.field = block_field(a, cur_b);
            src.nnx = g.nnx;
            src.nnxy = g.nnxy;
            src.nodes = g.nodes;
            src.err = a.err;
            src.dy = (3u * g.nnx) & 3u;
            src.dz = (3u * g.nnxy) & 3u;
        }
        src.sm = tsm + (size_t)b * a.buf_floats;
        src.lox = T.lo[0]; src.loy = T.lo[1]; src.loz = T.lo[2];
        src.cx = (uint32_t)(T.hi[0] - T.lo[0]); src.cy = (uint32_t)(T.hi[1] - T.lo[1]);
        src.cz = (uint32_t)(T.hi[2] - T.lo[2]);
        src.my = T.hi[1] - T.lo[1] + 1;
        {
            const uint64_t n0 = (uint64_t)T.lo[0] + g.nnx * ((uint64_t)T.lo[1] + (uint64_t)(g.nnxy / g.nnx) * T.lo[2]);
            src.d0 = (uint32_t)((reinterpret_cast<uintptr_t>(src.field) >> 2) + 3ull * n0) & 3u;
        }
        const float tlx = T.tlo[0], tly = T.tlo[1], tlz = T.tlo[2];
        const float thx = T.thi[0], thy = T.thi[1], thz = T.thi[2];
        const int capf = T.capf;
        const int64_t fbase = T.fbase;
        const float4 *rin_f = a.in + fbase;
        const float4 *rin_m = a.in + a.mbase + (int64_t)v.t * a.cm - v.nf;
        const int n = v.nf + v.nm;
        // chunks of 32 particles go to the warps in turn across tiles, so
        // that a tile smaller than 32 * NW particles leaves the idle warps
        // free to start on the next one
        const int nch = (n + 31) >> 5;
        for (int c = (warp - off + NW) % NW; c < nch; c += NW) {
            const int i = c * 32 + lane;
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            bool home = false, mover = false;
            if (i < n) {
                r = __ldcs(i < v.nf ? rin_f + i : rin_m + i);
                float3 x = make_float3(r.x, r.y, r.z), q;
                const int failed = rk4_step_src(x, src, g, s, q);
                if (failed == 0) {
                    r.x = x.x; r.y = x.y; r.z = x.z;
                    home = x.x >= tlx && x.x < thx && x.y >= tly && x.y < thy && x.z >= tlz && x.z < thz;
                    mover = !home;
                } else {
                    record_term(a, r, failed, q);
                }
            }
            const unsigned hm = __ballot_sync(kFull, home);
            if (hm) {
                const int leader = __ffs(hm) - 1;
                int pos = 0;
                if (lane == leader) pos = atomicAdd(&tail->scount[b], __popc(hm));
                pos = __shfl_sync(kFull, pos, leader) + __popc(hm & lt);
                if (home) {
                    if (pos < capf) __stcs(a.out + fbase + pos, r);
                    else append_overflow(a, r);
                }
            }
            if (mover) append_mover(a, bt, g, r);
        }
        off = (off + nch) % NW;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tail->empty[b]));
        // refill the buffer of tile j - 1 with tile j + NB - 1, once every
        // warp has finished tile j - 1 (warp 0 then writes its front count)
        TileView u;
        if (more && walk_next(a, sw, u, w0)) {
            const int jn = j + NB - 1, bn = jn % NB;
            if (j >= 1) {
                if (!mbar_wait(smem_u32(&tail->empty[bn]), (uint32_t)((j - 1) / NB) & 1u, abort_flag, a.err)) {
                    ok = false;
                    break;
                }
                if (w0 && lane == 0) {
                    a.front_out[tail->tile[bn]] = min(tail->scount[bn], __ldg(&a.tiles[tail->tile[bn]].capf));
                    tail->scount[bn] = 0;
                }
                fin = j;
            }
            if (w0 && lane == 0) tail->tile[bn] = u.t;
            __syncwarp();
            stage_share<LAYOUT>(a, u, tsm + (size_t)bn * a.buf_floats, smem_u32(&tail->full[bn]), warp, NW, false);
            ++staged;
        } else {
            more = false;
        }
    }
    if (ok && w0) {
        // front counts of the last tiles, as every warp finishes them
        for (int jj = fin; jj < j; ++jj) {
            const int bb = jj % NB;
            if (!mbar_wait(smem_u32(&tail->empty[bb]), (uint32_t)(jj / NB) & 1u, abort_flag, a.err)) {
                ok = false;
                break;
            }
            if (lane == 0) a.front_out[tail->tile[bb]] = min(tail->scount[bb], __ldg(&a.tiles[tail->tile[bb]].capf));
        }
    }
    if (!ok || *abort_flag) {
        // Let this warp's copies in flight land before the shared memory is
        // released; warp 0 then leaves every tile of the CTA empty: their
        // particles are lost and the error word says so.
        for (int jj = j; jj < staged; ++jj) mbar_drain(smem_u32(&tail->full[jj % NB]), (uint32_t)(jj / NB) & 1u);
        if (w0)
            for (int t = blockIdx.x + lane * (int)gridDim.x; t < a.ntiles; t += 32 * (int)gridDim.x) a.front_out[t] = 0;
        return;
    }
    advect_overflow<LAYOUT>(a, NW);
}

// Seeds of an interval, straight into the front regions of their tiles:
// slot tslot[i] holds seed tseed[i] (global id) at its lattice position.
__global__ void seed_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb, const int32_t *__restrict__ tseed,
                                  const int64_t *__restrict__ tslot, int64_t P, float4 *__restrict__ act) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const int32_t gid = tseed[i];
        const int b = nb == 1 ? 0 : find_block(blocks, nb, gid);
        const BlockDev &B = blocks[b];
        const int32_t p = (int32_t)(gid - B.base);
        const int32_t jx = p % B.S[0];
        const int32_t jy = (p / B.S[0]) % B.S[1];
        const int32_t jz = p / (B.S[0] * B.S[1]);
        act[tslot[i]] = make_float4((float)(jx * B.stride), (float)(jy * B.stride), (float)(jz * B.stride),
                                    __int_as_float(gid));
    }
}

// Live record at slot i of a tiled list, or false; *tile is the tile whose
// region holds the slot (-1: the overflow region).
__device__ __forceinline__ bool live_slot(const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                          const TileCounts &c, int64_t i, int *tile) {
    if (i < c.mbase) {
        const int t = unit_tile[i / kUnit];
        *tile = t;
        return i - tiles[t].fbase < min(max(c.front[t], 0), tiles[t].capf);
    }
    if (i < c.obase) {
        const int t = (int)((i - c.mbase) / c.cm);
        *tile = t;
        return (i - c.mbase) - (int64_t)t * c.cm < min(max(c.movein[t], 0), c.cm);
    }
    *tile = -1;
    return i - c.obase < min(max((int64_t)*c.ocnt, (int64_t)0), c.ocap);
}

__global__ void write_live_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                        const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                        const float4 *__restrict__ act, const TileCounts c,
                                        float *__restrict__ ends, uint8_t *__restrict__ valid,
                                        int32_t *__restrict__ exit_cycle) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.obase + c.ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, i, &t)) continue;
        const float4 r = act[i];
        const int64_t gid = __float_as_int(r.w);
        const BlockDev &B = blocks[t >= 0 ? tiles[t].b : (nb == 1 ? 0 : find_block(blocks, nb, gid))];
        ends[3 * gid + 0] = fmaf(r.x, B.h[0], B.origin[0]);
        ends[3 * gid + 1] = fmaf(r.y, B.h[1], B.origin[1]);
        ends[3 * gid + 2] = fmaf(r.z, B.h[2], B.origin[2]);
        if (valid) valid[gid] = 1;
        if (exit_cycle) exit_cycle[gid] = -1;
    }
}

// Diagnostics: live particles per block, then copied block by block (order
// inside a block unspecified; the id is stored block-local).
__global__ void count_live_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                        const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                        const float4 *__restrict__ act, const TileCounts c,
                                        unsigned long long *__restrict__ per_block) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.obase + c.ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, i, &t)) continue;
        const int b = t >= 0 ? tiles[t].b : (nb == 1 ? 0 : find_block(blocks, nb, __float_as_int(act[i].w)));
        atomicAdd(per_block + b, 1ull);
    }
}

__global__ void gather_live_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                         const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                         const float4 *__restrict__ act, const TileCounts c,
                                         unsigned long long *__restrict__ cursor, float4 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.obase + c.ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, i, &t)) continue;
        float4 r = act[i];
        const int64_t gid = __float_as_int(r.w);
        const int b = t >= 0 ? tiles[t].b : (nb == 1 ? 0 : find_block(blocks, nb, gid));
        const unsigned long long pos = atomicAdd(cursor + b, 1ull);
        r.w = __int_as_float((int32_t)(gid - blocks[b].base));
        out[pos] = r;
    }
}

// The attribute is a ceiling, not an allocation: it is set to the device's
// opt-in maximum so that contexts with different tile shapes can share the
// kernel; occupancy and launches use each context's own size.
template <int LAYOUT, int NW, int MINB>
cudaError_t tiled_occ(size_t smem, int *n) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(advect_tiled_kernel<LAYOUT, NW, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, advect_tiled_kernel<LAYOUT, NW, MINB>, 32 * NW, smem);
}

// Each cycle's grid is launched with programmatic stream serialisation, so
// its launch and CTA set-up overlap the previous cycle's tail.
template <int LAYOUT, int NW, int MINB>
cudaError_t tiled_launch_t(const TiledArgs &a, int grid, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32 * NW);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, advect_tiled_kernel<LAYOUT, NW, MINB>, a);
}

}  // namespace

BTO_BOUNDS_ACCESSOR(bounds_failures_tiled)

size_t tiled_box_bytes(int layout, const int32_t tdim[3], int32_t *pitch, int32_t *box_floats) {
    const int64_t mx = (int64_t)tdim[0] + 3;
    const int64_t row_bytes = layout == LAYOUT_F4 ? 16 * mx : ((12 * mx + 12 + 15) / 16) * 16;
    const int64_t rows = ((int64_t)tdim[1] + 3) * ((int64_t)tdim[2] + 3);
    *pitch = (int32_t)(row_bytes / 4);
    *box_floats = (int32_t)(row_bytes / 4 * rows);
    return (size_t)(row_bytes * rows);
}

size_t tiled_smem_bytes(size_t buffer_bytes, int nbuf) {
    return buffer_bytes * (size_t)nbuf + sizeof(SmemTail) + 16;
}

// nt = threads per CTA: 128, 256 or 512 (4, 8 or 16 warps, every one both
// staging and advecting).
#define BTO_TILED_SHAPES(X) X(LAYOUT_F3, 128, 4, 3) X(LAYOUT_F3, 256, 8, 2) X(LAYOUT_F3, 512, 16, 1) \
    X(LAYOUT_F4, 128, 4, 3) X(LAYOUT_F4, 256, 8, 2) X(LAYOUT_F4, 512, 16, 1)

cudaError_t tiled_prepare(int layout, int nt, size_t smem, int *ctas_per_sm) {
#define BTO_CASE(L, T, W, M) if (layout == L && nt == T) return tiled_occ<L, W, M>(smem, ctas_per_sm);
    BTO_TILED_SHAPES(BTO_CASE)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_advect_tiled(const TiledArgs &a, int layout, int nt, int grid, size_t smem, cudaStream_t s) {
    if (a.nbuf < 2 || a.nbuf > kMaxBufs) return cudaErrorInvalidValue;
#define BTO_CASE(L, T, W, M) if (layout == L && nt == T) return tiled_launch_t<L, W, M>(a, grid, smem, s);
    BTO_TILED_SHAPES(BTO_CASE)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

int tiled_max_buffers() { return kMaxBufs; }

cudaError_t launch_seed_tiled(const BlockDev *blocks, int32_t nb, const int32_t *tseed, const int64_t *tslot,
                              int64_t P, float4 *act, int grid, cudaStream_t s) {
    seed_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tseed, tslot, P, act);
    return cudaGetLastError();
}

cudaError_t launch_write_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt, float *ends,
                                    uint8_t *valid, int32_t *exit_cycle, int grid, cudaStream_t s) {
    write_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt, ends, valid, exit_cycle);
    return cudaGetLastError();
}

cudaError_t launch_count_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt, int64_t *per_block,
                                    int grid, cudaStream_t s) {
    count_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt,
                                                 reinterpret_cast<unsigned long long *>(per_block));
    return cudaGetLastError();
}

cudaError_t launch_gather_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                     const int32_t *unit_tile, const float4 *act, TileCounts cnt, int64_t *cursor,
                                     float4 *out, int grid, cudaStream_t s) {
    gather_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt,
                                                  reinterpret_cast<unsigned long long *>(cursor), out);
    return cudaGetLastError();
}

}  // namespace bto
