// K3t: tiled advection cycle for sm_103a.
//
// Same step as K3 (one RK4 step per live particle with trilinear sampling,
// Sec. 3.1 and Eq. 1; closed-box termination of every stage and end point,
// Sec. 3.1 and Sec. 3.3; terminated particles leave the live set, Sec. 3.1's
// particle management), organised around the field instead of the particles:
//
//  * each block's cells are cut into tiles; a tile's particles sit in its
//    bucket of list slots;
//  * a persistent CTA takes tiles in turn. For each it stages, with bulk
//    asynchronous copies (cp.async.bulk, completion on an mbarrier), the
//    nodes of the tile plus one cell of halo on every side (the step of a
//    particle moving at most one cell per step stays inside) and the tile's
//    particle records into one buffer of a ring of shared-memory buffers,
//    nbuf tiles ahead of the one being advected;
//  * the corners of a cell are read from shared memory; a cell outside the
//    staged box (a particle faster than one cell per step, or one in the
//    overflow region) is gathered from global memory, so results do not
//    depend on the tiling;
//  * a survivor still in its tile is written to the front of the tile's
//    next bucket (positions from a shared-memory counter); one that moved
//    to another tile is appended from the back of that tile's bucket
//    (warp-aggregated global atomics; see TileCounts); a full bucket sends
//    it to the overflow region, which the CTAs advect after the tiles.
//
// Staged rows: the F3 node row [x0, x1] of (y, z) is copied as the 16-byte
// aligned span that contains it; its first node then sits d = (field_word +
// 3 * node) mod 4 floats into the row's buffer. Reading the 16-byte chunks
// that hold field bytes never leaves the field's pages.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"
#include "bto_device.cuh"

namespace bto {
namespace {

using namespace dev;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBuf = 4;

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

// Bounded wait for a phase: gives up after about two seconds of SM clock, or
// as soon as another warp of the CTA has given up (abort flag); the first to
// give up raises the context's error word.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int32_t *err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 32)) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ int find_block(const BlockDev *__restrict__ blocks, int nb, int64_t i) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].base <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Cell source over a staged box, with the global gather as fallback.
template <int LAYOUT>
struct BoxSrc {
    const float *sm;
    const void *field;
    uint32_t nnx, nnxy;
    int x0, y0, z0, x1, y1, z1;   // staged nodes [x0, x1] x [y0, y1] x [z0, z1]
    int ry, pitch;
    uint32_t d0, dy, dz;          // F3 row offsets: (d0 + j dy + k dz) mod 4 floats

    __device__ __forceinline__ void load(int ix, int iy, int iz, uint32_t node, PCell &C) const {
        if (ix >= x0 && ix < x1 && iy >= y0 && iy < y1 && iz >= z0 && iz < z1) {
            const int j = iy - y0, k = iz - z0, xo = ix - x0;
            float e[4][6];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int b = q & 1, c = q >> 1;
                const int row = (j + b) + ry * (k + c);
                if (LAYOUT == LAYOUT_F4) {
                    const float4 *p = reinterpret_cast<const float4 *>(sm + row * pitch) + xo;
                    const float4 a0 = p[0], a1 = p[1];
                    e[q][0] = a0.x; e[q][1] = a0.y; e[q][2] = a0.z;
                    e[q][3] = a1.x; e[q][4] = a1.y; e[q][5] = a1.z;
                } else {
                    const uint32_t d = (d0 + (uint32_t)(j + b) * dy + (uint32_t)(k + c) * dz) & 3u;
                    const float *p = sm + row * pitch + d + 3 * xo;
#pragma unroll
                    for (int m = 0; m < 6; ++m) e[q][m] = p[m];
                }
            }
            pcell_set(C, e[0], e[1], e[2], e[3]);
        } else {
            load_pcell_global<LAYOUT>(field, nnx, nnxy, node, C);
        }
    }
};

__device__ __forceinline__ const void *block_field(const TiledArgs &a, int b) {
    return a.field ? a.field : a.fields[b];
}

// Particles of tile t (bucket capacity cap) in a list with counts c: front
// part, then back part. The counts are clamped to the bucket, so that no
// access leaves it whatever the counts hold.
__device__ __forceinline__ void tile_parts(const TileCounts &c, int t, int cap, int *nf, int *nm) {
    const int f = min(max(__ldcg(c.front + t), 0), cap);
    *nf = f;
    *nm = min(max(min(__ldcg(c.movein + t), __ldcg(c.lim + t)), 0), cap - f);
}


// Issue the copies of tile t (its staged box, then its particle records:
// front part, back part) into buffer dst; every thread arrives once on bar
// with the bytes of the copies it issued. A tile without particles copies
// nothing (the phase completes on the arrivals alone).
template <int LAYOUT, int NT>
__device__ __forceinline__ void stage_tile(const TiledArgs &a, int t, float *dst, uint32_t bar) {
    const TileDev T = a.tiles[t];
    int nf, nm;
    tile_parts(a.cin, t, T.cap, &nf, &nm);
    if (nf + nm == 0) {
        mbar_arrive(bar);
        return;
    }
    const BlockDev &B = a.blocks[T.b];
    const uint64_t nnx = (uint64_t)B.nn[0], nnxy = (uint64_t)B.nn[0] * (uint64_t)B.nn[1];
    const int ry = T.hi[1] - T.lo[1] + 1, rows = ry * (T.hi[2] - T.lo[2] + 1);
    const float inv_ry = 1.f / (float)ry;
    const uint64_t esz = LAYOUT == LAYOUT_F4 ? 16 : 12;
    const uint64_t mx = (uint64_t)(T.hi[0] - T.lo[0] + 1);
    const uintptr_t fbase = reinterpret_cast<uintptr_t>(block_field(a, T.b)) + esz * (uint64_t)T.n0;
    float *rec = dst + a.box_floats;
    // copy r < rows: staged row r; r == rows, rows + 1: the record ranges.
    // First the bytes this thread will copy (announced on the barrier with
    // its arrival), then the copies.
    auto span = [&](int r, uintptr_t &src, uint32_t &sdst) -> uint32_t {
        if (r < rows) {
            const int k = (int)(((float)r + 0.5f) * inv_ry);
            const int jy = r - k * ry;
            const uintptr_t lo = fbase + esz * (nnx * (uint64_t)jy + nnxy * (uint64_t)k);
            src = lo & ~(uintptr_t)15;
            sdst = smem_u32(dst + (size_t)r * a.pitch);
            return (uint32_t)(((lo + esz * mx + 15) & ~(uintptr_t)15) - src);
        }
        if (r == rows) {
            src = reinterpret_cast<uintptr_t>(a.in + T.base);
            sdst = smem_u32(rec);
            return 16u * (uint32_t)nf;
        }
        src = reinterpret_cast<uintptr_t>(a.in + T.base + T.cap - nm);
        sdst = smem_u32(rec + 4 * nf);
        return 16u * (uint32_t)nm;
    };
    const int ncopies = rows + (a.stage_rec ? 2 : 0);
    uint32_t bytes = 0;
    for (int r = threadIdx.x; r < ncopies; r += NT) {
        uintptr_t src;
        uint32_t sdst;
        bytes += span(r, src, sdst);
    }
    // test hook: CTA 0 announces 16 bytes that no copy delivers, so that its
    // bounded wait runs out (the error path of bto_test_wait_timeout)
    if (a.inject_stall && blockIdx.x == 0 && threadIdx.x == 0) bytes += 16;
    mbar_arrive_expect(bar, bytes);
    for (int r = threadIdx.x; r < ncopies; r += NT) {
        uintptr_t src;
        uint32_t sdst;
        const uint32_t n = span(r, src, sdst);
        if (n) bulk_g2s(sdst, reinterpret_cast<const void *>(src), n, bar);
    }
}

__device__ __forceinline__ void record_term(const TiledArgs &a, const float4 &r, int failed, float3 q) {
    const int64_t gid = __float_as_int(r.w);
    __stcs(a.term + gid, make_float4(r.x, r.y, r.z, __int_as_float(a.cycle)));
    if (a.clip) __stcs(a.clip + gid, make_float4(q.x, q.y, q.z, __int_as_float(failed)));
}

// Tile of a survivor's new cell (same block).
__device__ __forceinline__ int dest_tile(const TiledArgs &a, const BlockTiles &bt, const Geo &g, float x, float y,
                                         float z) {
    const int ix = min(max(__float2int_rd(x), 0), g.nx - 1);
    const int iy = min(max(__float2int_rd(y), 0), g.ny - 1);
    const int iz = min(max(__float2int_rd(z), 0), g.nz - 1);
    return bt.first + (ix >> a.tsh[0]) + bt.nt[0] * ((iy >> a.tsh[1]) + bt.nt[1] * (iz >> a.tsh[2]));
}

// Survivors that left their tile (mover = true on the lanes concerned):
// appended from the back of the destination bucket, beyond the particles
// the destination holds this cycle; overflow when that room is used up.
__device__ __forceinline__ void emit_movers(const TiledArgs &a, bool mover, int dest, const float4 &r) {
    const unsigned mm = __ballot_sync(kFull, mover);
    if (!mover) return;
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(mm, dest);
    const int leader = __ffs(peers) - 1;
    int q = 0;
    if (lane == leader) q = atomicAdd(a.movein_out + dest, __popc(peers));
    q = __shfl_sync(peers, q, leader) + __popc(peers & ((1u << lane) - 1u));
    const int cap = __ldg(&a.tiles[dest].cap);
    int nf, nm;
    tile_parts(a.cin, dest, cap, &nf, &nm);
    if (q < cap - (nf + nm)) {
        __stcs(a.out + __ldg(&a.tiles[dest].base) + (cap - 1 - q), r);
    } else {
        const int o = atomicAdd(a.ocnt_out, 1);
        __stcs(a.out + a.obase + o, r);
    }
}

// Advect the n particles of tile t from its staged buffer. Survivors in
// the tile go to the front of its next bucket through the shared counter.
template <int LAYOUT, int NT>
__device__ __forceinline__ void advect_tile(const TiledArgs &a, int t, const float *buf, int nf, int n, int *scount,
                                            int &cur_b, Geo &g, float3 &s, BlockTiles &bt, BoxSrc<LAYOUT> &src,
                                            uint32_t &fw) {
    const TileDev T = a.tiles[t];
    if (T.b != cur_b) {
        cur_b = T.b;
        const BlockDev &B = a.blocks[cur_b];
        g = load_geo(B);
        s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
        bt = a.btiles[cur_b];
        src.field = block_field(a, cur_b);
        src.nnx = g.nnx;
        src.nnxy = g.nnxy;
        fw = (uint32_t)(reinterpret_cast<uintptr_t>(src.field) >> 2);
        src.dy = (3u * g.nnx) & 3u;
        src.dz = (3u * g.nnxy) & 3u;
    }
    src.sm = buf;
    src.x0 = T.lo[0]; src.y0 = T.lo[1]; src.z0 = T.lo[2];
    src.x1 = T.hi[0]; src.y1 = T.hi[1]; src.z1 = T.hi[2];
    src.ry = T.hi[1] - T.lo[1] + 1;
    src.d0 = (fw + 3u * (uint32_t)T.n0) & 3u;
    const float4 *rec = reinterpret_cast<const float4 *>(buf + a.box_floats);
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < n; i0 += NT) {
        const int i = i0 + threadIdx.x;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        bool home = false, mover = false;
        int dest = -1;
        if (i < n) {
            r = a.stage_rec ? rec[i] : __ldcs(a.in + T.base + (i < nf ? i : T.cap - n + i));
            float3 x = make_float3(r.x, r.y, r.z), q;
            const int failed = rk4_step_src(x, src, g, s, q);
            if (failed == 0) {
                r.x = x.x; r.y = x.y; r.z = x.z;
                dest = dest_tile(a, bt, g, x.x, x.y, x.z);
                home = dest == t;
                mover = !home;
            } else {
                record_term(a, r, failed, q);
            }
        }
        const unsigned hm = __ballot_sync(kFull, home);
        if (hm) {
            const int leader = __ffs(hm) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(scount, __popc(hm));
            pos = __shfl_sync(kFull, pos, leader) + __popc(hm & ((1u << lane) - 1u));
            if (home) __stcs(a.out + T.base + pos, r);
        }
        emit_movers(a, mover, dest, r);
    }
}

// Overflow particles: gathered from global memory (block from the id); every
// survivor is a mover.
template <int LAYOUT, int NT>
__device__ void advect_overflow(const TiledArgs &a) {
    const int64_t n = min(max((int64_t)__ldcg(a.ocnt_in), (int64_t)0), a.ocap);
    for (int64_t i0 = (int64_t)blockIdx.x * NT; i0 < n; i0 += (int64_t)gridDim.x * NT) {
        const int64_t i = i0 + threadIdx.x;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        bool mover = false;
        int dest = -1;
        if (i < n) {
            r = __ldcs(a.in + a.obase + i);
            const int b = a.nb == 1 ? 0 : find_block(a.blocks, a.nb, __float_as_int(r.w));
            const BlockDev &B = a.blocks[b];
            const Geo g = load_geo(B);
            const float3 s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
            float3 x = make_float3(r.x, r.y, r.z), q;
            const int failed = rk4_step<LAYOUT>(x, block_field(a, b), g, s, q);
            if (failed == 0) {
                r.x = x.x; r.y = x.y; r.z = x.z;
                mover = true;
                dest = dest_tile(a, a.btiles[b], g, x.x, x.y, x.z);
            } else {
                record_term(a, r, failed, q);
            }
        }
        emit_movers(a, mover, dest, r);
    }
}

template <int LAYOUT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) advect_tiled_kernel(const TiledArgs a) {
    extern __shared__ __align__(128) float tsm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(tsm + (size_t)a.nbuf * a.buf_floats);
    const uint32_t full0 = smem_u32(bars);
    int *scount = reinterpret_cast<int *>(bars + kMaxBuf);
    if (threadIdx.x == 0) {
        for (int k = 0; k < a.nbuf; ++k) mbar_init(full0 + 8u * k, NT);
        *scount = 0;
        mbar_fence_init();
    }
    // counts of the cycle after next start at zero
    for (int t = blockIdx.x * NT + threadIdx.x; t < a.ntiles; t += gridDim.x * NT) a.movein_zero[t] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.ocnt_zero = 0;
    __syncthreads();

    const int G = gridDim.x;
    for (int k = 0; k < a.nbuf; ++k) {
        const int t = blockIdx.x + k * G;
        if (t < a.ntiles) stage_tile<LAYOUT, NT>(a, t, tsm + (size_t)k * a.buf_floats, full0 + 8u * k);
    }
    int cur_b = -1;
    Geo g{};
    float3 s = make_float3(0.f, 0.f, 0.f);
    BlockTiles bt{};
    BoxSrc<LAYOUT> src;
    src.pitch = a.pitch;
    uint32_t fw = 0;
    volatile int no_abort = 0;
    for (int j = 0, t = blockIdx.x; t < a.ntiles; ++j, t += G) {
        const int buf = j % a.nbuf;
        const uint32_t bar = full0 + 8u * buf;
        const bool ok = __syncthreads_and(mbar_wait(bar, (uint32_t)(j / a.nbuf) & 1u, &no_abort, a.err));
        if (!ok) {
            // the copies of the next tiles are already in flight: wait for
            // them (bounded) before the CTA's shared memory is released
            for (int k = 1; k < a.nbuf && t + k * G < a.ntiles; ++k)
                mbar_wait(full0 + 8u * ((j + k) % a.nbuf), (uint32_t)((j + k) / a.nbuf) & 1u, &no_abort, a.err);
            // this CTA's tiles, from the current one on, are left empty and
            // consistent (their particles are lost; the error word says so)
            for (int t2 = t + threadIdx.x * G; t2 < a.ntiles; t2 += NT * G) {
                a.front_out[t2] = 0;
                a.lim_out[t2] = __ldg(&a.tiles[t2].cap);
            }
            return;
        }
        int nf, nm;
        tile_parts(a.cin, t, __ldg(&a.tiles[t].cap), &nf, &nm);
        float *b = tsm + (size_t)buf * a.buf_floats;
        advect_tile<LAYOUT, NT>(a, t, b, nf, nf + nm, scount, cur_b, g, s, bt, src, fw);
        __syncthreads();
        if (threadIdx.x == 0) {
            a.front_out[t] = *scount;
            a.lim_out[t] = __ldg(&a.tiles[t].cap) - (nf + nm);
            *scount = 0;
        }
        const int tn = t + a.nbuf * G;
        if (tn < a.ntiles) stage_tile<LAYOUT, NT>(a, tn, b, bar);
    }
    advect_overflow<LAYOUT, NT>(a);
}

// Seeds of an interval, straight into the front of their tiles' buckets:
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

// Live record at slot i of a tiled list, or false (tile -1: overflow).
__device__ __forceinline__ bool live_slot(const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                          const TileCounts &c, const int32_t *__restrict__ ocnt, int64_t obase,
                                          int64_t ocap, int64_t i, int *tile) {
    if (i < obase) {
        const int t = unit_tile[i / kUnit];
        const TileDev &T = tiles[t];
        *tile = t;
        int nf, nm;
        tile_parts(c, t, T.cap, &nf, &nm);
        const int64_t k = i - T.base;
        return k < nf || k >= T.cap - nm;
    }
    *tile = -1;
    return i - obase < min(max((int64_t)*ocnt, (int64_t)0), ocap);
}

__global__ void write_live_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                        const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                        const float4 *__restrict__ act, const TileCounts c,
                                        const int32_t *__restrict__ ocnt, int64_t obase, int64_t ocap,
                                        float *__restrict__ ends, uint8_t *__restrict__ valid,
                                        int32_t *__restrict__ exit_cycle) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < obase + ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, ocnt, obase, ocap, i, &t)) continue;
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
                                        const int32_t *__restrict__ ocnt, int64_t obase, int64_t ocap,
                                        unsigned long long *__restrict__ per_block) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < obase + ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, ocnt, obase, ocap, i, &t)) continue;
        const int b = t >= 0 ? tiles[t].b : (nb == 1 ? 0 : find_block(blocks, nb, __float_as_int(act[i].w)));
        atomicAdd(per_block + b, 1ull);
    }
}

__global__ void gather_live_tiled_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                         const TileDev *__restrict__ tiles, const int32_t *__restrict__ unit_tile,
                                         const float4 *__restrict__ act, const TileCounts c,
                                         const int32_t *__restrict__ ocnt, int64_t obase, int64_t ocap,
                                         unsigned long long *__restrict__ cursor, float4 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < obase + ocap; i += stride) {
        int t;
        if (!live_slot(tiles, unit_tile, c, ocnt, obase, ocap, i, &t)) continue;
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
template <int LAYOUT, int NT, int MINB>
cudaError_t tiled_occ(size_t smem, int *n) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(advect_tiled_kernel<LAYOUT, NT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, advect_tiled_kernel<LAYOUT, NT, MINB>, NT, smem);
}

}  // namespace

size_t tiled_box_bytes(int layout, const int32_t tdim[3], int32_t *pitch, int32_t *box_floats) {
    const int64_t mx = (int64_t)tdim[0] + 3;
    const int64_t row_bytes = layout == LAYOUT_F4 ? 16 * mx : ((12 * mx + 12 + 15) / 16) * 16;
    const int64_t rows = ((int64_t)tdim[1] + 3) * ((int64_t)tdim[2] + 3);
    *pitch = (int32_t)(row_bytes / 4);
    *box_floats = (int32_t)(row_bytes / 4 * rows);
    return (size_t)(row_bytes * rows);
}

size_t tiled_smem_bytes(size_t buffer_bytes, int nbuf) {
    return buffer_bytes * (size_t)nbuf + kMaxBuf * sizeof(uint64_t) + 16;
}

cudaError_t tiled_prepare(int layout, int nt, size_t smem, int *ctas_per_sm) {
    if (layout == LAYOUT_F3 && nt == 128) return tiled_occ<LAYOUT_F3, 128, 4>(smem, ctas_per_sm);
    if (layout == LAYOUT_F3 && nt == 256) return tiled_occ<LAYOUT_F3, 256, 2>(smem, ctas_per_sm);
    if (layout == LAYOUT_F4 && nt == 128) return tiled_occ<LAYOUT_F4, 128, 4>(smem, ctas_per_sm);
    if (layout == LAYOUT_F4 && nt == 256) return tiled_occ<LAYOUT_F4, 256, 2>(smem, ctas_per_sm);
    return cudaErrorInvalidValue;
}

cudaError_t launch_advect_tiled(const TiledArgs &a, int layout, int nt, int grid, size_t smem, cudaStream_t s) {
    if (a.nbuf < 2 || a.nbuf > kMaxBuf) return cudaErrorInvalidValue;
    if (layout == LAYOUT_F3 && nt == 128) advect_tiled_kernel<LAYOUT_F3, 128, 4><<<grid, 128, smem, s>>>(a);
    else if (layout == LAYOUT_F3 && nt == 256) advect_tiled_kernel<LAYOUT_F3, 256, 2><<<grid, 256, smem, s>>>(a);
    else if (layout == LAYOUT_F4 && nt == 128) advect_tiled_kernel<LAYOUT_F4, 128, 4><<<grid, 128, smem, s>>>(a);
    else if (layout == LAYOUT_F4 && nt == 256) advect_tiled_kernel<LAYOUT_F4, 256, 2><<<grid, 256, smem, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_seed_tiled(const BlockDev *blocks, int32_t nb, const int32_t *tseed, const int64_t *tslot,
                              int64_t P, float4 *act, int grid, cudaStream_t s) {
    seed_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tseed, tslot, P, act);
    return cudaGetLastError();
}

cudaError_t launch_write_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                    const int32_t *ocnt, int64_t obase, int64_t ocap, float *ends,
                                    uint8_t *valid, int32_t *exit_cycle, int grid, cudaStream_t s) {
    write_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt, ocnt, obase, ocap, ends,
                                                 valid, exit_cycle);
    return cudaGetLastError();
}

cudaError_t launch_count_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                    const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                    const int32_t *ocnt, int64_t obase, int64_t ocap, int64_t *per_block,
                                    int grid, cudaStream_t s) {
    count_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt, ocnt, obase, ocap,
                                                 reinterpret_cast<unsigned long long *>(per_block));
    return cudaGetLastError();
}

cudaError_t launch_gather_live_tiled(const BlockDev *blocks, int32_t nb, const TileDev *tiles,
                                     const int32_t *unit_tile, const float4 *act, TileCounts cnt,
                                     const int32_t *ocnt, int64_t obase, int64_t ocap, int64_t *cursor,
                                     float4 *out, int grid, cudaStream_t s) {
    gather_live_tiled_kernel<<<grid, 256, 0, s>>>(blocks, nb, tiles, unit_tile, act, cnt, ocnt, obase, ocap,
                                                  reinterpret_cast<unsigned long long *>(cursor), out);
    return cudaGetLastError();
}

}  // namespace bto
