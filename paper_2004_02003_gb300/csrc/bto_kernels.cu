// libbto kernels for sm_103a.
//
//   K2 seed_kernel        lattice seeds in brick order (Sec. 2.3)
//   K3 advect_kernel      one RK4 step per live particle with trilinear
//                         sampling (Sec. 3.1, Eq. 1), closed-box termination
//                         of stage and end points (Sec. 3.1, Sec. 3.3), and
//                         compaction of survivors so that terminated
//                         particles occupy no thread in later cycles
//                         (Sec. 3.1, particle management)
//   K4 write_live_kernel  basis flows of surviving particles (Sec. 2.3)
//      write_term_kernel  seeds and basis flows of terminated particles
//
// Design (GB300): the hot kernel is a gather over the velocity nodes, bound
// by memory traffic, not by arithmetic; there is no dense contraction, so the
// tensor cores are not used. Particles are stored in brick order of their
// seeds (runs of 32 seeds along x, the runs in Morton order) so that the
// lanes of a warp touch few node rows and neighbouring warps neighbouring
// rows (L1/L2 reuse of each node); the 8 corners of a cell stay in
// registers across the four RK4 stages and are reloaded only when a stage
// point lands in another cell; each warp owns groups of 32*PPT particles
// and compacts the survivors of a group inside that group (ballot/popc, no
// barrier, no atomic); the grid is persistent (a multiple of the SM count).
// The post hoc kernels (lattice fill, stitching) are in bto_posthoc.cu.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"
#include "bto_device.cuh"

namespace bto {
namespace {

using namespace dev;

constexpr unsigned kFull = 0xffffffffu;

// Index of the block holding global slot/id i (blocks sorted by base).
__device__ __forceinline__ int find_block(const BlockDev *__restrict__ blocks, int nb, int64_t i) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].base <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// K3: advection cycle. The particle list is cut into groups of G = 32*PPT
// slots; one warp owns a group for the cycle: it advects the group's live
// particles (PPT rounds of 32) and writes them back in place. When none of
// them terminated, only the positions are rewritten, in their slots; when
// some did, the survivors (positions and ids) are compacted, in order, to
// the front of the group. Warps take groups g, g + W, g + 2W, ... (W =
// warps in the grid), so the groups in flight at any time are neighbours
// in brick order. There is no barrier and no atomic: a terminated particle
// only leaves the group's live prefix.
// ---------------------------------------------------------------------------
template <int LAYOUT, int NT, int PPT, bool BATCHED, int MINB>
__global__ void __launch_bounds__(NT, MINB) advect_kernel(const AdvectArgs a) {
    // Programmatic dependent launch: the grid may be scheduled while the
    // previous cycle's grid drains; it reads nothing before that grid has
    // completed and its writes are visible (a no-op when launched without
    // the dependency). Then the next cycle's grid may be scheduled.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int G = 32 * PPT;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
    int cur_b = -1;
    Geo g{};
    float3 s = make_float3(0.f, 0.f, 0.f);
    const void *field = nullptr;
    int64_t idbase = 0;
    int64_t nseeds = 0;
    const PartList P = a.p;

    for (int64_t grp = (((int64_t)blockIdx.x * NT) + threadIdx.x) >> 5; grp < a.ngroups;
         grp += nwarps) {
        int cnt = __ldcg(P.gcnt + grp);
        if (!BTO_IN_BOUNDS(cnt >= 0 && cnt <= G, a.err)) cnt = 0;
        if (cnt == 0) continue;
        const int b = BATCHED ? __ldg(a.gblock + grp * PPT) : 0;
        if (b != cur_b) {
            cur_b = b;
            const BlockDev &B = a.blocks[b];
            field = a.field ? a.field : a.fields[b];
            g = load_geo(B);
            s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
            idbase = B.base;
            nseeds = B.nseeds;
        }
        const int64_t s0 = grp * G;
        float3 r[PPT];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int i = k * 32 + lane;
            const float *u = P.rec + ((s0 >> 5) + k) * 128 + lane;
            r[k] = make_float3(0.f, 0.f, 0.f);
            if (i < cnt) r[k] = make_float3(__ldcs(u), __ldcs(u + 32), __ldcs(u + 64));
        }
        unsigned surv = 0;   // bit k: the lane's particle of round k survived
        bool term = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int i = k * 32 + lane;
            if (i < cnt) {
                float3 x = r[k], q;
                const int failed = rk4_step<LAYOUT>(x, field, g, s, q, a.err);
                if (failed == 0) {
                    r[k] = x;
                    surv |= 1u << k;
                } else {
                    term = true;
                    const int32_t id = __float_as_int(__ldcs(P.rec + ((s0 >> 5) + k) * 128 + 96 + lane));
                    if (BTO_IN_BOUNDS(id >= 0 && id < nseeds, a.err)) {
                        const int64_t gid = idbase + id;
                        __stcs(a.term + gid, make_float4(r[k].x, r[k].y, r[k].z, __int_as_float(a.cycle)));
                        // first outside point and its stage; clipped at the interval end
                        if (a.clip) __stcs(a.clip + gid, make_float4(q.x, q.y, q.z, __int_as_float(failed)));
                    }
                }
            }
        }
        if (!__any_sync(kFull, term)) {
            // nobody left: positions back in their slots, ids untouched
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                float *u = P.rec + ((s0 >> 5) + k) * 128 + lane;
                if (k * 32 + lane < cnt) {
                    __stcs(u, r[k].x);
                    __stcs(u + 32, r[k].y);
                    __stcs(u + 64, r[k].z);
                }
            }
        } else {
            // survivors to the front of the group; every id of the group is
            // read before the first write
            float id[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                id[k] = (surv >> k) & 1u ? __ldcs(P.rec + ((s0 >> 5) + k) * 128 + 96 + lane) : 0.f;
            int kept = 0;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const bool sv = (surv >> k) & 1u;
                const unsigned m = __ballot_sync(kFull, sv);
                if (sv) {
                    float *u = P.rec + part_at(s0 + kept + __popc(m & lt), 0);
                    __stcs(u, r[k].x);
                    __stcs(u + 32, r[k].y);
                    __stcs(u + 64, r[k].z);
                    __stcs(u + 96, id[k]);
                }
                kept += __popc(m);
            }
            if (lane == 0) P.gcnt[grp] = kept;
        }
    }
}

// ---------------------------------------------------------------------------
// K2: seeds. Slot i of block b's region holds the lattice point perm[base + m]
// (m = i - slot_base; brick order of the lattice); positions are the exact
// integers j*s in cell units. Also sets every group's live count.
// ---------------------------------------------------------------------------
__global__ void seed_kernel(const BlockDev *__restrict__ blocks, const int32_t *__restrict__ gblock,
                            const int32_t *__restrict__ perm, int64_t slots, int group, PartList P) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
        const BlockDev &B = blocks[gblock[i / kUnit]];
        const int64_t m = i - B.slot_base;
        if (i % group == 0) {
            const int64_t left = B.nseeds - m;
            P.gcnt[i / group] = (int32_t)(left < 0 ? 0 : (left > group ? group : left));
        }
        if (m >= B.nseeds) continue;
        const int32_t p = perm[B.base + m];
        const int32_t jx = p % B.S[0];
        const int32_t jy = (p / B.S[0]) % B.S[1];
        const int32_t jz = p / (B.S[0] * B.S[1]);
        float *u = P.rec + part_at(i, 0);
        u[0] = (float)(jx * B.stride);
        u[32] = (float)(jy * B.stride);
        u[64] = (float)(jz * B.stride);
        u[96] = __int_as_float(p);
    }
}

// K4a: particles alive at the end of the interval.
__global__ void write_live_kernel(const BlockDev *__restrict__ blocks,
                                  const int32_t *__restrict__ gblock, const PartList P,
                                  int64_t slots, int group, float *__restrict__ ends,
                                  uint8_t *__restrict__ valid, int32_t *__restrict__ exit_cycle,
                                  int32_t *__restrict__ err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
        if (i % group >= P.gcnt[i / group]) continue;
        const BlockDev &B = blocks[gblock[i / kUnit]];
        const float *u = P.rec + part_at(i, 0);
        const int32_t id = __float_as_int(u[96]);
        if (!BTO_IN_BOUNDS(id >= 0 && id < B.nseeds, err)) continue;
        const int64_t gid = B.base + id;
        ends[3 * gid + 0] = fmaf(u[0], B.h[0], B.origin[0]);
        ends[3 * gid + 1] = fmaf(u[32], B.h[1], B.origin[1]);
        ends[3 * gid + 2] = fmaf(u[64], B.h[2], B.origin[2]);
        if (valid) valid[gid] = 1;
        if (exit_cycle) exit_cycle[gid] = -1;
    }
}

// K4b: seeds of every particle, plus end/valid/exit of the terminated ones
// (and, when asked, their clipped exit location and time); clears the
// termination record for the next interval.
__global__ void write_term_kernel(const BlockDev *__restrict__ blocks, int32_t nb, int64_t P,
                                  float4 *__restrict__ term, float *__restrict__ seeds,
                                  float *__restrict__ ends, uint8_t *__restrict__ valid,
                                  int32_t *__restrict__ exit_cycle, const float4 *__restrict__ clip,
                                  float *__restrict__ exit_pos, float *__restrict__ exit_time) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < P; gid += stride) {
        const int b = nb == 1 ? 0 : find_block(blocks, nb, gid);
        const BlockDev &B = blocks[b];
        const int32_t p = (int32_t)(gid - B.base);
        if (seeds) {
            const int32_t jx = p % B.S[0];
            const int32_t jy = (p / B.S[0]) % B.S[1];
            const int32_t jz = p / (B.S[0] * B.S[1]);
            seeds[3 * gid + 0] = fmaf((float)(jx * B.stride), B.h[0], B.origin[0]);
            seeds[3 * gid + 1] = fmaf((float)(jy * B.stride), B.h[1], B.origin[1]);
            seeds[3 * gid + 2] = fmaf((float)(jz * B.stride), B.h[2], B.origin[2]);
        }
        const float4 r = term[gid];
        const int e = __float_as_int(r.w);
        if (e >= 0) {
            if (ends) {
                ends[3 * gid + 0] = fmaf(r.x, B.h[0], B.origin[0]);
                ends[3 * gid + 1] = fmaf(r.y, B.h[1], B.origin[1]);
                ends[3 * gid + 2] = fmaf(r.z, B.h[2], B.origin[2]);
            }
            if (valid) valid[gid] = 0;
            if (exit_cycle) exit_cycle[gid] = e;
            if (clip && (exit_pos || exit_time)) {
                const float4 qs = clip[gid];
                const float4 cl = clip_exit(make_float3((float)B.n[0], (float)B.n[1], (float)B.n[2]),
                                            make_float3(r.x, r.y, r.z), make_float3(qs.x, qs.y, qs.z),
                                            __float_as_int(qs.w), e);
                if (exit_pos) {
                    exit_pos[3 * gid + 0] = fmaf(cl.x, B.h[0], B.origin[0]);
                    exit_pos[3 * gid + 1] = fmaf(cl.y, B.h[1], B.origin[1]);
                    exit_pos[3 * gid + 2] = fmaf(cl.z, B.h[2], B.origin[2]);
                }
                if (exit_time) exit_time[gid] = cl.w;
            }
            term[gid] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        } else if (exit_pos || exit_time) {
            const float nan = __int_as_float(0x7fc00000);
            if (exit_pos) {
                exit_pos[3 * gid + 0] = nan;
                exit_pos[3 * gid + 1] = nan;
                exit_pos[3 * gid + 2] = nan;
            }
            if (exit_time) exit_time[gid] = nan;
        }
    }
}

// Diagnostics: live particles of each group copied to dst[g] + k as
// (xi, block-local id bits).
__global__ void gather_live_kernel(const PartList P, const int64_t *__restrict__ dst, int64_t slots,
                                   int group, float4 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
        const int64_t g = i / group;
        const int k = (int)(i % group);
        if (k < P.gcnt[g]) {
            const float *u = P.rec + part_at(i, 0);
            out[dst[g] + k] = make_float4(u[0], u[32], u[64], u[96]);
        }
    }
}

// H1 ingest: repack one block's F3 field (12 bytes per node) into F4 (16 bytes
// per node, pad 0) so that the advection kernel can gather a node with one
// 16-byte load. Four nodes per thread: three 16-byte loads of 48 contiguous
// bytes, four 16-byte stores (scalar loads when the field is not 16-byte
// aligned and for the last nodes).
__global__ void ingest_f3_f4_kernel(const void *__restrict__ field, const void *const *__restrict__ fields,
                                    int b, int64_t nodes, float4 *__restrict__ out) {
    const float *f = reinterpret_cast<const float *>(field ? field : fields[b]);
    const bool vec = (reinterpret_cast<uintptr_t>(f) & 15u) == 0;
    const int64_t quads = nodes / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += stride) {
        float v[12];
        if (vec) {
            const float4 *p = reinterpret_cast<const float4 *>(f) + 3 * q;
            const float4 a = __ldcs(p), bb = __ldcs(p + 1), c = __ldcs(p + 2);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = bb.x; v[5] = bb.y;
            v[6] = bb.z; v[7] = bb.w; v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = __ldcs(f + 12 * q + k);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) out[4 * q + k] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], 0.f);
    }
    for (int64_t i = quads * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += stride)
        out[i] = make_float4(__ldcs(f + 3 * i), __ldcs(f + 3 * i + 1), __ldcs(f + 3 * i + 2), 0.f);
}

// Each cycle's grid is launched with programmatic stream serialisation, so
// its launch and CTA set-up overlap the previous cycle's tail.
template <int LAYOUT, int NT, int PPT, bool BATCHED, int MINB>
cudaError_t launch_t(const AdvectArgs &a, int grid, size_t dyn, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, advect_kernel<LAYOUT, NT, PPT, BATCHED, MINB>, a);
}

template <int LAYOUT, int NT, int PPT, bool BATCHED, int MINB>
cudaError_t occ_t(size_t dyn, int *n) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        n, advect_kernel<LAYOUT, NT, PPT, BATCHED, MINB>, NT, dyn);
}

// Dispatch over the compiled launch shapes: threads per CTA, particles per
// thread, and whether registers are capped at 80 (768 threads per SM).
#define BTO_SHAPES(X, L, B)                                                                  \
    X(L, 128, 1, B, 1) X(L, 128, 2, B, 1) X(L, 128, 4, B, 1) X(L, 256, 1, B, 1)                \
    X(L, 256, 2, B, 1) X(L, 256, 4, B, 1) X(L, 128, 1, B, 6) X(L, 128, 2, B, 6)                \
    X(L, 128, 4, B, 6) X(L, 256, 1, B, 3) X(L, 256, 2, B, 3) X(L, 256, 4, B, 3)

}  // namespace

BTO_BOUNDS_ACCESSOR(bounds_failures_kernels)

cudaError_t launch_advect(const AdvectArgs &a, int layout, int nt, int ppt, bool cap, int grid,
                          size_t dyn, cudaStream_t s) {
    const bool batched = a.nb > 1;
#define BTO_CASE(L, T, P, B, M)                                                     \
    if (layout == L && nt == T && ppt == P && batched == B && cap == (M > 1))       \
        return launch_t<L, T, P, B, M>(a, grid, dyn, s);
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, true)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, true)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

cudaError_t advect_occupancy(int layout, int nt, int ppt, bool cap, bool batched, size_t dyn,
                             int *n) {
#define BTO_CASE(L, T, P, B, M)                                                     \
    if (layout == L && nt == T && ppt == P && batched == B && cap == (M > 1))       \
        return occ_t<L, T, P, B, M>(dyn, n);
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, true)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, true)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_seed(const BlockDev *blocks, const int32_t *gblock, const int32_t *perm,
                        int64_t slots, int group, PartList p, int grid, cudaStream_t s) {
    seed_kernel<<<grid, 256, 0, s>>>(blocks, gblock, perm, slots, group, p);
    return cudaGetLastError();
}

cudaError_t launch_write_live(const BlockDev *blocks, const int32_t *gblock, PartList p, int64_t slots,
                              int group, float *ends, uint8_t *valid, int32_t *exit_cycle, int grid,
                              cudaStream_t s, int32_t *err) {
    write_live_kernel<<<grid, 256, 0, s>>>(blocks, gblock, p, slots, group, ends, valid, exit_cycle, err);
    return cudaGetLastError();
}

cudaError_t launch_gather_live(PartList p, const int64_t *dst, int64_t slots, int group, float4 *out,
                               int grid, cudaStream_t s) {
    gather_live_kernel<<<grid, 256, 0, s>>>(p, dst, slots, group, out);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const void *field, const void *const *fields, int b, int64_t nodes, float4 *out,
                          int grid, cudaStream_t s) {
    ingest_f3_f4_kernel<<<grid, 256, 0, s>>>(field, fields, b, nodes, out);
    return cudaGetLastError();
}

cudaError_t launch_write_term(const BlockDev *blocks, int32_t nb, int64_t P, float4 *term,
                              float *seeds, float *ends, uint8_t *valid, int32_t *exit_cycle,
                              int grid, cudaStream_t s, const float4 *clip, float *exit_pos,
                              float *exit_time) {
    write_term_kernel<<<grid, 256, 0, s>>>(blocks, nb, P, term, seeds, ends, valid, exit_cycle, clip,
                                           exit_pos, exit_time);
    return cudaGetLastError();
}

}  // namespace bto
