// libbto kernels for sm_103a.
//
//   K2 seed_kernel        lattice seeds in Morton order (Sec. 2.3)
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
// tensor cores are not used. Particles are stored in Morton order of their
// seeds so that neighbouring threads touch neighbouring cells (L1/L2 reuse
// of each node); the 8 corners of a cell stay in registers across the four
// RK4 stages and are reloaded only when a stage point lands in another cell;
// survivors are compacted per chunk of NT*PPT particles with one atomic per
// chunk; the grid is persistent (a multiple of the SM count) and takes
// chunks from an atomic queue in list order.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"

namespace bto {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Trilinear sampling: Eq. (1) along x on the four cell edges, then along y,
// then along z, for each component (Sec. 3.3).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lerp1(float a, float b, float t) { return fmaf(t, b - a, a); }

struct Cell {
    int ix, iy, iz;
    float v[8][3];  // corner (a, b, c) -> index a + 2b + 4c
};

template <int LAYOUT>
__device__ __forceinline__ void load_cell(const void *__restrict__ field, uint32_t nnx,
                                          uint32_t nnxy, int ix, int iy, int iz,
                                          float (&v)[8][3]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const uint32_t node = (uint32_t)ix + nnx * (uint32_t)(iy + b) + nnxy * (uint32_t)(iz + c);
            const int k0 = 2 * b + 4 * c;
            if (LAYOUT == LAYOUT_F4) {
                const float4 *f = reinterpret_cast<const float4 *>(field) + node;
                const float4 a0 = __ldg(f);
                const float4 a1 = __ldg(f + 1);
                v[k0][0] = a0.x; v[k0][1] = a0.y; v[k0][2] = a0.z;
                v[k0 + 1][0] = a1.x; v[k0 + 1][1] = a1.y; v[k0 + 1][2] = a1.z;
            } else {
                const float *f = reinterpret_cast<const float *>(field) + 3ull * node;
                v[k0][0] = __ldg(f + 0); v[k0][1] = __ldg(f + 1); v[k0][2] = __ldg(f + 2);
                v[k0 + 1][0] = __ldg(f + 3); v[k0 + 1][1] = __ldg(f + 4); v[k0 + 1][2] = __ldg(f + 5);
            }
        }
    }
}

__device__ __forceinline__ float3 trilerp(const float (&v)[8][3], float fx, float fy, float fz) {
    float r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float c00 = lerp1(v[0][k], v[1][k], fx);
        const float c10 = lerp1(v[2][k], v[3][k], fx);
        const float c01 = lerp1(v[4][k], v[5][k], fx);
        const float c11 = lerp1(v[6][k], v[7][k], fx);
        const float c0 = lerp1(c00, c10, fy);
        const float c1 = lerp1(c01, c11, fy);
        r[k] = lerp1(c0, c1, fz);
    }
    return make_float3(r[0], r[1], r[2]);
}

// Block geometry held in registers while a chunk is processed.
struct Geo {
    int nx, ny, nz;        // cells
    float fnx, fny, fnz;   // cells as float (closed-box test)
    uint32_t nnx, nnxy;    // node strides
};

__device__ __forceinline__ Geo load_geo(const BlockDev &B) {
    Geo g;
    g.nx = B.n[0]; g.ny = B.n[1]; g.nz = B.n[2];
    g.fnx = (float)g.nx; g.fny = (float)g.ny; g.fnz = (float)g.nz;
    g.nnx = (uint32_t)B.nn[0];
    g.nnxy = (uint32_t)B.nn[0] * (uint32_t)B.nn[1];
    return g;
}

// Closed box [0, n] in cell coordinates; NaN compares false and so is outside.
__device__ __forceinline__ bool inside(const Geo &g, float x, float y, float z) {
    return x >= 0.f && x <= g.fnx && y >= 0.f && y <= g.fny && z >= 0.f && z <= g.fnz;
}

template <int LAYOUT>
__device__ __forceinline__ float3 sample(Cell &C, const void *__restrict__ field, const Geo &g,
                                         float x, float y, float z) {
    // cell index clamp(floor(xi), 0, n-1): the upper face uses the last cell
    const int ix = min(max(__float2int_rd(x), 0), g.nx - 1);
    const int iy = min(max(__float2int_rd(y), 0), g.ny - 1);
    const int iz = min(max(__float2int_rd(z), 0), g.nz - 1);
    if (ix != C.ix || iy != C.iy || iz != C.iz) {
        load_cell<LAYOUT>(field, g.nnx, g.nnxy, ix, iy, iz, C.v);
        C.ix = ix; C.iy = iy; C.iz = iz;
    }
    return trilerp(C.v, x - (float)ix, y - (float)iy, z - (float)iz);
}

// One RK4 step in cell units (s = dt / h per axis). Returns false, leaving x
// unchanged, as soon as a stage point or the end point leaves the block.
template <int LAYOUT>
__device__ __forceinline__ bool rk4_step(float3 &x, const void *__restrict__ field, const Geo &g,
                                         const float3 s) {
    const float3 hs = make_float3(0.5f * s.x, 0.5f * s.y, 0.5f * s.z);
    Cell C;
    C.ix = -1; C.iy = -1; C.iz = -1;
    const float3 k1 = sample<LAYOUT>(C, field, g, x.x, x.y, x.z);
    float px = fmaf(hs.x, k1.x, x.x), py = fmaf(hs.y, k1.y, x.y), pz = fmaf(hs.z, k1.z, x.z);
    if (!inside(g, px, py, pz)) return false;
    const float3 k2 = sample<LAYOUT>(C, field, g, px, py, pz);
    float3 acc = make_float3(k1.x + 2.f * k2.x, k1.y + 2.f * k2.y, k1.z + 2.f * k2.z);
    px = fmaf(hs.x, k2.x, x.x); py = fmaf(hs.y, k2.y, x.y); pz = fmaf(hs.z, k2.z, x.z);
    if (!inside(g, px, py, pz)) return false;
    const float3 k3 = sample<LAYOUT>(C, field, g, px, py, pz);
    acc.x = fmaf(2.f, k3.x, acc.x); acc.y = fmaf(2.f, k3.y, acc.y); acc.z = fmaf(2.f, k3.z, acc.z);
    px = fmaf(s.x, k3.x, x.x); py = fmaf(s.y, k3.y, x.y); pz = fmaf(s.z, k3.z, x.z);
    if (!inside(g, px, py, pz)) return false;
    const float3 k4 = sample<LAYOUT>(C, field, g, px, py, pz);
    acc.x += k4.x; acc.y += k4.y; acc.z += k4.z;
    const float sx6 = s.x * (1.f / 6.f), sy6 = s.y * (1.f / 6.f), sz6 = s.z * (1.f / 6.f);
    px = fmaf(sx6, acc.x, x.x); py = fmaf(sy6, acc.y, x.y); pz = fmaf(sz6, acc.z, x.z);
    if (!inside(g, px, py, pz)) return false;
    x = make_float3(px, py, pz);
    return true;
}

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
// K3: advection cycle. Persistent CTAs take chunks of CH = NT*PPT particles
// of one block from an atomic queue; survivors of a chunk are written as one
// contiguous run at a position reserved with one atomicAdd on the block's
// output count (stable order inside the chunk).
// ---------------------------------------------------------------------------
template <int LAYOUT, int NT, int PPT, bool BATCHED>
__global__ void __launch_bounds__(NT) advect_kernel(const AdvectArgs a) {
    constexpr int NW = NT / 32;
    constexpr int CH = NT * PPT;
    static_assert(PPT * NW <= 32, "per-chunk warp counts must fit one warp scan");
    __shared__ float4 s_buf[CH];
    __shared__ int s_wcnt[PPT * NW];
    __shared__ int s_wofs[PPT * NW];
    __shared__ int s_g, s_base, s_total;
    __shared__ int s_warp_sum[NW];
    extern __shared__ int s_prefix[];  // BATCHED: nb + 1 chunk offsets

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (blockIdx.x == 0) {
        for (int b = tid; b < a.nb; b += NT) a.cnt_zero[b] = 0;
        if (tid == 0) *a.work_zero = 0;
    }

    int total;
    if (BATCHED) {
        // exclusive scan of per-block chunk counts into s_prefix[0..nb]
        const int per = (a.nb + NT - 1) / NT;
        const int b0 = tid * per, b1 = min(a.nb, b0 + per);
        int local = 0;
        for (int b = b0; b < b1; ++b) local += (__ldcg(a.cnt_in + b) + CH - 1) / CH;
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp_sum[warp] = incl;
        __syncthreads();
        int wofs = 0;
        for (int w = 0; w < warp; ++w) wofs += s_warp_sum[w];
        int run = wofs + incl - local;
        for (int b = b0; b < b1; ++b) {
            s_prefix[b] = run;
            run += (__ldcg(a.cnt_in + b) + CH - 1) / CH;
        }
        if (tid == NT - 1) { s_prefix[a.nb] = wofs + incl; s_total = wofs + incl; }
        __syncthreads();
        total = s_total;
    } else {
        total = (__ldcg(a.cnt_in) + CH - 1) / CH;
    }

    int cur_b = -1;
    Geo g{};
    float3 s = make_float3(0.f, 0.f, 0.f);
    const void *field = nullptr;
    int64_t base = 0;
    int Lb = 0;

    for (;;) {
        if (tid == 0) s_g = atomicAdd(a.work, 1);
        __syncthreads();
        const int gi = s_g;
        if (gi >= total) break;
        int b = 0, j = gi;
        if (BATCHED) {
            int lo = 0, hi = a.nb - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_prefix[mid] <= gi) lo = mid; else hi = mid - 1;
            }
            b = lo;
            j = gi - s_prefix[b];
        }
        if (b != cur_b) {
            cur_b = b;
            const BlockDev &B = a.blocks[b];
            g = load_geo(B);
            s = make_float3(a.dt * B.inv_h[0], a.dt * B.inv_h[1], a.dt * B.inv_h[2]);
            base = B.base;
            field = a.field ? a.field : a.fields[b];
            Lb = __ldcg(a.cnt_in + b);
        }

        unsigned mask = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int i = j * CH + k * NT + tid;
            bool surv = false;
            if (i < Lb) {
                const float4 r = __ldcs(a.in + base + i);
                float3 x = make_float3(r.x, r.y, r.z);
                if (rk4_step<LAYOUT>(x, field, g, s)) {
                    s_buf[k * NT + tid] = make_float4(x.x, x.y, x.z, r.w);
                    surv = true;
                } else {
                    const int pid = __float_as_int(r.w);
                    __stcs(a.term + base + pid, make_float4(r.x, r.y, r.z, __int_as_float(a.cycle)));
                }
            }
            const unsigned bal = __ballot_sync(kFull, surv);
            if (lane == 0) s_wcnt[k * NW + warp] = __popc(bal);
            mask |= (unsigned)surv << k;
        }
        __syncthreads();
        if (warp == 0) {
            const int v = lane < PPT * NW ? s_wcnt[lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane < PPT * NW) s_wofs[lane] = incl - v;
            const int tot = __shfl_sync(kFull, incl, 31);
            if (lane == 0) s_base = tot ? atomicAdd(a.cnt_out + b, tot) : 0;
        }
        __syncthreads();
        const int obase = s_base;
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const bool surv = (mask >> k) & 1u;
            const unsigned bal = __ballot_sync(kFull, surv);
            if (surv) {
                const int rank = s_wofs[k * NW + warp] + __popc(bal & lt);
                __stcs(a.out + base + obase + rank, s_buf[k * NT + tid]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K2: seeds. Slot i of block b holds lattice point perm[i] (Morton order of
// the lattice); positions are exact integers j*s in cell units.
// Also initialises the count ring for cycle 0.
// ---------------------------------------------------------------------------
__global__ void seed_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                            const int32_t *__restrict__ perm, int64_t P, float4 *__restrict__ act,
                            int32_t *cnt0, int32_t *cnt1, int32_t *work0) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            cnt0[b] = (int32_t)blocks[b].nseeds;
            cnt1[b] = 0;
        }
        if (threadIdx.x == 0) *work0 = 0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const int b = nb == 1 ? 0 : find_block(blocks, nb, i);
        const BlockDev &B = blocks[b];
        const int32_t p = perm[i];
        const int32_t jx = p % B.S[0];
        const int32_t jy = (p / B.S[0]) % B.S[1];
        const int32_t jz = p / (B.S[0] * B.S[1]);
        act[i] = make_float4((float)(jx * B.stride), (float)(jy * B.stride), (float)(jz * B.stride),
                             __int_as_float(p));
    }
}

// K4a: particles alive at the end of the interval.
__global__ void write_live_kernel(const BlockDev *__restrict__ blocks, int32_t nb,
                                  const float4 *__restrict__ act, const int32_t *__restrict__ cnt,
                                  int64_t P, float *__restrict__ ends, uint8_t *__restrict__ valid,
                                  int32_t *__restrict__ exit_cycle) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const int b = nb == 1 ? 0 : find_block(blocks, nb, i);
        const BlockDev &B = blocks[b];
        if (i - B.base >= (int64_t)cnt[b]) continue;
        const float4 r = act[i];
        const int64_t gid = B.base + __float_as_int(r.w);
        ends[3 * gid + 0] = fmaf(r.x, B.h[0], B.origin[0]);
        ends[3 * gid + 1] = fmaf(r.y, B.h[1], B.origin[1]);
        ends[3 * gid + 2] = fmaf(r.z, B.h[2], B.origin[2]);
        if (valid) valid[gid] = 1;
        if (exit_cycle) exit_cycle[gid] = -1;
    }
}

// K4b: seeds of every particle, plus end/valid/exit of the terminated ones;
// clears the termination record for the next interval.
__global__ void write_term_kernel(const BlockDev *__restrict__ blocks, int32_t nb, int64_t P,
                                  float4 *__restrict__ term, float *__restrict__ seeds,
                                  float *__restrict__ ends, uint8_t *__restrict__ valid,
                                  int32_t *__restrict__ exit_cycle) {
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
            term[gid] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        }
    }
}

template <int LAYOUT, int NT, int PPT, bool BATCHED>
cudaError_t launch_t(const AdvectArgs &a, int grid, size_t dyn, cudaStream_t s) {
    advect_kernel<LAYOUT, NT, PPT, BATCHED><<<grid, NT, dyn, s>>>(a);
    return cudaGetLastError();
}

template <int LAYOUT, int NT, int PPT, bool BATCHED>
cudaError_t occ_t(size_t dyn, int *n) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, advect_kernel<LAYOUT, NT, PPT, BATCHED>,
                                                         NT, dyn);
}

// Dispatch over the compiled launch shapes.
#define BTO_SHAPES(X, L, B)                                                        \
    X(L, 128, 1, B) X(L, 128, 2, B) X(L, 128, 4, B) X(L, 256, 1, B) X(L, 256, 2, B) \
    X(L, 256, 4, B)

}  // namespace

cudaError_t launch_advect(const AdvectArgs &a, int layout, int nt, int ppt, int grid,
                          size_t dyn, cudaStream_t s) {
    const bool batched = a.nb > 1;
#define BTO_CASE(L, T, P, B)                                            \
    if (layout == L && nt == T && ppt == P && batched == B)             \
        return launch_t<L, T, P, B>(a, grid, dyn, s);
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, true)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, true)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

cudaError_t advect_occupancy(int layout, int nt, int ppt, bool batched, size_t dyn, int *n) {
#define BTO_CASE(L, T, P, B)                                            \
    if (layout == L && nt == T && ppt == P && batched == B) return occ_t<L, T, P, B>(dyn, n);
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, false)
    BTO_SHAPES(BTO_CASE, LAYOUT_F3, true)
    BTO_SHAPES(BTO_CASE, LAYOUT_F4, true)
#undef BTO_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_seed(const BlockDev *blocks, int32_t nb, const int32_t *perm, int64_t P,
                        float4 *act, int32_t *cnt0, int32_t *cnt1, int32_t *work0, int grid,
                        cudaStream_t s) {
    seed_kernel<<<grid, 256, 0, s>>>(blocks, nb, perm, P, act, cnt0, cnt1, work0);
    return cudaGetLastError();
}

cudaError_t launch_write_live(const BlockDev *blocks, int32_t nb, const float4 *act,
                              const int32_t *cnt, int64_t P, float *ends, uint8_t *valid,
                              int32_t *exit_cycle, int grid, cudaStream_t s) {
    write_live_kernel<<<grid, 256, 0, s>>>(blocks, nb, act, cnt, P, ends, valid, exit_cycle);
    return cudaGetLastError();
}

cudaError_t launch_write_term(const BlockDev *blocks, int32_t nb, int64_t P, float4 *term,
                              float *seeds, float *ends, uint8_t *valid, int32_t *exit_cycle,
                              int grid, cudaStream_t s) {
    write_term_kernel<<<grid, 256, 0, s>>>(blocks, nb, P, term, seeds, ends, valid, exit_cycle);
    return cudaGetLastError();
}

}  // namespace bto
