// Device functions shared by the advection kernels (bto_kernels.cu) and the
// adjoint kernels (bto_adjoint.cu): trilinear sampling of a block's node
// field and one RK4 step with the closed-box tests, in block-local cell
// coordinates xi = (x - origin) / h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"

namespace bto {
namespace dev {

// ---------------------------------------------------------------------------
// Trilinear sampling: Eq. (1) along x on the four cell edges, then along y,
// then along z, for each component (Sec. 3.3).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lerp1(float a, float b, float t) { return fmaf(t, b - a, a); }


// The 8 corner nodes of cell (ix, iy, iz) as v[a + 2b + 4c][component], for
// the adjoint's sampler, which also differentiates the weights.
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

// Block geometry held in registers while a group is processed.
struct Geo {
    int nx, ny, nz;        // cells
    float fnx, fny, fnz;   // cells as float (closed-box test)
    float cmx, cmy, cmz;   // 2^23 + (cells - 1): the last cell, in the biased form of cell_coord
    uint32_t nnx, nnxy;    // node strides
    uint32_t nodes;        // nodes of the block
};

__device__ __forceinline__ Geo load_geo(const BlockDev &B) {
    Geo g;
    g.nx = B.n[0]; g.ny = B.n[1]; g.nz = B.n[2];
    g.fnx = (float)g.nx; g.fny = (float)g.ny; g.fnz = (float)g.nz;
    g.cmx = 8388608.f + (float)(g.nx - 1);
    g.cmy = 8388608.f + (float)(g.ny - 1);
    g.cmz = 8388608.f + (float)(g.nz - 1);
    g.nnx = (uint32_t)B.nn[0];
    g.nnxy = (uint32_t)B.nn[0] * (uint32_t)B.nn[1];
    g.nodes = g.nnxy * (uint32_t)B.nn[2];
    return g;
}

// Closed box [0, n] in cell coordinates; NaN compares false and so is outside.
__device__ __forceinline__ bool inside(const Geo &g, float x, float y, float z) {
    return x >= 0.f && x <= g.fnx && y >= 0.f && y <= g.fny && z >= 0.f && z <= g.fnz;
}

// Cell index clamp(floor(xi), 0, n-1) and fraction xi - index, for a point
// of the closed box (0 <= xi <= n <= 2^23). Adding 2^23 with rounding toward
// minus infinity leaves floor(xi) + 2^23 exactly (the spacing of floats in
// [2^23, 2^24] is 1), so the index is read from the bits and the fraction
// is exact; this takes full-rate adds where a float-to-integer conversion
// runs at an eighth of the rate. cm = 2^23 + (n - 1) clamps the upper face
// into the last cell.
__device__ __forceinline__ void cell_coord(float x, float cm, int &i, float &f) {
    const float t = fminf(__fadd_rd(x, 8388608.f), cm);
    i = __float_as_int(t) - 0x4B000000;
    f = x - (t - 8388608.f);
}

// Packed f32x2 arithmetic (sm_100 family): each half is one IEEE operation,
// so results are bitwise those of the scalar forms.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Cached cell in packed x-edge difference form. Corner (a, b, c) is the
// node (ix + a, iy + b, iz + c); the x-edge (b, c) is kept as its a = 0
// value and its difference v(a = 1) - v(a = 0). Per component k:
//   p0[k] = (value of edge (0,0), value of edge (0,1))
//   q0[k] = (difference of edge (0,0), difference of edge (0,1))
//   p1[k], q1[k]: the same for edges (1,0) and (1,1).
struct PCell {
    uint32_t node;   // node index of corner (0,0,0); ~0u when empty
    float2 p0[3], q0[3], p1[3], q1[3];
};

// Fills a PCell from the 8 corners given as four x-neighbour pairs of
// float3 rows: e(b,c) = (corner (0,b,c), corner (1,b,c)).
__device__ __forceinline__ void pcell_set(PCell &C, const float (&e00)[6], const float (&e10)[6],
                                          const float (&e01)[6], const float (&e11)[6]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        C.p0[k] = make_float2(e00[k], e01[k]);
        C.q0[k] = sub2(make_float2(e00[3 + k], e01[3 + k]), C.p0[k]);
        C.p1[k] = make_float2(e10[k], e11[k]);
        C.q1[k] = sub2(make_float2(e10[3 + k], e11[3 + k]), C.p1[k]);
    }
}

// Trilinear interpolation (Eq. 1 along x, then y, then z) from a PCell:
// the x step gives (c00, c01) and (c10, c11), the y step (c0, c1), the z
// step the value; every operation is the one lerp1 would perform.
__device__ __forceinline__ float3 trilerp_packed(const PCell &C, float fx, float fy, float fz) {
    const float2 fx2 = make_float2(fx, fx), fy2 = make_float2(fy, fy);
    float r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 a = fma2(fx2, C.q0[k], C.p0[k]);   // (c00, c01)
        const float2 b = fma2(fx2, C.q1[k], C.p1[k]);   // (c10, c11)
        const float2 y = fma2(fy2, sub2(b, a), a);      // (c0, c1)
        r[k] = fmaf(fz, y.y - y.x, y.x);
    }
    return make_float3(r[0], r[1], r[2]);
}

// The 8 corners of the cell at node index `node` from the block's field in
// global memory. F4 nodes are one 16-byte load each; F3 nodes are three
// 4-byte loads each (their 12-byte stride leaves no common alignment for
// wider loads; 8-, 16- and 32-byte variants with in-register selection were
// measured slower).
template <int LAYOUT>
__device__ __forceinline__ void load_pcell_global(const void *__restrict__ field, uint32_t nnx, uint32_t nnxy,
                                                  uint32_t node, PCell &C, uint32_t nodes = 0xffffffffu,
                                                  int32_t *err = nullptr) {
    float e[4][6];
    // the cell's last corner, node + nnx + nnxy + 1, must be a node of the block
    if (!BTO_IN_BOUNDS((uint64_t)node + nnx + nnxy + 1 < nodes, err)) node = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t nd = node + ((q & 1) ? nnx : 0u) + ((q & 2) ? nnxy : 0u);
        if (LAYOUT == LAYOUT_F4) {
            const float4 *f = reinterpret_cast<const float4 *>(field) + nd;
            const float4 a0 = __ldg(f);
            const float4 a1 = __ldg(f + 1);
            e[q][0] = a0.x; e[q][1] = a0.y; e[q][2] = a0.z;
            e[q][3] = a1.x; e[q][4] = a1.y; e[q][5] = a1.z;
        } else {
            const float *f = reinterpret_cast<const float *>(field) + 3ull * nd;
#pragma unroll
            for (int m = 0; m < 6; ++m) e[q][m] = __ldg(f + m);
        }
    }
    pcell_set(C, e[0], e[1], e[2], e[3]);
}

// Where a sampler takes a cell's corners from: GlobalSrc gathers them from
// the block's node field in global memory; the tiled kernel's source reads a
// shared-memory copy of the nodes around its tile and falls back to this one.
template <int LAYOUT>
struct GlobalSrc {
    const void *field;
    uint32_t nnx, nnxy;
    uint32_t nodes;   // nodes of the block (bounds-checked builds)
    int32_t *err;     // context error word (bounds-checked builds)
    __device__ __forceinline__ void load(int, int, int, uint32_t node, PCell &C) const {
        load_pcell_global<LAYOUT>(field, nnx, nnxy, node, C, nodes, err);
    }
};

template <class Src>
__device__ __forceinline__ float3 sample(PCell &C, const Src &src, const Geo &g, float x, float y, float z) {
    int ix, iy, iz;
    float fx, fy, fz;
    cell_coord(x, g.cmx, ix, fx);
    cell_coord(y, g.cmy, iy, fy);
    cell_coord(z, g.cmz, iz, fz);
    const uint32_t node = (uint32_t)ix + g.nnx * (uint32_t)iy + g.nnxy * (uint32_t)iz;
    if (node != C.node) {
        src.load(ix, iy, iz, node, C);
        C.node = node;
    }
    return trilerp_packed(C, fx, fy, fz);
}

// One RK4 step in cell units (s = dt / h per axis). Returns 0 and moves x
// when every tested point stays in the block; otherwise returns the stage
// whose point left first (1 = p2, 2 = p3, 3 = p4, 4 = end point), leaves x
// unchanged and stores that point in q. Every sampled point has passed the
// closed-box test (x itself is inside), so cell_coord's range holds.
template <class Src>
__device__ __forceinline__ int rk4_step_src(float3 &x, const Src &src, const Geo &g, const float3 s,
                                            float3 &q) {
    const float3 hs = make_float3(0.5f * s.x, 0.5f * s.y, 0.5f * s.z);
    PCell C;
    C.node = ~0u;
    const float3 k1 = sample(C, src, g, x.x, x.y, x.z);
    float px = fmaf(hs.x, k1.x, x.x), py = fmaf(hs.y, k1.y, x.y), pz = fmaf(hs.z, k1.z, x.z);
    if (!inside(g, px, py, pz)) { q = make_float3(px, py, pz); return 1; }
    const float3 k2 = sample(C, src, g, px, py, pz);
    float3 acc = make_float3(k1.x + 2.f * k2.x, k1.y + 2.f * k2.y, k1.z + 2.f * k2.z);
    px = fmaf(hs.x, k2.x, x.x); py = fmaf(hs.y, k2.y, x.y); pz = fmaf(hs.z, k2.z, x.z);
    if (!inside(g, px, py, pz)) { q = make_float3(px, py, pz); return 2; }
    const float3 k3 = sample(C, src, g, px, py, pz);
    acc.x = fmaf(2.f, k3.x, acc.x); acc.y = fmaf(2.f, k3.y, acc.y); acc.z = fmaf(2.f, k3.z, acc.z);
    px = fmaf(s.x, k3.x, x.x); py = fmaf(s.y, k3.y, x.y); pz = fmaf(s.z, k3.z, x.z);
    if (!inside(g, px, py, pz)) { q = make_float3(px, py, pz); return 3; }
    const float3 k4 = sample(C, src, g, px, py, pz);
    acc.x += k4.x; acc.y += k4.y; acc.z += k4.z;
    const float sx6 = s.x * (1.f / 6.f), sy6 = s.y * (1.f / 6.f), sz6 = s.z * (1.f / 6.f);
    px = fmaf(sx6, acc.x, x.x); py = fmaf(sy6, acc.y, x.y); pz = fmaf(sz6, acc.z, x.z);
    if (!inside(g, px, py, pz)) { q = make_float3(px, py, pz); return 4; }
    x = make_float3(px, py, pz);
    return 0;
}

template <int LAYOUT>
__device__ __forceinline__ int rk4_step(float3 &x, const void *__restrict__ field, const Geo &g,
                                        const float3 s, float3 &q, int32_t *err = nullptr) {
    return rk4_step_src(x, GlobalSrc<LAYOUT>{field, g.nnx, g.nnxy, g.nodes, err}, g, s, q);
}

// Termination location (the paper's future work, Sec. 6): the chord from the
// last in-block position x to the first point q found outside is clipped to
// the block, t = largest value in [0, 1] with x + t (q - x) inside; the exit
// time is the cycle plus t times the fraction of the step at which q was
// taken (1/2 for p2 and p3, 1 for p4 and the end point). A q with a NaN
// component gives no direction: the location is x and t = 0.
__device__ __forceinline__ float4 clip_exit(float3 nf, float3 x, float3 q, int stage, int cycle) {
    if (!(q.x == q.x && q.y == q.y && q.z == q.z)) return make_float4(x.x, x.y, x.z, (float)cycle);
    float t = 1.f;
    const float xs[3] = {x.x, x.y, x.z}, qs[3] = {q.x, q.y, q.z}, ns[3] = {nf.x, nf.y, nf.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (qs[a] > ns[a]) t = fminf(t, (ns[a] - xs[a]) / (qs[a] - xs[a]));
        if (qs[a] < 0.f) t = fminf(t, (0.f - xs[a]) / (qs[a] - xs[a]));
    }
    t = fmaxf(t, 0.f);
    const float cx = fminf(fmaxf(fmaf(t, q.x - x.x, x.x), 0.f), nf.x);
    const float cy = fminf(fmaxf(fmaf(t, q.y - x.y, x.y), 0.f), nf.y);
    const float cz = fminf(fmaxf(fmaf(t, q.z - x.z, x.z), 0.f), nf.z);
    return make_float4(cx, cy, cz, (float)cycle + t * (stage <= 2 ? 0.5f : 1.f));
}


}  // namespace dev
}  // namespace bto
