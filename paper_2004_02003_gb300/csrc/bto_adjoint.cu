// K7: checkpointed discrete adjoint of one BTO interval.
//
// Forward: particles start at caller-given positions (the lattice seeds for a
// flow map, Sec. 2.3) and take one RK4 step per cycle through that cycle's
// field, with the closed-box termination of the advection kernel (the same
// device functions, bto_device.cuh). Positions are kept every K cycles.
// Backward: for each K-cycle segment, last to first, the positions inside
// the segment are recomputed from its checkpoint, then the reverse of each
// cycle maps dL/dx after the cycle to dL/dx before it and adds the node
// velocity gradients of the cycle (scatter with atomics). A terminated
// particle's end is its last in-block position, so its gradient flows back
// only through the cycles before its exit cycle.
//
// All fields of the interval are resident in the tape's table and the
// particles are independent, so each of the forward and the reverse sweep is
// one launch with one thread per particle (per particle and Jacobian row for
// the Jacobian), looping over the cycles: no per-cycle launches, and the
// adjoint stays in registers across the whole sweep.
//
// Reverse of x' = x + s/6 (k1 + 2 k2 + 2 k3 + k4) (cell units, s = dt/h),
// k1 = v(x), k2 = v(x + s/2 k1), k3 = v(x + s/2 k2), k4 = v(x + s k3),
// given lam = dL/dx':  g1 = s/6 lam, g2 = g3 = s/3 lam, g4 = s/6 lam;
// stage 4, 3, 2: qbar = (dv/dq)^T g; lam_x += qbar; previous stage's g gets
// (s or s/2) qbar; stage 1: lam = lam_x + (dv/dx)^T g1. Every stage adds its
// trilinear weights times g to the 8 corner nodes' velocity gradients.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>

#include <cuda_runtime.h>

#include "../../include/bto.h"
#include "bto_device.cuh"
#include "bto_internal.h"

using bto::BlockDev;

struct bto_tape {
    bto::DevAlloc mem;           // device allocator captured at creation
    int device = 0;
    int sm_count = 0;
    BlockDev B{};
    int64_t P = 0;
    int32_t L = 0, K = 0, nck = 0;
    float4 *ckpt = nullptr;     // nck * P positions (cell units) at cycles 0, K, 2K, ... and L
    float4 *seg = nullptr;      // K * 3P positions inside one segment, per sweep thread
    float4 *lam = nullptr;      // 3P adjoints (cell units): one per sweep thread
    BlockDev *d_block = nullptr;
    int32_t *exitc = nullptr;   // P exit cycle, -1 while valid
    const void *const *table = nullptr;
    float dt = 0.f;
    bool have_forward = false;
};

namespace {

using namespace bto::dev;

struct Stage {
    int ix, iy, iz;
    float fx, fy, fz;
};

// Trilinear value, its Jacobian d v / d xi (cell units) and the cell.
__device__ __forceinline__ void sample_jac(const float *__restrict__ f, const Geo &g, float x, float y,
                                           float z, float3 &v, float (&J)[3][3], Stage &st) {
    st.ix = min(max(__float2int_rd(x), 0), g.nx - 1);
    st.iy = min(max(__float2int_rd(y), 0), g.ny - 1);
    st.iz = min(max(__float2int_rd(z), 0), g.nz - 1);
    st.fx = x - (float)st.ix;
    st.fy = y - (float)st.iy;
    st.fz = z - (float)st.iz;
    float c[8][3];
    load_cell<bto::LAYOUT_F3>(f, g.nnx, g.nnxy, st.ix, st.iy, st.iz, c);
    v = trilerp(c, st.fx, st.fy, st.fz);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // d/dfx: x-differences blended in y, z; likewise for y and z
        const float dx00 = c[1][k] - c[0][k], dx10 = c[3][k] - c[2][k];
        const float dx01 = c[5][k] - c[4][k], dx11 = c[7][k] - c[6][k];
        J[k][0] = lerp1(lerp1(dx00, dx10, st.fy), lerp1(dx01, dx11, st.fy), st.fz);
        const float dy0 = lerp1(c[2][k], c[3][k], st.fx) - lerp1(c[0][k], c[1][k], st.fx);
        const float dy1 = lerp1(c[6][k], c[7][k], st.fx) - lerp1(c[4][k], c[5][k], st.fx);
        J[k][1] = lerp1(dy0, dy1, st.fz);
        const float z0 = lerp1(lerp1(c[0][k], c[1][k], st.fx), lerp1(c[2][k], c[3][k], st.fx), st.fy);
        const float z1 = lerp1(lerp1(c[4][k], c[5][k], st.fx), lerp1(c[6][k], c[7][k], st.fx), st.fy);
        J[k][2] = z1 - z0;
    }
}

__device__ __forceinline__ float3 jt_times(const float (&J)[3][3], float3 gvec) {
    return make_float3(J[0][0] * gvec.x + J[1][0] * gvec.y + J[2][0] * gvec.z,
                       J[0][1] * gvec.x + J[1][1] * gvec.y + J[2][1] * gvec.z,
                       J[0][2] * gvec.x + J[1][2] * gvec.y + J[2][2] * gvec.z);
}

__device__ __forceinline__ bool alive_at(int32_t e, int32_t c) { return e < 0 || c < e; }

__global__ void tape_init_kernel(const BlockDev *__restrict__ blk, int64_t P, const float *__restrict__ seeds,
                                 float4 *__restrict__ x0, int32_t *__restrict__ exitc) {
    const BlockDev &B = *blk;
    const Geo g = load_geo(B);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = (seeds[3 * i + 0] - B.origin[0]) * B.inv_h[0];
        const float y = (seeds[3 * i + 1] - B.origin[1]) * B.inv_h[1];
        const float z = (seeds[3 * i + 2] - B.origin[2]) * B.inv_h[2];
        x0[i] = make_float4(x, y, z, 0.f);
        exitc[i] = inside(g, x, y, z) ? -1 : 0;   // a start outside the block never moves
    }
}

// Forward over the whole interval, one thread per particle (the fields of
// every cycle are resident in the tape's table, and particles are
// independent): cycle after cycle, the RK4 step with the closed-box tests of
// the advection kernel; a failing step records its cycle. Positions are kept
// at cycles 0, K, 2K, ... (checkpoint m at cycle m K) and at L (the last
// checkpoint).
__global__ void tape_forward_kernel(const BlockDev *__restrict__ blk, const void *const *__restrict__ table,
                                    int32_t L, int32_t K, float dt, int64_t P, float4 *__restrict__ ckpt,
                                    int32_t *__restrict__ exitc) {
    const BlockDev &B = *blk;
    const Geo g = load_geo(B);
    const float3 s = make_float3(dt * B.inv_h[0], dt * B.inv_h[1], dt * B.inv_h[2]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float4 r = ckpt[i];
        int32_t e = exitc[i];
        for (int32_t c = 0; c < L; ++c) {
            if (alive_at(e, c)) {
                float3 x = make_float3(r.x, r.y, r.z), q;
                if (rk4_step<bto::LAYOUT_F3>(x, table[c], g, s, q) == 0) {
                    r.x = x.x; r.y = x.y; r.z = x.z;
                } else {
                    e = c;
                }
            }
            if ((c + 1) % K == 0 || c + 1 == L) ckpt[(size_t)((c + K) / K) * P + i] = r;
        }
        exitc[i] = e;
    }
}

// Node-velocity gradients of one reverse cycle: stage k adds w_k(corner) g_k
// to the 8 corners of its cell. Stages whose points lie in the same cell are
// summed per corner first, so that each distinct cell takes 24 atomic adds
// (the stages of a step mostly share a cell).
__device__ __forceinline__ float stage_w(const Stage &st, int a, int b, int c) {
    return (a ? st.fx : 1.f - st.fx) * (b ? st.fy : 1.f - st.fy) * (c ? st.fz : 1.f - st.fz);
}

__device__ __forceinline__ void scatter_step(float *__restrict__ gF, const Geo &g, const Stage (&st)[4],
                                             const float3 (&gs)[4]) {
    if (!gF) return;
    unsigned done = 0;
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        if (done & (1u << k)) continue;
        bool in[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            in[j] = j <= k && !(done & (1u << j)) && st[j].ix == st[k].ix && st[j].iy == st[k].iy &&
                    st[j].iz == st[k].iz;
            if (in[j]) done |= 1u << j;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
                    for (int j = 3; j >= 0; --j) {
                        if (!in[j]) continue;
                        const float w = stage_w(st[j], a, b, c);
                        vx = fmaf(w, gs[j].x, vx);
                        vy = fmaf(w, gs[j].y, vy);
                        vz = fmaf(w, gs[j].z, vz);
                    }
                    const uint32_t node = (uint32_t)(st[k].ix + a) + g.nnx * (uint32_t)(st[k].iy + b) +
                                          g.nnxy * (uint32_t)(st[k].iz + c);
                    float *p = gF + 3ull * node;
                    atomicAdd(p + 0, vx);
                    atomicAdd(p + 1, vy);
                    atomicAdd(p + 2, vz);
                }
    }
}

// Reverse of one cycle for one particle at xc (cell units) with adjoint lm
// (see the header of this file); adds the node-velocity gradients to gF
// when it is not NULL. Returns the adjoint before the cycle.
__device__ __forceinline__ float3 adj_step(const float *__restrict__ f, float *__restrict__ gF, const Geo &g,
                                           const float3 s, const float4 r, const float3 Lm) {
    float3 k1, k2, k3, k4;
    float J1[3][3], J2[3][3], J3[3][3], J4[3][3];
    Stage st[4];
    sample_jac(f, g, r.x, r.y, r.z, k1, J1, st[0]);
    sample_jac(f, g, fmaf(0.5f * s.x, k1.x, r.x), fmaf(0.5f * s.y, k1.y, r.y), fmaf(0.5f * s.z, k1.z, r.z),
               k2, J2, st[1]);
    sample_jac(f, g, fmaf(0.5f * s.x, k2.x, r.x), fmaf(0.5f * s.y, k2.y, r.y), fmaf(0.5f * s.z, k2.z, r.z),
               k3, J3, st[2]);
    sample_jac(f, g, fmaf(s.x, k3.x, r.x), fmaf(s.y, k3.y, r.y), fmaf(s.z, k3.z, r.z), k4, J4, st[3]);
    const float3 s6 = make_float3(s.x / 6.f, s.y / 6.f, s.z / 6.f);
    const float3 s3v = make_float3(s.x / 3.f, s.y / 3.f, s.z / 3.f);
    float3 gs[4];
    gs[0] = make_float3(s6.x * Lm.x, s6.y * Lm.y, s6.z * Lm.z);
    gs[1] = make_float3(s3v.x * Lm.x, s3v.y * Lm.y, s3v.z * Lm.z);
    gs[2] = gs[1];
    gs[3] = gs[0];
    float3 lx = Lm;
    float3 q = jt_times(J4, gs[3]);
    lx.x += q.x; lx.y += q.y; lx.z += q.z;
    gs[2].x = fmaf(s.x, q.x, gs[2].x); gs[2].y = fmaf(s.y, q.y, gs[2].y); gs[2].z = fmaf(s.z, q.z, gs[2].z);
    q = jt_times(J3, gs[2]);
    lx.x += q.x; lx.y += q.y; lx.z += q.z;
    gs[1].x = fmaf(0.5f * s.x, q.x, gs[1].x); gs[1].y = fmaf(0.5f * s.y, q.y, gs[1].y);
    gs[1].z = fmaf(0.5f * s.z, q.z, gs[1].z);
    q = jt_times(J2, gs[1]);
    lx.x += q.x; lx.y += q.y; lx.z += q.z;
    gs[0].x = fmaf(0.5f * s.x, q.x, gs[0].x); gs[0].y = fmaf(0.5f * s.y, q.y, gs[0].y);
    gs[0].z = fmaf(0.5f * s.z, q.z, gs[0].z);
    q = jt_times(J1, gs[0]);
    scatter_step(gF, g, st, gs);
    return make_float3(lx.x + q.x, lx.y + q.y, lx.z + q.z);
}

// One reverse sweep over the interval, one thread per (adjoint, particle):
// thread t carries the adjoint lam[t] of particle t mod P through the
// segments, last to first; each segment's positions are recomputed from its
// checkpoint into the thread's own slots of seg, then the segment's cycles
// are reversed. nthr = P for a gradient sweep, 3 P for the three rows of the
// flow-map Jacobian (one sweep each, side by side).
__global__ void tape_reverse_kernel(const BlockDev *__restrict__ blk, const void *const *__restrict__ table,
                                    float *const *__restrict__ gtable, int32_t L, int32_t K, int32_t nck,
                                    float dt, int64_t P, int64_t nthr, const float4 *__restrict__ ckpt,
                                    float4 *__restrict__ seg, const int32_t *__restrict__ exitc,
                                    float4 *__restrict__ lam) {
    const BlockDev &B = *blk;
    const Geo g = load_geo(B);
    const float3 s = make_float3(dt * B.inv_h[0], dt * B.inv_h[1], dt * B.inv_h[2]);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nthr; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % P;
        const int32_t e = exitc[i];
        const float4 L4 = lam[t];
        float3 lm = make_float3(L4.x, L4.y, L4.z);
        for (int32_t sg = nck - 2; sg >= 0; --sg) {
            const int32_t c0 = sg * K;
            const int32_t c1 = min(c0 + K, L);
            float4 r = ckpt[(size_t)sg * P + i];
            seg[t] = r;
            for (int32_t c = c0; c + 1 < c1; ++c) {
                if (alive_at(e, c)) {
                    float3 x = make_float3(r.x, r.y, r.z), q;
                    if (rk4_step<bto::LAYOUT_F3>(x, table[c], g, s, q) == 0) {
                        r.x = x.x; r.y = x.y; r.z = x.z;
                    }
                }
                seg[(size_t)(c - c0 + 1) * nthr + t] = r;
            }
            for (int32_t c = c1 - 1; c >= c0; --c) {
                if (!alive_at(e, c)) continue;
                lm = adj_step(reinterpret_cast<const float *>(table[c]), gtable ? gtable[c] : nullptr, g, s,
                              seg[(size_t)(c - c0) * nthr + t], lm);
            }
        }
        lam[t] = make_float4(lm.x, lm.y, lm.z, 0.f);
    }
}

// Outputs of the forward: physical end positions, valid flags, exit cycles.
__global__ void tape_out_kernel(const BlockDev *__restrict__ blk, int64_t P, const float4 *__restrict__ x,
                                const int32_t *__restrict__ exitc, float *__restrict__ ends,
                                uint8_t *__restrict__ valid, int32_t *__restrict__ exit_out) {
    const BlockDev &B = *blk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 r = x[i];
        ends[3 * i + 0] = fmaf(r.x, B.h[0], B.origin[0]);
        ends[3 * i + 1] = fmaf(r.y, B.h[1], B.origin[1]);
        ends[3 * i + 2] = fmaf(r.z, B.h[2], B.origin[2]);
        valid[i] = exitc[i] < 0 ? 1 : 0;
        if (exit_out) exit_out[i] = exitc[i];
    }
}

// lam = h * dL/d(end) (physical -> cell units); with grad == NULL, the unit
// vector of axis `axis` for every particle (a Jacobian sweep).
__global__ void tape_lam_init_kernel(const BlockDev *__restrict__ blk, int64_t P, const float *__restrict__ grad,
                                     int axis, float4 *__restrict__ lam) {
    const BlockDev &B = *blk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float gx, gy, gz;
        if (grad) {
            gx = grad[3 * i + 0]; gy = grad[3 * i + 1]; gz = grad[3 * i + 2];
        } else {
            gx = axis == 0 ? 1.f : 0.f; gy = axis == 1 ? 1.f : 0.f; gz = axis == 2 ? 1.f : 0.f;
        }
        lam[i] = make_float4(gx * B.h[0], gy * B.h[1], gz * B.h[2], 0.f);
    }
}

// dL/d(start) = lam / h; written to out[stride * i + offset + a].
__global__ void tape_lam_out_kernel(const BlockDev *__restrict__ blk, int64_t P, const float4 *__restrict__ lam,
                                    float *__restrict__ out, int stride, int offset) {
    const BlockDev &B = *blk;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 l = lam[i];
        out[stride * i + offset + 0] = l.x * B.inv_h[0];
        out[stride * i + offset + 1] = l.y * B.inv_h[1];
        out[stride * i + offset + 2] = l.z * B.inv_h[2];
    }
}

// Largest eigenvalue of the symmetric 3x3 matrix C (closed form of the
// characteristic cubic, trigonometric solution), in double.
__device__ double sym3_max_eig(const double C[3][3]) {
    const double p1 = C[0][1] * C[0][1] + C[0][2] * C[0][2] + C[1][2] * C[1][2];
    const double q = (C[0][0] + C[1][1] + C[2][2]) / 3.0;
    if (p1 <= 1e-300 * (q * q + 1.0)) return fmax(C[0][0], fmax(C[1][1], C[2][2]));
    const double p2 = (C[0][0] - q) * (C[0][0] - q) + (C[1][1] - q) * (C[1][1] - q) +
                      (C[2][2] - q) * (C[2][2] - q) + 2.0 * p1;
    const double p = sqrt(p2 / 6.0);
    double Bm[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Bm[a][b] = (C[a][b] - (a == b ? q : 0.0)) / p;
    const double detB = Bm[0][0] * (Bm[1][1] * Bm[2][2] - Bm[1][2] * Bm[2][1]) -
                        Bm[0][1] * (Bm[1][0] * Bm[2][2] - Bm[1][2] * Bm[2][0]) +
                        Bm[0][2] * (Bm[1][0] * Bm[2][1] - Bm[1][1] * Bm[2][0]);
    const double r = fmin(1.0, fmax(-1.0, detB / 2.0));
    const double phi = acos(r) / 3.0;
    return q + 2.0 * p * cos(phi);
}

// FTLE = ln(sqrt(lambda_max(J^T J))) / |T| for valid particles, NaN for the
// others (their trajectory does not span the interval).
__global__ void tape_ftle_kernel(int64_t P, const float *__restrict__ jac, const int32_t *__restrict__ exitc,
                                 double T, float *__restrict__ ftle) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (exitc[i] >= 0) {
            ftle[i] = __int_as_float(0x7fc00000);
            continue;
        }
        double J[3][3], C[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) J[a][b] = jac[9 * i + 3 * a + b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C[a][b] = J[0][a] * J[0][b] + J[1][a] * J[1][b] + J[2][a] * J[2][b];
        const double lmax = sym3_max_eig(C);
        ftle[i] = (float)(0.5 * log(fmax(lmax, 1e-300)) / T);
    }
}

bto_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return BTO_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BTO_ERR_OOM : BTO_ERR_CUDA;
}

int grid_of(const bto_tape *t) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((t->P + 255) / 256, (int64_t)t->sm_count * 8));
}

void free_tape(bto_tape *t) {
    if (!t) return;
    t->mem.put(t->ckpt);
    t->mem.put(t->seg);
    t->mem.put(t->lam);
    t->mem.put(t->d_block);
    t->mem.put(t->exitc);
    delete t;
}

// One reverse sweep of nthr adjoints (P or 3 P) from the lam already
// initialised: a single launch.
bto_status reverse_sweep(bto_tape *t, float *const *gtable, int64_t nthr, cudaStream_t s) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nthr + 127) / 128, (int64_t)t->sm_count * 16));
    tape_reverse_kernel<<<grid, 128, 0, s>>>(t->d_block, t->table, gtable, t->L, t->K, t->nck, t->dt, t->P, nthr,
                                             t->ckpt, t->seg, t->exitc, t->lam);
    return cuda_st(cudaGetLastError());
}

}  // namespace

extern "C" {

bto_status bto_tape_create(const int32_t extent_cells[3], const float origin[3], const float spacing[3],
                           int64_t num_particles, int32_t cycles, int32_t checkpoint_every, bto_tape **out) {
    if (!extent_cells || !origin || !spacing || !out) return BTO_ERR_INVALID_ARG;
    if (num_particles < 1 || num_particles > (1ll << 30) || cycles < 1 || checkpoint_every < 1)
        return BTO_ERR_INVALID_ARG;
    BlockDev B{};
    int64_t nodes = 1;
    for (int a = 0; a < 3; ++a) {
        const int32_t n = extent_cells[a];
        if (n < 1 || n > (1 << 23) || !std::isfinite(origin[a]) || !std::isfinite(spacing[a]) || !(spacing[a] > 0.f))
            return BTO_ERR_INVALID_ARG;
        B.n[a] = n;
        B.nn[a] = n + 1;
        B.S[a] = 1;
        B.inv_h[a] = 1.0f / spacing[a];
        B.origin[a] = origin[a];
        B.h[a] = spacing[a];
        nodes *= (int64_t)(n + 1);
    }
    if (nodes > (1ll << 29)) return BTO_ERR_INVALID_ARG;
    B.stride = 1;
    B.nseeds = num_particles;
    bto_tape *t = new (std::nothrow) bto_tape();
    if (!t) return BTO_ERR_OOM;
    t->mem = bto::current_allocator();
    t->B = B;
    t->P = num_particles;
    t->L = cycles;
    t->K = std::min(checkpoint_every, cycles);
    t->nck = (cycles + t->K - 1) / t->K + 1;
    cudaError_t e = cudaGetDevice(&t->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->device);
    const size_t P = (size_t)num_particles;
    if (e == cudaSuccess) e = t->mem.get(&t->ckpt, sizeof(float4) * P * (size_t)t->nck);
    if (e == cudaSuccess) e = t->mem.get(&t->seg, sizeof(float4) * 3 * P * (size_t)t->K);
    if (e == cudaSuccess) e = t->mem.get(&t->lam, sizeof(float4) * 3 * P);
    if (e == cudaSuccess) e = t->mem.get(&t->d_block, sizeof(BlockDev));
    if (e == cudaSuccess) e = t->mem.get(&t->exitc, sizeof(int32_t) * P);
    if (e == cudaSuccess) e = cudaMemcpy(t->d_block, &t->B, sizeof(BlockDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_tape(t);
        return e == cudaErrorMemoryAllocation ? BTO_ERR_OOM : BTO_ERR_CUDA;
    }
    *out = t;
    return BTO_OK;
}

int64_t bto_tape_num_particles(const bto_tape *t) { return t ? t->P : -1; }

bto_status bto_tape_forward(bto_tape *t, const float *d_seeds, const void *const *d_field_table, float dt,
                            float *d_ends, uint8_t *d_valid, int32_t *d_exit_cycle, bto_stream stream) {
    if (!t || !d_seeds || !d_field_table || !d_ends || !d_valid || !std::isfinite(dt)) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_seeds) % 4 || reinterpret_cast<uintptr_t>(d_ends) % 4 ||
        reinterpret_cast<uintptr_t>(d_exit_cycle) % 4 ||
        reinterpret_cast<uintptr_t>(d_field_table) % alignof(void *))
        return BTO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = grid_of(t);
    const size_t P = (size_t)t->P;
    t->table = d_field_table;
    t->dt = dt;
    t->have_forward = false;
    tape_init_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, d_seeds, t->ckpt, t->exitc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>((t->P + 127) / 128, (int64_t)t->sm_count * 16));
        tape_forward_kernel<<<g1, 128, 0, s>>>(t->d_block, d_field_table, t->L, t->K, dt, t->P, t->ckpt, t->exitc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        tape_out_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, t->ckpt + (size_t)(t->nck - 1) * P, t->exitc, d_ends,
                                             d_valid, d_exit_cycle);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_st(e);
    t->have_forward = true;
    return BTO_OK;
}

bto_status bto_tape_backward(bto_tape *t, const float *d_grad_ends, float *d_grad_seeds,
                             float *const *d_grad_field_table, bto_stream stream) {
    if (!t || !d_grad_ends || !d_grad_seeds) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_grad_ends) % 4 || reinterpret_cast<uintptr_t>(d_grad_seeds) % 4 ||
        reinterpret_cast<uintptr_t>(d_grad_field_table) % alignof(void *))
        return BTO_ERR_INVALID_ARG;
    if (!t->have_forward) return BTO_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = grid_of(t);
    tape_lam_init_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, d_grad_ends, 0, t->lam);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_st(e);
    const bto_status st = reverse_sweep(t, d_grad_field_table, t->P, s);
    if (st != BTO_OK) return st;
    tape_lam_out_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, t->lam, d_grad_seeds, 3, 0);
    return cuda_st(cudaGetLastError());
}

bto_status bto_tape_jacobian(bto_tape *t, float *d_jac, bto_stream stream) {
    if (!t || !d_jac || reinterpret_cast<uintptr_t>(d_jac) % 4) return BTO_ERR_INVALID_ARG;
    if (!t->have_forward) return BTO_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = grid_of(t);
    // lam = e_axis for the three axes side by side: the sweep returns row
    // `axis` of d end / d start in lam[axis P + i]
    for (int axis = 0; axis < 3; ++axis) {
        tape_lam_init_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, nullptr, axis, t->lam + (size_t)axis * t->P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_st(e);
    }
    const bto_status st = reverse_sweep(t, nullptr, 3 * t->P, s);
    if (st != BTO_OK) return st;
    for (int axis = 0; axis < 3; ++axis) {
        tape_lam_out_kernel<<<grid, 256, 0, s>>>(t->d_block, t->P, t->lam + (size_t)axis * t->P, d_jac, 9, 3 * axis);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_st(e);
    }
    return BTO_OK;
}

bto_status bto_tape_ftle(bto_tape *t, const float *d_jac, float *d_ftle, bto_stream stream) {
    if (!t || !d_jac || !d_ftle) return BTO_ERR_INVALID_ARG;
    if (!t->have_forward) return BTO_ERR_STATE;
    const double T = std::fabs((double)t->dt * (double)t->L);
    if (!(T > 0.0)) return BTO_ERR_INVALID_ARG;
    tape_ftle_kernel<<<grid_of(t), 256, 0, (cudaStream_t)stream>>>(t->P, d_jac, t->exitc, T, d_ftle);
    return cuda_st(cudaGetLastError());
}

void bto_tape_destroy(bto_tape *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    free_tape(t);
}

}  // extern "C"
