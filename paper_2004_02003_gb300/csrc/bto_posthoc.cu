// Post hoc kernels of libbto for sm_103a (Sec. 3.2): reconstruction of
// missing basis flows on the seed lattice (row f2) and pathline stitching
// through successive intervals' basis flows (row f3). They run after the
// in situ intervals, on their outputs, and share no code with the
// advection kernels.
#include <cstdint>
#include <cuda_runtime.h>

#include "bto_internal.h"

namespace bto {
namespace {

// Post hoc lattice reconstruction (Sec. 3.2 / Sec. 3.3, Eq. 2): a missing
// basis flow at lattice point J takes, along the axis whose nearest valid
// neighbours on both sides are closest (a + b smallest; ties x, y, z), the
// linear interpolant (Eq. 1) of their end positions at J:
//   end(J) = (b end(J - a e) + a end(J + b e)) / (a + b).
// Eq. (2): interpolating from the filled value afterwards equals
// interpolating from the two neighbours directly. Entries with no axis
// holding valid neighbours on both sides stay missing.
__global__ void fill_lattice_kernel(int3 S, const float *__restrict__ ends, const uint8_t *__restrict__ valid,
                                    float *__restrict__ out, uint8_t *__restrict__ status) {
    const int64_t P = (int64_t)S.x * S.y * S.z;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
        if (valid[p]) {
            out[3 * p] = ends[3 * p]; out[3 * p + 1] = ends[3 * p + 1]; out[3 * p + 2] = ends[3 * p + 2];
            if (status) status[p] = 1;
            continue;
        }
        const int jx = (int)(p % S.x), jy = (int)((p / S.x) % S.y), jz = (int)(p / ((int64_t)S.x * S.y));
        const int j[3] = {jx, jy, jz};
        const int ext[3] = {S.x, S.y, S.z};
        const int64_t step[3] = {1, S.x, (int64_t)S.x * S.y};
        int best_axis = -1, best_a = 0, best_b = 0;
        for (int ax = 0; ax < 3; ++ax) {
            int a = 1;
            while (j[ax] - a >= 0 && !valid[p - a * step[ax]]) ++a;
            if (j[ax] - a < 0) continue;
            int b = 1;
            while (j[ax] + b < ext[ax] && !valid[p + b * step[ax]]) ++b;
            if (j[ax] + b >= ext[ax]) continue;
            if (best_axis < 0 || a + b < best_a + best_b) { best_axis = ax; best_a = a; best_b = b; }
        }
        if (best_axis < 0) {
            const float nan = __int_as_float(0x7fc00000);
            out[3 * p] = nan; out[3 * p + 1] = nan; out[3 * p + 2] = nan;
            if (status) status[p] = 0;
            continue;
        }
        int64_t pl = p - best_a * step[best_axis], pr = p + best_b * step[best_axis];
        if (!BTO_IN_BOUNDS(pl >= 0 && pr < P, nullptr)) pl = pr = p;
        const float wl = (float)best_b / (float)(best_a + best_b), wr = (float)best_a / (float)(best_a + best_b);
#pragma unroll
        for (int k = 0; k < 3; ++k) out[3 * p + k] = wl * ends[3 * pl + k] + wr * ends[3 * pr + k];
        if (status) status[p] = 2;
    }
}

// Pathline stitching (Sec. 3.2): a new particle follows the basis flows of
// successive intervals. At the start of interval k it sits in a cell of the
// seed lattice; its position at the end of the interval interpolates the end
// positions of that cell's basis flows:
//   trilinear    the 8 corners, Eq. 1 per axis;
//   barycentric  the 4 vertices of the cell's Kuhn tetrahedron holding it
//                (the paper's barycentric coordinates over a Delaunay
//                neighbourhood; the cells of a full lattice are cospherical,
//                so the Kuhn split is a Delaunay triangulation): with the
//                fractional coordinates sorted t_a >= t_b >= t_c (a stable
//                sort, ties in axis order), vertices 0, e_a, e_a + e_b,
//                (1, 1, 1) and weights 1 - t_a, t_a - t_b, t_b - t_c, t_c.
// A particle outside the lattice, or next to a missing basis flow (NaN) that
// its interpolant uses, stops: its later positions are NaN.
template <bool BARY>
__global__ void stitch_kernel(int3 S, float3 origin, float3 inv_sp, int32_t intervals,
                              const float *const *__restrict__ ends_table, int64_t nq,
                              const float *__restrict__ start, float *__restrict__ path) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float nan = __int_as_float(0x7fc00000);
    const int64_t P = (int64_t)S.x * S.y * S.z;
    (void)P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += stride) {
        float x = start[3 * i], y = start[3 * i + 1], z = start[3 * i + 2];
        path[3 * i] = x; path[3 * i + 1] = y; path[3 * i + 2] = z;
        for (int32_t k = 0; k < intervals; ++k) {
            float nx = nan, ny = nan, nz = nan;
            const float u = (x - origin.x) * inv_sp.x, v = (y - origin.y) * inv_sp.y, w = (z - origin.z) * inv_sp.z;
            const bool in = u >= 0.f && v >= 0.f && w >= 0.f && u <= (float)(S.x - 1) &&
                            v <= (float)(S.y - 1) && w <= (float)(S.z - 1);
            if (in) {
                const int ix = min((int)u, max(S.x - 2, 0)), iy = min((int)v, max(S.y - 2, 0)),
                          iz = min((int)w, max(S.z - 2, 0));
                const float fx = u - ix, fy = v - iy, fz = w - iz;
                const float *E = ends_table[k];
                float acc[3] = {0.f, 0.f, 0.f};
                if (BARY) {
                    // stable descending sort of (fx, fy, fz) with the axes
                    int ax[3] = {0, 1, 2};
                    float t[3] = {fx, fy, fz};
                    if (t[1] > t[0]) { float q = t[0]; t[0] = t[1]; t[1] = q; int r = ax[0]; ax[0] = ax[1]; ax[1] = r; }
                    if (t[2] > t[1]) {
                        float q = t[1]; t[1] = t[2]; t[2] = q; int r = ax[1]; ax[1] = ax[2]; ax[2] = r;
                        if (t[1] > t[0]) { q = t[0]; t[0] = t[1]; t[1] = q; r = ax[0]; ax[0] = ax[1]; ax[1] = r; }
                    }
                    int j[3] = {ix, iy, iz};
                    const int ext[3] = {S.x, S.y, S.z};
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (m > 0) j[ax[m - 1]] = min(j[ax[m - 1]] + 1, ext[ax[m - 1]] - 1);
                        const float wgt = m == 0 ? 1.f - t[0] : (m == 3 ? t[2] : t[m - 1] - t[m]);
                        int64_t p = j[0] + (int64_t)S.x * (j[1] + (int64_t)S.y * j[2]);
                        if (!BTO_IN_BOUNDS(p >= 0 && p < P, nullptr)) p = 0;
#pragma unroll
                        for (int d = 0; d < 3; ++d) acc[d] = fmaf(wgt, E[3 * p + d], acc[d]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 2; ++c)
#pragma unroll
                        for (int b = 0; b < 2; ++b)
#pragma unroll
                            for (int a = 0; a < 2; ++a) {
                                const int jx = min(ix + a, S.x - 1), jy = min(iy + b, S.y - 1), jz = min(iz + c, S.z - 1);
                                const float wgt = (a ? fx : 1.f - fx) * (b ? fy : 1.f - fy) * (c ? fz : 1.f - fz);
                                int64_t p = jx + (int64_t)S.x * (jy + (int64_t)S.y * jz);
                                if (!BTO_IN_BOUNDS(p >= 0 && p < P, nullptr)) p = 0;
#pragma unroll
                                for (int d = 0; d < 3; ++d) acc[d] = fmaf(wgt, E[3 * p + d], acc[d]);
                            }
                }
                nx = acc[0]; ny = acc[1]; nz = acc[2];
            }
            x = nx; y = ny; z = nz;
            const int64_t o = 3 * ((int64_t)(k + 1) * nq + i);
            path[o] = x; path[o + 1] = y; path[o + 2] = z;
        }
    }
}

}  // namespace

BTO_BOUNDS_ACCESSOR(bounds_failures_posthoc)

cudaError_t launch_stitch(const int32_t S[3], const float origin[3], const float spacing[3], int32_t intervals,
                          const float *const *ends_table, int64_t nq, const float *start, float *path, int grid,
                          cudaStream_t s, bool barycentric) {
    const int3 S3 = make_int3(S[0], S[1], S[2]);
    const float3 o = make_float3(origin[0], origin[1], origin[2]);
    const float3 inv = make_float3(1.f / spacing[0], 1.f / spacing[1], 1.f / spacing[2]);
    if (barycentric)
        stitch_kernel<true><<<grid, 256, 0, s>>>(S3, o, inv, intervals, ends_table, nq, start, path);
    else
        stitch_kernel<false><<<grid, 256, 0, s>>>(S3, o, inv, intervals, ends_table, nq, start, path);
    return cudaGetLastError();
}

cudaError_t launch_fill_lattice(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                uint8_t *status, int grid, cudaStream_t s) {
    fill_lattice_kernel<<<grid, 256, 0, s>>>(make_int3(S[0], S[1], S[2]), ends, valid, out, status);
    return cudaGetLastError();
}

}  // namespace bto
