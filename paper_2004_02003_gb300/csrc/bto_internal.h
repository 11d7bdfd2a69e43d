// Internal declarations shared by the host API (bto_api.cu) and the kernels
// (bto_kernels.cu) of libbto. Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bto {

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

// Arguments of one advection cycle (kernel K3: RK4 + termination + compaction).
// The active list is cut into groups of G = 32 * ppt slots; group g holds
// gcnt[g] live particles in its first slots, in Morton order of their seeds.
struct AdvectArgs {
    const BlockDev *blocks;      // [nb] device
    const int32_t *gblock;       // [slots / 32] block of each 32-slot unit
    int32_t nb;
    int32_t cycle;               // cycle index within the interval
    const void *field;           // single field pointer (nb == 1 calls), or NULL
    const void *const *fields;   // device array [nb] used when field == NULL
    const float4 *in;            // active list at cycle start (xi, id bits)
    float4 *out;                 // active list after the cycle
    const int32_t *gcnt_in;      // [ngroups] live particles per group at cycle start
    int32_t *gcnt_out;           // [ngroups] survivors per group
    int64_t ngroups;
    float4 *term;                // [P] termination record per canonical id
    float4 *clip;                // [P] first outside point (xi) and its RK4 stage, or NULL
    float dt;
};

enum { LAYOUT_F3 = 0, LAYOUT_F4 = 1 };

// Kernel launchers (bto_kernels.cu). Each returns cudaGetLastError().
cudaError_t launch_advect(const AdvectArgs &a, int layout, int nt, int ppt, bool cap, int grid,
                          size_t dyn_smem, cudaStream_t s);
cudaError_t advect_occupancy(int layout, int nt, int ppt, bool cap, bool batched, size_t dyn_smem,
                             int *ctas_per_sm);
cudaError_t launch_seed(const BlockDev *blocks, const int32_t *gblock, const int32_t *perm,
                        int64_t slots, int group, float4 *act, int32_t *gcnt, int grid,
                        cudaStream_t s);
cudaError_t launch_write_live(const BlockDev *blocks, const int32_t *gblock, const float4 *act,
                              const int32_t *gcnt, int64_t slots, int group, float *ends,
                              uint8_t *valid, int32_t *exit_cycle, int grid, cudaStream_t s);
cudaError_t launch_gather_live(const float4 *act, const int32_t *gcnt, const int64_t *dst,
                               int64_t slots, int group, float4 *out, int grid, cudaStream_t s);
cudaError_t launch_ingest(const void *field, const void *const *fields, int b, int64_t nodes, float4 *out,
                          int grid, cudaStream_t s);
cudaError_t launch_stitch(const int32_t S[3], const float origin[3], const float spacing[3], int32_t intervals,
                          const float *const *ends_table, int64_t nq, const float *start, float *path, int grid,
                          cudaStream_t s);
cudaError_t launch_fill_lattice(const int32_t S[3], const float *ends, const uint8_t *valid, float *out,
                                uint8_t *status, int grid, cudaStream_t s);
cudaError_t launch_write_term(const BlockDev *blocks, int32_t nb, int64_t P, float4 *term,
                              float *seeds, float *ends, uint8_t *valid, int32_t *exit_cycle,
                              int grid, cudaStream_t s, const float4 *clip = nullptr,
                              float *exit_pos = nullptr, float *exit_time = nullptr);

}  // namespace bto
