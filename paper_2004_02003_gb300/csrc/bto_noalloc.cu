// bto_interval_noalloc: one whole interval of one block without any device
// allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: an in situ simulation
// that hands all device memory to its own pool allocator at start-up, and
// forbids allocations by analysis libraries during its time steps, cannot
// use bto_create (which allocates the particle state). This entry point keeps
// that state in a fixed-size array that lives in the library's own device
// image instead. The caller still passes the fields and the output buffers.
//
// The scratch array below is a file-scope __device__ variable of this
// translation unit's device module. Under the runtime's lazy module loading
// the module, and with it the array's BTO_NOALLOC_SCRATCH_BYTES, is loaded
// on a device by the first call made there; it stays until the process
// exits, and every call on that device shares it. Host code cannot use the
// array's name as a device address; the first call on each device asks the
// runtime for the array's device address (cudaGetSymbolAddress, with that
// device current) and keeps it for later calls.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/bto.h"
#include "bto_internal.h"

namespace {

using bto::BlockDev;

constexpr int64_t kMaxSeeds = BTO_NOALLOC_MAX_SEEDS;
constexpr int64_t kMaxSlots = (kMaxSeeds + bto::kRegionAlign - 1) / bto::kRegionAlign * bto::kRegionAlign;
constexpr int64_t kMaxUnits = kMaxSlots / bto::kUnit;

// Byte offsets of the parts of the scratch array (each 256-byte aligned):
// the particle list (units of 32 slots: x, y, z, id), the termination records, the
// group counts, the seed order, the 32-slot-unit block map and the block.
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffPart = 0;
constexpr size_t kOffTerm = kOffPart + align256(4 * sizeof(float) * kMaxSlots);
constexpr size_t kOffGcnt = kOffTerm + align256(sizeof(float4) * kMaxSeeds);
constexpr size_t kOffPerm = kOffGcnt + align256(sizeof(int32_t) * kMaxUnits);
constexpr size_t kOffGblock = kOffPerm + align256(sizeof(int32_t) * kMaxSeeds);
constexpr size_t kOffBlock = kOffGblock + align256(sizeof(int32_t) * kMaxUnits);
constexpr size_t kScratchBytes = kOffBlock + align256(sizeof(BlockDev));
static_assert(kScratchBytes == BTO_NOALLOC_SCRATCH_BYTES,
              "BTO_NOALLOC_SCRATCH_BYTES in include/bto.h must match the scratch layout");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, filled on the first call
// made with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

bto_status scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return BTO_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return BTO_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return BTO_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return BTO_OK;
}

// Writes the block descriptor, an identity seed order (canonical lattice
// order), the 32-slot-unit block map and "not terminated" records: every
// part of the shared array that a call reads before writing it.
__global__ void noalloc_init_kernel(BlockDev B, int64_t slots, BlockDev *blk, int32_t *perm,
                                    int32_t *gblock, float4 *term) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) *blk = B;
    for (int64_t i = i0; i < B.nseeds; i += stride) {
        perm[i] = (int32_t)i;
        term[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    }
    for (int64_t u = i0; u < slots / bto::kUnit; u += stride) gblock[u] = 0;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

}  // namespace

extern "C" bto_status bto_interval_noalloc(const int32_t extent_cells[3], const float origin[3],
                                           const float spacing[3], int32_t seed_stride,
                                           int32_t interval_cycles,
                                           const void *const *d_field_table, float dt,
                                           float *d_seeds, float *d_ends, uint8_t *d_valid,
                                           int32_t *d_exit_cycle, bto_stream stream) {
    if (!extent_cells || !origin || !spacing || !d_field_table || !d_seeds || !d_ends || !d_valid)
        return BTO_ERR_INVALID_ARG;
    if (seed_stride < 1 || interval_cycles < 1 || !std::isfinite(dt)) return BTO_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_field_table) % alignof(void *) ||
        reinterpret_cast<uintptr_t>(d_seeds) % 4 || reinterpret_cast<uintptr_t>(d_ends) % 4 ||
        reinterpret_cast<uintptr_t>(d_exit_cycle) % 4)
        return BTO_ERR_INVALID_ARG;
    BlockDev B{};
    int64_t nodes = 1;
    for (int a = 0; a < 3; ++a) {
        const int32_t n = extent_cells[a];
        if (n < 1 || n > (1 << 23) || !std::isfinite(origin[a]) || !finite_pos(spacing[a]))
            return BTO_ERR_INVALID_ARG;
        B.n[a] = n;
        B.nn[a] = n + 1;
        B.S[a] = (n + seed_stride - 1) / seed_stride;
        B.inv_h[a] = 1.0f / spacing[a];
        B.origin[a] = origin[a];
        B.h[a] = spacing[a];
        nodes *= (int64_t)(n + 1);
    }
    if (nodes > (1ll << 29)) return BTO_ERR_INVALID_ARG;
    B.stride = seed_stride;
    B.nseeds = (int64_t)B.S[0] * B.S[1] * B.S[2];
    B.base = 0;
    B.slot_base = 0;
    if (B.nseeds > kMaxSeeds) return BTO_ERR_UNSUPPORTED;  // beyond the static scratch

    unsigned char *base = nullptr;
    const bto_status st = scratch_address(&base);
    if (st != BTO_OK) return st;
    float4 *term = reinterpret_cast<float4 *>(base + kOffTerm);
    int32_t *perm = reinterpret_cast<int32_t *>(base + kOffPerm);
    int32_t *gblock = reinterpret_cast<int32_t *>(base + kOffGblock);
    BlockDev *blk = reinterpret_cast<BlockDev *>(base + kOffBlock);

    const int64_t slots = (B.nseeds + bto::kRegionAlign - 1) / bto::kRegionAlign * bto::kRegionAlign;
    const int nt = 128, ppt = 2, group = 32 * ppt;
    bto::PartList part;
    part.rec = reinterpret_cast<float *>(base + kOffPart);
    part.gcnt = reinterpret_cast<int32_t *>(base + kOffGcnt);
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = bto::advect_occupancy(bto::LAYOUT_F3, nt, ppt, false, false, 0, &occ);
    if (e != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        return BTO_ERR_CUDA;
    }
    const int64_t ngroups = slots / group;
    const int64_t need = (ngroups + nt / 32 - 1) / (nt / 32);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * occ, need));
    const int aux = (int)std::max<int64_t>(1, std::min<int64_t>((slots + 255) / 256, (int64_t)sms * 8));
    cudaStream_t s = (cudaStream_t)stream;

    noalloc_init_kernel<<<aux, 256, 0, s>>>(B, slots, blk, perm, gblock, term);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = bto::launch_seed(blk, gblock, perm, slots, group, part, aux, s);
    for (int32_t c = 0; c < interval_cycles && e == cudaSuccess; ++c) {
        bto::AdvectArgs a{};
        a.blocks = blk;
        a.gblock = gblock;
        a.nb = 1;
        a.cycle = c;
        a.field = nullptr;
        a.fields = d_field_table + c;
        a.p = part;
        a.ngroups = ngroups;
        a.term = term;
        a.dt = dt;
        e = bto::launch_advect(a, bto::LAYOUT_F3, nt, ppt, false, grid, 0, s);
    }
    if (e == cudaSuccess)
        e = bto::launch_write_live(blk, gblock, part, slots, group, d_ends, d_valid, d_exit_cycle, aux, s);
    if (e == cudaSuccess)
        e = bto::launch_write_term(blk, 1, B.nseeds, term, d_seeds, d_ends, d_valid, d_exit_cycle, aux, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return BTO_ERR_CUDA;
    }
    return BTO_OK;
}
