// sg_internal.h -- launch entry points shared between the libsg translation
// units (not part of the public ABI; see include/sg.h for that).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace sg {

enum : int { kMapLambda = 0, kMapBBox = 1, kMapLut = 2, kMapUnroll = 3 };

enum : int { kStoreAuto = 0, kStoreScatter = 1, kStoreStaged = 2, kStoreTma = 3, kStoreFill = 4,
              kStoreSector = 5, kStoreMerge = 6, kStoreMasked = 7,
              // internal: the fill contract through the staged kernel's plain
              // stores, reading nothing (grids in host memory)
              kStoreFillPlain = 100 };

// Launch knobs.  ctas_per_sm <= 0 selects the occupancy maximum; order is a
// traversal order of the block space (kOrderRowMajor / kOrderInterleaved);
// store selects how the write pass stores (kStore*).
struct LaunchCfg {
    int ctas_per_sm = 0;
    int order = 1;
    int store = kStoreAuto;
};

// Number of SMs of the current device (cached per device).
int sm_count(int *err);

}  // namespace sg
#include "sg.h"
namespace sg {

// sg_launch_opts (NULL = defaults) -> LaunchCfg; false on a bad value.
bool read_launch_opts(const sg_launch_opts *o, LaunchCfg *cfg);

// Record a message for sg_last_error_string().
void set_last_error_message(const char *msg);

// Record a CUDA error for sg_last_error_string(); returns SG_ECUDA
// (SG_EUNSUPPORTED for cudaErrorNotSupported).
sg_status set_last_cuda_error(cudaError_t e);

cudaError_t launch_write_u8(int r, int s, int map, int vk, uint8_t *grid,
                            uint64_t vs, cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_write_f32(int r, int s, int map, int vk, float *grid,
                             uint64_t vs, cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_ca(int r, int s, int map, const uint8_t *in, uint8_t *out,
                      cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_diffuse(int r, int s, int map, const float *in, float *out,
                           float alpha, cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_ca_fused(int r, int s, int map, const uint8_t *in, uint8_t *out, int k,
                            cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_diffuse_fused(int r, int s, int map, const float *in, float *out,
                                 float alpha, int k, cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_block_map(int rb, int order, uint32_t *bx, uint32_t *by,
                             cudaStream_t st);

// Persistent grid size: min(work units, SMs * resident CTAs).  `occ_cache`
// (one per kernel instance) keeps the occupancy query off the launch path
// after the first call; the value depends only on the kernel and the arch.
template <typename K>
inline cudaError_t persistent_grid(K kernel, int threads, size_t smem,
                                   uint64_t units, const LaunchCfg &cfg,
                                   unsigned *grid, std::atomic<int> *occ_cache)
{
    int err = 0;
    const int sms = sm_count(&err);
    if (err) return (cudaError_t)err;
    int occ = cfg.ctas_per_sm;
    if (occ <= 0) {
        occ = occ_cache->load(std::memory_order_relaxed);
        if (occ <= 0) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel,
                                                                          threads, smem);
            if (e != cudaSuccess) return e;
            if (occ < 1) occ = 1;
            occ_cache->store(occ, std::memory_order_relaxed);
        }
    }
    uint64_t g = (uint64_t)sms * (uint64_t)occ;
    if (units < g) g = units;
    if (g < 1) g = 1;
    *grid = (unsigned)g;
    return cudaSuccess;
}

}  // namespace sg
