// sg_stencil_tma.cuh -- the warp-per-tile single-step stencils with the tile
// and its halo staged by one 2-D bulk tensor copy (TMA) instead of 16-byte
// cp.async chunks (selected with SG_STORE_TMA in sg_launch_opts).
//
// The staged region is the cp.async form's: rho + 2 rows of whole 16-byte
// chunks from one chunk left of the tile to one chunk right of it, laid out
// densely with the same row pitch, so the compute is shared.  The copy's box
// starts at (x0 - one chunk, y0 - 1): its x is a multiple of 16 bytes, a
// negative or out-of-range coordinate reads 0, and chunks that hold no gasket
// cell read the 0 the grid holds there (the ABI's precondition), so the
// staged tile is the same as the cp.async one.  The difference is that the
// box moves every chunk of the region, where the cp.async form skips the ones
// without gasket cells.
//
// Each warp waits on an mbarrier of its own, bounded as every wait in the
// library: a wait that gives up records SG_ETIMEOUT, waits (bounded) once
// more for its copy, and the warp returns.
#pragma once

#include "sg_stencil.cuh"
#include "sg_tma.cuh"

namespace sg {

template <typename T, int S> struct TmaStage {
    using G = StencilGroup<T, S>;
    static constexpr int BOX_W = G::PC * G::CE;                  // elements per box row
    static constexpr int BOX_H = G::ROWS;
    static constexpr int BYTES = BOX_W * BOX_H * (int)sizeof(T); // = the staged tile
    static constexpr int SLOT = (BYTES + 127) / 128 * 128;       // 128-byte aligned slots
    static constexpr int SMEM = kWarpTileWarps * SLOT + 128;     // + alignment slack
    static_assert(BOX_W * (int)sizeof(T) % 16 == 0 && BOX_W <= 256 && BOX_H <= 256,
                  "a tensor-copy box row is a multiple of 16 bytes, sides at most 256");
    static_assert(BYTES == G::TILE * (int)sizeof(T), "the box is the staged tile");
};

// Stage the tile at (x0, y0) into sm with one tensor copy; true when it
// landed (false: the wait gave up, recorded, and the copy was waited for).
template <typename T, int S>
__device__ __forceinline__ bool tma_stage_tile(T *sm, const CUtensorMap *tmap, uint64_t *bar,
                                               uint32_t &phase, int x0, int y0, int lane,
                                               int *status)
{
    using G = StencilGroup<T, S>;
    using TS = TmaStage<T, S>;
    // the previous tile's shared-memory reads come before the copy's writes
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)TS::BYTES);
        tma_load_2d(sm, tmap, x0 - G::CE, y0 - 1, bar);
    }
    const bool got = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar, phase));
    if (!got) {
        if (lane == 0) record_device_error(status, kDevTimeout);
        (void)mbar_wait_bounded(bar, phase);
        return false;
    }
    phase ^= 1u;
    return true;
}

template <typename T, int S>
__device__ __forceinline__ T *tma_warp_slot(unsigned char *raw, int warp)
{
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(raw) + 127) & ~(uintptr_t)127);
    return reinterpret_cast<T *>(base + (size_t)warp * TmaStage<T, S>::SLOT);
}

template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
ca_warp_tma_kernel(const __grid_constant__ CUtensorMap tmap, uint8_t *__restrict__ out, int r,
                   int order, uint64_t ntiles, int *status)
{
    using G = StencilGroup<uint8_t, S>;
    extern __shared__ unsigned char tma_stencil_smem[];
    __shared__ __align__(8) uint64_t bar[kWarpTileWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *sm = tma_warp_slot<uint8_t, S>(tma_stencil_smem, warp);
    if (lane == 0) mbar_init(&bar[warp], 1);
    mbar_init_fence();
    __syncwarp();
    const int rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    uint32_t phase = 0;
    const uint64_t stride = (uint64_t)gridDim.x * kWarpTileWarps;
    for (uint64_t q = (uint64_t)blockIdx.x * kWarpTileWarps + warp; q < ntiles; q += stride) {
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        if (c.x == kNoTile) continue;                                // uniform in the warp
        if (!tma_stage_tile<uint8_t, S>(sm, &tmap, &bar[warp], phase, (int)(c.x << S),
                                        (int)(c.y << S), lane, status))
            return;
        const StencilTile<uint8_t> tl{c.x, c.y, r, nullptr, out};
        for (int k = lane; k < G::CHUNKS; k += 32) ca_chunk<S>(sm, tl, 0, k);
        __syncwarp();
    }
}

template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
diffuse_warp_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ out, int r,
                        int order, uint64_t ntiles, float alpha, int *status)
{
    using G = StencilGroup<float, S>;
    extern __shared__ unsigned char tma_stencil_smem[];
    __shared__ __align__(8) uint64_t bar[kWarpTileWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sm = tma_warp_slot<float, S>(tma_stencil_smem, warp);
    if (lane == 0) mbar_init(&bar[warp], 1);
    mbar_init_fence();
    __syncwarp();
    const int rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    uint32_t phase = 0;
    const uint64_t stride = (uint64_t)gridDim.x * kWarpTileWarps;
    for (uint64_t q = (uint64_t)blockIdx.x * kWarpTileWarps + warp; q < ntiles; q += stride) {
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        if (c.x == kNoTile) continue;                                // uniform in the warp
        if (!tma_stage_tile<float, S>(sm, &tmap, &bar[warp], phase, (int)(c.x << S),
                                      (int)(c.y << S), lane, status))
            return;
        const StencilTile<float> tl{c.x, c.y, r, nullptr, out};
        for (int k = lane; k < G::CHUNKS; k += 32) diffuse_chunk<S>(sm, tl, 0, k, alpha);
        __syncwarp();
    }
}

template <int S, int MAP>
cudaError_t launch_ca_tma(int r, const uint8_t *in, uint8_t *out, uint64_t ntiles,
                          cudaStream_t st, const LaunchCfg &cfg)
{
    using TS = TmaStage<uint8_t, S>;
    CUtensorMap map;
    cudaError_t e = make_box_tensor_map(&map, const_cast<uint8_t *>(in), r, 1, TS::BOX_W,
                                        TS::BOX_H);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = device_status_ptr(&status);
    if (e != cudaSuccess) return e;
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    auto k = ca_warp_tma_kernel<S, MAP>;
    unsigned grid = 1;
    e = dyn_smem_grid(k, TS::SMEM, (ntiles + kWarpTileWarps - 1) / kWarpTileWarps, cfg, &grid,
                      &occ, &attr);
    if (e != cudaSuccess) return e;
    k<<<grid, kStencilThreads, TS::SMEM, st>>>(map, out, r, cfg.order, ntiles, status);
    return cudaGetLastError();
}

template <int S, int MAP>
cudaError_t launch_diffuse_tma(int r, const float *in, float *out, float alpha, uint64_t ntiles,
                               cudaStream_t st, const LaunchCfg &cfg)
{
    using TS = TmaStage<float, S>;
    CUtensorMap map;
    cudaError_t e = make_box_tensor_map(&map, const_cast<float *>(in), r, 4, TS::BOX_W,
                                        TS::BOX_H);
    if (e != cudaSuccess) return e;
    int *status = nullptr;
    e = device_status_ptr(&status);
    if (e != cudaSuccess) return e;
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    auto k = diffuse_warp_tma_kernel<S, MAP>;
    unsigned grid = 1;
    e = dyn_smem_grid(k, TS::SMEM, (ntiles + kWarpTileWarps - 1) / kWarpTileWarps, cfg, &grid,
                      &occ, &attr);
    if (e != cudaSuccess) return e;
    k<<<grid, kStencilThreads, TS::SMEM, st>>>(map, out, r, cfg.order, ntiles, alpha, status);
    return cudaGetLastError();
}

}  // namespace sg
