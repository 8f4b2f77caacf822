// sg_stencil.cu -- per-cell stencils over the embedded gasket: the B3/S23
// cellular automaton (uint8) and explicit diffusion (float32).
//
// The embedded layout keeps (x +- 1, y +- 1) a neighbourhood of the gasket
// (Section I), so a tile's update needs the tile plus a one-cell halo.  The
// CA at rho = 32, 64 and diffusion at rho = 16, 32 run one warp per tile
// (below).  For the other vector sizes -- CA rho = 16, diffusion rho = 4,
// 8, 64 -- a CTA processes groups of TPC tiles (TPC * tile chunks ~ 256
// threads; stencil_pipeline in sg_stencil.cuh):
//   1. decode:  one warp per tile runs the lambda(omega) reduction of
//               Theorem 1 (LambdaLane) or the bounding-box identity map;
//   2. stage:   the tile and a one-chunk halo are copied to shared memory in
//               16-byte chunks with cp.async, double-buffered (the next
//               group's copies are in flight while this one is computed);
//               only chunks holding in-grid gasket cells are read from HBM,
//               the others are zero-filled;
//   3. compute: each thread produces 16-byte chunks of the output tile from
//               shared memory and stores them by whole 32-byte sectors where
//               the sector holds gasket cells.
// Smaller tiles take one cell per thread and read the halo cell by cell (in
// a non-empty tile the gasket leaves at most the right column, the bottom
// row and five isolated cells of it).
// Off-gasket cells are 0 in every state (precondition of the ABI), so a
// neighbour sum over the plain neighbourhood only ever sees gasket cells.
//
// Tiles that hold no gasket cell are never launched by lambda; under the
// bounding-box map every tile is visited and the cells of an empty tile drop
// out at their membership test.
#include "sg_stencil.cuh"
#include "sg_stencil_tma.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// CA, rho >= 16: 16-cell chunks.
// ---------------------------------------------------------------------------
template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
ca_vec_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r,
              int order, uint64_t ntiles)
{
    using G = StencilGroup<uint8_t, S>;
    __shared__ __align__(16) uint8_t sm[2 * G::TPC * G::TILE];
    __shared__ StencilTile<uint8_t> tiles[2 * G::TPC];

    const int rb = r - S;
    LambdaLane ll;
    ll.init(threadIdx.x & 31, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t groups = (ntiles + G::TPC - 1) / G::TPC;
    auto decode = [&](uint64_t g, StencilTile<uint8_t> *dst) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int t = warp; t < G::TPC; t += kStencilThreads / 32) {
            const uint2 c = decode_tile<MAP>(g * G::TPC + t, ntiles, rb, W, ll);
            if (lane == 0) dst[t] = StencilTile<uint8_t>{c.x, c.y, r, in, out};
        }
    };
    auto compute = [](const uint8_t *buf, const StencilTile<uint8_t> *slot) {
        ca_compute_group<S>(buf, slot);
    };
    stencil_pipeline<uint8_t, S>(sm, tiles, groups, decode, compute);
}

// ---------------------------------------------------------------------------
// One warp per tile (CA for rho = 32, 64; diffusion for rho = 16, 32).  Each
// warp stages its own tile and halo (cp.async, chunks without in-grid gasket
// cells zero-filled), waits for its own copies, and computes the tile: no
// CTA barrier anywhere, so a warp that waits for memory holds up no other
// warp, and eight resident warps per CTA keep the SM busy.  Measured faster
// than the CTA-wide pipeline at these sizes; larger float tiles do not fit
// eight warps' shared memory, and at rho = 16 a byte tile gives a warp too
// little work.
// ---------------------------------------------------------------------------
template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
ca_warp_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r, int order,
               uint64_t ntiles)
{
    using G = StencilGroup<uint8_t, S>;
    extern __shared__ __align__(16) unsigned char warp_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *sm = warp_smem + warp * G::TILE;
    const int rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t stride = (uint64_t)gridDim.x * kWarpTileWarps;
    for (uint64_t q = (uint64_t)blockIdx.x * kWarpTileWarps + warp; q < ntiles; q += stride) {
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        if (c.x == kNoTile) continue;                                // uniform in the warp
        warp_stage<uint8_t, S>(sm, in, r, (int)(c.x << S), (int)(c.y << S), lane);
        const StencilTile<uint8_t> tl{c.x, c.y, r, in, out};
        for (int k = lane; k < G::CHUNKS; k += 32) ca_chunk<S>(sm, tl, 0, k);
        __syncwarp();                    // the tile is read before the next staging
    }
}

template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
diffuse_warp_kernel(const float *__restrict__ in, float *__restrict__ out, int r, int order,
                    uint64_t ntiles, float alpha)
{
    using G = StencilGroup<float, S>;
    extern __shared__ __align__(16) unsigned char warp_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sm = reinterpret_cast<float *>(warp_smem) + warp * G::TILE;
    const int rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t stride = (uint64_t)gridDim.x * kWarpTileWarps;
    for (uint64_t q = (uint64_t)blockIdx.x * kWarpTileWarps + warp; q < ntiles; q += stride) {
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        if (c.x == kNoTile) continue;                                // uniform in the warp
        warp_stage<float, S>(sm, in, r, (int)(c.x << S), (int)(c.y << S), lane);
        const StencilTile<float> tl{c.x, c.y, r, in, out};
        for (int k = lane; k < G::CHUNKS; k += 32) diffuse_chunk<S>(sm, tl, 0, k, alpha);
        __syncwarp();                    // the tile is read before the next staging
    }
}

// ---------------------------------------------------------------------------
// CA, rho <= 8: one cell per thread.
// ---------------------------------------------------------------------------
template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
ca_cell_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r,
               int order, uint64_t ntiles)
{
    constexpr int RHO = 1 << S, CELLS = RHO * RHO;
    constexpr int TPC = kStencilThreads / CELLS;
    constexpr int P = RHO + 2, TILE = P * P, HALO = 4 * RHO + 4;
    __shared__ uint8_t sm[TPC * TILE];
    __shared__ uint2 coord[TPC];

    const int rb = r - S;
    LambdaLane ll;
    ll.init(threadIdx.x & 31, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t groups = (ntiles + TPC - 1) / TPC;

    for (uint64_t g = blockIdx.x; g < groups; g += gridDim.x) {
        __syncthreads();
        decode_tiles<MAP>(coord, TPC, g, ntiles, rb, W, ll);
        __syncthreads();
        {
            const int c = threadIdx.x, t = c / CELLS, k = c % CELLS;
            const int ty = k / RHO, tx = k % RHO;
            const uint2 b = coord[t];
            uint8_t v = 0;
            if (b.x != kNoTile)
                v = load_cell(in, r, (int64_t)(b.x << S) + tx, (int64_t)(b.y << S) + ty);
            sm[t * TILE + (ty + 1) * P + tx + 1] = v;
        }
        for (int c = threadIdx.x; c < TPC * HALO; c += kStencilThreads) {
            const int t = c / HALO, h = c % HALO;
            int row, col;
            halo_slot<RHO>(h, row, col);
            const uint2 b = coord[t];
            uint8_t v = 0;
            if (b.x != kNoTile)
                v = load_cell(in, r, (int64_t)(b.x << S) + col, (int64_t)(b.y << S) + row);
            sm[t * TILE + (row + 1) * P + col + 1] = v;
        }
        __syncthreads();
        {
            const int c = threadIdx.x, t = c / CELLS, k = c % CELLS;
            const int ty = k / RHO, tx = k % RHO;
            const uint2 b = coord[t];
            if (b.x != kNoTile) {
                const uint32_t x = (b.x << S) + tx, y = (b.y << S) + ty;
                if (in_gasket(x, y)) {
                    const uint8_t *p = sm + t * TILE + (ty + 1) * P + tx + 1;
                    const int cnt = p[-P - 1] + p[-P] + p[-P + 1] + p[-1] + p[1] +
                                    p[P - 1] + p[P] + p[P + 1];
                    out[((uint64_t)y << r) + x] = (uint8_t)((cnt | p[0]) == 3);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Diffusion (diffuse_cell, in sg_stencil.cuh, gives one cell's update).
// ---------------------------------------------------------------------------
// rho >= 4: 4-cell chunks (float4).
template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
diffuse_vec_kernel(const float *__restrict__ in, float *__restrict__ out, int r,
                   int order, uint64_t ntiles, float alpha)
{
    using G = StencilGroup<float, S>;
    __shared__ __align__(16) float sm[2 * G::TPC * G::TILE];
    __shared__ StencilTile<float> tiles[2 * G::TPC];

    const int rb = r - S;
    LambdaLane ll;
    ll.init(threadIdx.x & 31, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t groups = (ntiles + G::TPC - 1) / G::TPC;
    auto decode = [&](uint64_t g, StencilTile<float> *dst) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int t = warp; t < G::TPC; t += kStencilThreads / 32) {
            const uint2 c = decode_tile<MAP>(g * G::TPC + t, ntiles, rb, W, ll);
            if (lane == 0) dst[t] = StencilTile<float>{c.x, c.y, r, in, out};
        }
    };
    auto compute = [alpha](const float *buf, const StencilTile<float> *slot) {
        diffuse_compute_group<S>(buf, slot, alpha);
    };
    stencil_pipeline<float, S>(sm, tiles, groups, decode, compute);
}

// rho <= 2: one cell per thread.
template <int S, int MAP>
__global__ void __launch_bounds__(kStencilThreads)
diffuse_cell_kernel(const float *__restrict__ in, float *__restrict__ out, int r,
                    int order, uint64_t ntiles, float alpha)
{
    constexpr int RHO = 1 << S, CELLS = RHO * RHO;
    constexpr int TPC = kStencilThreads / CELLS;
    constexpr int P = RHO + 2, TILE = P * P, HALO = 4 * RHO + 4;
    __shared__ float sm[TPC * TILE];
    __shared__ uint2 coord[TPC];

    const int rb = r - S;
    const uint32_t n = 1u << r;
    LambdaLane ll;
    ll.init(threadIdx.x & 31, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t groups = (ntiles + TPC - 1) / TPC;

    for (uint64_t g = blockIdx.x; g < groups; g += gridDim.x) {
        __syncthreads();
        decode_tiles<MAP>(coord, TPC, g, ntiles, rb, W, ll);
        __syncthreads();
        {
            const int c = threadIdx.x, t = c / CELLS, k = c % CELLS;
            const int ty = k / RHO, tx = k % RHO;
            const uint2 b = coord[t];
            float v = 0.f;
            if (b.x != kNoTile)
                v = load_cell(in, r, (int64_t)(b.x << S) + tx, (int64_t)(b.y << S) + ty);
            sm[t * TILE + (ty + 1) * P + tx + 1] = v;
        }
        for (int c = threadIdx.x; c < TPC * HALO; c += kStencilThreads) {
            const int t = c / HALO, h = c % HALO;
            int row, col;
            halo_slot<RHO>(h, row, col);
            const uint2 b = coord[t];
            float v = 0.f;
            if (b.x != kNoTile)
                v = load_cell(in, r, (int64_t)(b.x << S) + col, (int64_t)(b.y << S) + row);
            sm[t * TILE + (row + 1) * P + col + 1] = v;
        }
        __syncthreads();
        {
            const int c = threadIdx.x, t = c / CELLS, k = c % CELLS;
            const int ty = k / RHO, tx = k % RHO;
            const uint2 b = coord[t];
            if (b.x != kNoTile) {
                const uint32_t x = (b.x << S) + tx, y = (b.y << S) + ty;
                if (in_gasket(x, y)) {
                    const float *p = sm + t * TILE + (ty + 1) * P + tx + 1;
                    out[((uint64_t)y << r) + x] =
                        diffuse_cell(x, y, n, p[0], p[-1], p[1], p[-P], p[P], alpha);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int S, int MAP>
cudaError_t launch_ca_t(int r, const uint8_t *in, uint8_t *out, cudaStream_t st,
                        const LaunchCfg &cfg)
{
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    constexpr int TPC = S >= 4 ? StencilGroup<uint8_t, (S >= 4 ? S : 4)>::TPC
                               : kStencilThreads / ((1 << S) * (1 << S));
    const uint64_t groups = (ntiles + TPC - 1) / TPC;
    unsigned grid = 1;
    cudaError_t e;
    if (cfg.store == kStoreTma) {          // tile and halo by one tensor copy
        if constexpr (S >= 5) return launch_ca_tma<S, MAP>(r, in, out, ntiles, st, cfg);
        else return cudaErrorNotSupported;
    }
    if constexpr (S >= 5) {
        static std::atomic<int> occ{0};
        static std::atomic<uint64_t> attr{0};
        auto k = ca_warp_kernel<S, MAP>;
        constexpr int smem = kWarpTileWarps * StencilGroup<uint8_t, (S >= 4 ? S : 4)>::TILE;
        e = dyn_smem_grid(k, smem, (ntiles + kWarpTileWarps - 1) / kWarpTileWarps, cfg, &grid,
                          &occ, &attr);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, smem, st>>>(in, out, r, cfg.order, ntiles);
    } else if constexpr (S == 4) {
        static std::atomic<int> occ{0};
        auto k = ca_vec_kernel<S, MAP>;
        e = persistent_grid(k, kStencilThreads, 0, groups, cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, 0, st>>>(in, out, r, cfg.order, ntiles);
    } else {
        static std::atomic<int> occ{0};
        auto k = ca_cell_kernel<S, MAP>;
        e = persistent_grid(k, kStencilThreads, 0, groups, cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, 0, st>>>(in, out, r, cfg.order, ntiles);
    }
    return cudaGetLastError();
}

template <int S, int MAP>
cudaError_t launch_diffuse_t(int r, const float *in, float *out, float alpha,
                             cudaStream_t st, const LaunchCfg &cfg)
{
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    constexpr int TPC = S >= 2 ? StencilGroup<float, (S >= 2 ? S : 2)>::TPC
                               : kStencilThreads / ((1 << S) * (1 << S));
    const uint64_t groups = (ntiles + TPC - 1) / TPC;
    unsigned grid = 1;
    cudaError_t e;
    if (cfg.store == kStoreTma) {          // tile and halo by one tensor copy
        if constexpr (S == 4 || S == 5)
            return launch_diffuse_tma<S, MAP>(r, in, out, alpha, ntiles, st, cfg);
        else return cudaErrorNotSupported;
    }
    if constexpr (S == 4 || S == 5) {
        static std::atomic<int> occ{0};
        static std::atomic<uint64_t> attr{0};
        auto k = diffuse_warp_kernel<S, MAP>;
        constexpr int smem = kWarpTileWarps * StencilGroup<float, (S >= 2 ? S : 2)>::TILE *
                             (int)sizeof(float);
        e = dyn_smem_grid(k, smem, (ntiles + kWarpTileWarps - 1) / kWarpTileWarps, cfg, &grid,
                          &occ, &attr);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, smem, st>>>(in, out, r, cfg.order, ntiles, alpha);
    } else if constexpr (S >= 2) {
        static std::atomic<int> occ{0};
        auto k = diffuse_vec_kernel<S, MAP>;
        e = persistent_grid(k, kStencilThreads, 0, groups, cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, 0, st>>>(in, out, r, cfg.order, ntiles, alpha);
    } else {
        static std::atomic<int> occ{0};
        auto k = diffuse_cell_kernel<S, MAP>;
        e = persistent_grid(k, kStencilThreads, 0, groups, cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, 0, st>>>(in, out, r, cfg.order, ntiles, alpha);
    }
    return cudaGetLastError();
}

#define SG_S_SWITCH(s, CALL)                 \
    switch (s) {                             \
    case 0: return CALL(0);                  \
    case 1: return CALL(1);                  \
    case 2: return CALL(2);                  \
    case 3: return CALL(3);                  \
    case 4: return CALL(4);                  \
    case 5: return CALL(5);                  \
    case 6: return CALL(6);                  \
    default: return cudaErrorInvalidValue;   \
    }

cudaError_t launch_ca(int r, int s, int map, const uint8_t *in, uint8_t *out,
                      cudaStream_t st, const LaunchCfg &cfg)
{
    if (map == kMapBBox) {
#define CALL(S) launch_ca_t<S, kMapBBox>(r, in, out, st, cfg)
        SG_S_SWITCH(s, CALL)
#undef CALL
    }
#define CALL(S) launch_ca_t<S, kMapLambda>(r, in, out, st, cfg)
    SG_S_SWITCH(s, CALL)
#undef CALL
}

cudaError_t launch_diffuse(int r, int s, int map, const float *in, float *out,
                           float alpha, cudaStream_t st, const LaunchCfg &cfg)
{
    if (map == kMapBBox) {
#define CALL(S) launch_diffuse_t<S, kMapBBox>(r, in, out, alpha, st, cfg)
        SG_S_SWITCH(s, CALL)
#undef CALL
    }
#define CALL(S) launch_diffuse_t<S, kMapLambda>(r, in, out, alpha, st, cfg)
    SG_S_SWITCH(s, CALL)
#undef CALL
}

}  // namespace sg
