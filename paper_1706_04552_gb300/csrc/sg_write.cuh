// sg_write.cuh -- the map-and-write pass (Section IV of the paper): every
// gasket cell of a level-r grid receives v(x, y), nothing else is touched.
//
// One persistent kernel template serves the four maps.  A "team" (one warp
// for rho <= 16, the whole 256-thread CTA for rho >= 32) owns one tile at a
// time and walks its share of the tile list with a fixed stride:
//   lambda (all three intra-tile variants): the team decodes its tile with
//     the warp-parallel lambda(omega) of Theorem 1 (LambdaLane);
//   bounding box: tile q is (q mod n_b, q div n_b), the identity map.
// Inside a tile each thread visits a fixed list of tile-relative offsets,
// which does not depend on the tile, so it is computed once and kept in
// registers:
//   sub-box (lambda, bounding box): every slot of the rho x rho tile, each
//     tested with (x & y) == 0 (Section III-D, Bounding Sub-boxes);
//   lookup table: the 3^s member slots in row-major order, built once per
//     CTA in shared memory (Section III-D, Shared Lookup Table);
//   further unrolling: slot e is mapped by lambda applied at thread level
//     (Section III-D, Further Unrolling).
// Threads of a warp visit consecutive slots of a tile row, so stores of
// a warp fall in few 32-byte sectors; u8 stores are byte stores merged by
// the coalescer (only gasket bytes may change, so a wider store would
// overwrite cells the pass must leave alone).
#pragma once

#include "sg_device.cuh"
#include "sg_internal.h"

namespace sg {

constexpr int kWriteThreads = 256;

template <int S> struct WriteShape {
    static constexpr int RHO = 1 << S;
    static constexpr int SLOTS = RHO * RHO;
    static constexpr int MEMBERS = pow3i(S);
    static constexpr int TEAM = (S >= 5) ? kWriteThreads : 32;
};

// Row-major rank of member slot (tx, ty) among the 3^S members of a level-S
// tile: all members of earlier rows, then the members of row ty left of tx.
// Row t holds 2^(S - popcount(t)) members (the subsets of ~t); inside a row
// the members, ordered by tx, are the bits of tx at the zero positions of ty.
template <int S>
__device__ __forceinline__ int member_rank(int tx, int ty)
{
    int rank = 0;
    for (int t = 0; t < ty; ++t) rank += 1 << (S - __popc(t));
    int k = 0, bit = 0;
#pragma unroll
    for (int b = 0; b < S; ++b)
        if (!((ty >> b) & 1)) { k |= ((tx >> b) & 1) << bit; ++bit; }
    return rank + k;
}

// Slot e of a level-S tile under further unrolling: lambda of Theorem 1 at
// thread level (omega = (e mod 3^floor(S/2), e div 3^floor(S/2))), mirrored
// into the (x & y) == 0 orientation.  Returns tx | ty << 8.
template <int S>
__device__ __forceinline__ uint32_t unrolled_offset(int e)
{
    constexpr int WS = pow3i(S / 2);
    const int wx = e % WS, wy = e / WS;
    int lx = 0, ly = 0;
#pragma unroll
    for (int mu = 1; mu <= S; ++mu) {
        int w = (mu & 1) ? wy : wx;
        for (int i = 0; i < (mu + 1) / 2 - 1; ++i) w /= 3;
        const int beta = w % 3;
        const int dx = beta >> 1, dy = beta - dx;
        lx += dx << (mu - 1);
        ly += dy << (mu - 1);
    }
    return (uint32_t)lx | ((uint32_t)((1 << S) - 1 - ly) << 8);
}

template <typename T, int VK, int S, int MAP>
__global__ void __launch_bounds__(kWriteThreads)
write_kernel(T *__restrict__ grid, int r, uint64_t vs, uint64_t ntiles, uint32_t W)
{
    using WS = WriteShape<S>;
    constexpr int RHO = WS::RHO;
    constexpr int TEAM = WS::TEAM;
    constexpr bool SUBBOX = (MAP == kMapLambda || MAP == kMapBBox);
    constexpr int NSLOT = SUBBOX ? WS::SLOTS : WS::MEMBERS;
    constexpr int ITERS = (NSLOT + TEAM - 1) / TEAM;
    constexpr int TEAMS_PER_CTA = kWriteThreads / TEAM;

    const int lane = threadIdx.x & 31;
    const int t_in_team = threadIdx.x % TEAM;
    const uint64_t team = (uint64_t)blockIdx.x * TEAMS_PER_CTA + threadIdx.x / TEAM;
    const uint64_t nteams = (uint64_t)gridDim.x * TEAMS_PER_CTA;
    const int rb = r - S;
    const uint64_t seedmix = vs * kGoldenGamma;

    // Tile-independent offsets of this thread: tx | ty << 8, or ~0u if none.
    uint32_t off[ITERS];
    if constexpr (MAP == kMapLut) {
        __shared__ uint16_t lut[WS::MEMBERS];
        for (int slot = threadIdx.x; slot < WS::SLOTS; slot += kWriteThreads) {
            const int tx = slot & (RHO - 1), ty = slot >> S;
            if ((tx & ty) == 0) lut[member_rank<S>(tx, ty)] = (uint16_t)(tx | (ty << 8));
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int e = t_in_team + j * TEAM;
            off[j] = (e < WS::MEMBERS) ? (uint32_t)lut[e] : ~0u;
        }
    } else if constexpr (MAP == kMapUnroll) {
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int e = t_in_team + j * TEAM;
            off[j] = (e < WS::MEMBERS) ? unrolled_offset<S>(e) : ~0u;
        }
    } else {
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int slot = t_in_team + j * TEAM;
            off[j] = (slot < WS::SLOTS)
                         ? (uint32_t)((slot & (RHO - 1)) | ((slot >> S) << 8)) : ~0u;
        }
    }

    LambdaLane ll;
    OmegaWalker ow;
    if constexpr (MAP != kMapBBox) {
        ll.init(lane, rb);
        ow.init((uint32_t)team, (uint32_t)nteams, W);
    }
    for (uint64_t q = team; q < ntiles; q += nteams) {
        uint32_t bx, by;
        if constexpr (MAP == kMapBBox) {
            bx = (uint32_t)(q & ((1ull << rb) - 1));
            by = (uint32_t)(q >> rb);
        } else {
            const uint2 b = ll.decode(ow.wx, ow.wy);
            bx = b.x;
            by = b.y;
            ow.advance();
        }
        const uint32_t x0 = bx << S, y0 = by << S;
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            if (off[j] == ~0u) continue;
            // offsets are masked to the tile, so every address stays inside it
            const uint32_t x = x0 + (off[j] & (RHO - 1)), y = y0 + ((off[j] >> 8) & (RHO - 1));
            if (SUBBOX && !in_gasket(x, y)) continue;
            grid[((uint64_t)y << r) + x] = Value<T>::template at<VK>(x, y, r, vs, seedmix);
        }
    }
}

template <typename T, int VK, int S, int MAP>
cudaError_t launch_write_t(int r, T *grid, uint64_t vs, cudaStream_t st,
                           const LaunchCfg &cfg)
{
    using WS = WriteShape<S>;
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    const uint32_t W = (uint32_t)pow3i(rb / 2);
    auto kern = write_kernel<T, VK, S, MAP>;
    const uint64_t units = (ntiles * WS::TEAM + kWriteThreads - 1) / kWriteThreads;
    unsigned grid_ctas = 1;
    cudaError_t e = persistent_grid(kern, kWriteThreads, 0, units, cfg, &grid_ctas);
    if (e != cudaSuccess) return e;
    kern<<<grid_ctas, kWriteThreads, 0, st>>>(grid, r, vs, ntiles, W);
    return cudaGetLastError();
}

template <typename T, int VK, int MAP>
cudaError_t launch_write_s(int r, int s, T *grid, uint64_t vs, cudaStream_t st,
                           const LaunchCfg &cfg)
{
    switch (s) {
    case 0: return launch_write_t<T, VK, 0, MAP>(r, grid, vs, st, cfg);
    case 1: return launch_write_t<T, VK, 1, MAP>(r, grid, vs, st, cfg);
    case 2: return launch_write_t<T, VK, 2, MAP>(r, grid, vs, st, cfg);
    case 3: return launch_write_t<T, VK, 3, MAP>(r, grid, vs, st, cfg);
    case 4: return launch_write_t<T, VK, 4, MAP>(r, grid, vs, st, cfg);
    case 5: return launch_write_t<T, VK, 5, MAP>(r, grid, vs, st, cfg);
    case 6: return launch_write_t<T, VK, 6, MAP>(r, grid, vs, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int VK>
cudaError_t launch_write_m(int r, int s, int map, T *grid, uint64_t vs,
                           cudaStream_t st, const LaunchCfg &cfg)
{
    switch (map) {
    case kMapLambda: return launch_write_s<T, VK, kMapLambda>(r, s, grid, vs, st, cfg);
    case kMapBBox: return launch_write_s<T, VK, kMapBBox>(r, s, grid, vs, st, cfg);
    case kMapLut: return launch_write_s<T, VK, kMapLut>(r, s, grid, vs, st, cfg);
    case kMapUnroll: return launch_write_s<T, VK, kMapUnroll>(r, s, grid, vs, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_write_any(int r, int s, int map, int vk, T *grid, uint64_t vs,
                             cudaStream_t st, const LaunchCfg &cfg)
{
    switch (vk) {
    case kValConst: return launch_write_m<T, kValConst>(r, s, map, grid, vs, st, cfg);
    case kValLinear31: return launch_write_m<T, kValLinear31>(r, s, map, grid, vs, st, cfg);
    case kValHash: return launch_write_m<T, kValHash>(r, s, map, grid, vs, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sg
