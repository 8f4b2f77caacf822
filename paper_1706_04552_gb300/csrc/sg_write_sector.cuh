// sg_write_sector.cuh -- the map-and-write pass (Section IV) with one lane per
// unit and 32-byte sector accesses.
//
// A unit is a U x U piece of a rho-tile: U = 32 for uint8 grids (a tile row
// of 32 bytes is one sector) and U = min(rho, 32) for float32 (8 floats a
// sector).  A 64-tile is its units that hold gasket cells (three for lambda;
// for the bounding box four, the empty one skipped).  Lane l of a warp takes
// unit 32 t + l of the warp's task t, so the 32 lanes work on 32 units side by
// side and every 32-byte access instruction of the warp moves 32 whole
// sectors.
//
// A sector on row y starting at column x0 (a multiple of the sector's E
// elements) holds a gasket cell iff (x0 & y) == 0, and then its gasket cells
// are the x0 + j with (j & y & (E - 1)) == 0.  Inside a unit both tests depend
// only on the row, so every lane of a warp walks the same rows and sectors in
// the same order and computes the same cells of its own unit; the per-row
// tests are uniform branches, the per-cell ones compile-time constants.
//
// Three ways to store:
//   kStoreSector (write-only): each sector holding gasket cells is written
//     whole, v(x, y) at its gasket cells and 0 elsewhere; nothing is read.
//     Equal to the preserving modes whenever the grid is 0 off the gasket.
//   kStoreMerge: each such sector is read, its gasket cells replaced, and
//     written back whole (a read-modify-write; no other kernel may write the
//     grid meanwhile).
//   kStoreMasked: only the gasket cells are stored (a 4-, 2- or 1-byte store
//     per group of neighbouring gasket cells); the L2 merges them into the
//     sector, reading what it does not hold from DRAM.  Only gasket cells ever
//     change.
//
// The tile of each unit comes from the lambda(omega) decode of Theorem 1
// (LambdaLane, one warp reduction per tile; the warp decodes the tiles its 32
// units span, one after the other) or from the bounding-box identity map, in
// which a lane whose tile holds no gasket cell does nothing, as the empty
// blocks of the paper's bounding-box launch do.
#pragma once

#include "sg_device.cuh"
#include "sg_internal.h"

namespace sg {

// 32-byte global accesses (sm_100 and later: 256-bit vector loads and stores).
__device__ __forceinline__ void st_global_v8(void *p, const uint32_t (&v)[8])
{
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void ld_global_v8(const void *p, uint32_t (&v)[8])
{
    asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "l"(p)
                 : "memory");
}

constexpr int kSectorThreads = 256;
constexpr uint32_t kNoUnit = 0xFFFFFFFFu;

template <typename T, int S> struct SectorShape {
    static constexpr int E = 32 / (int)sizeof(T);                 // elements per sector
    static constexpr int US = sizeof(T) == 1 ? 32 : ((1 << S) < 32 ? (1 << S) : 32);
    static constexpr int LU = sizeof(T) == 1 ? 5 : (S < 5 ? S : 5);   // log2(US)
    static constexpr int SUB = S - LU;                            // unit levels in a tile
    static constexpr bool OK = (1 << S) * (int)sizeof(T) >= 32;
};

// The value of each cell of one row of a unit: a per-row part and a per-cell
// constant, as CellValue computes them (the hash state is
// (seed * gamma) ^ (y * n + x), the linear value x * 31 + y).
template <typename T, int VK> struct RowValue {
    uint32_t seed_hi, cval;
    uint32_t row;      // hash: low word of the state for (x0, y); linear: x0 * 31 + y
    __device__ __forceinline__ void set_row(uint64_t seedmix, uint32_t x0, uint32_t y, int r)
    {
        if constexpr (VK == kValHash) row = (uint32_t)seedmix ^ ((y << r) | x0);
        else if constexpr (VK == kValLinear31) row = x0 * 31u + y;
    }
    // raw bits of the value of cell x0 + dx (low byte for uint8)
    __device__ __forceinline__ uint32_t bits(uint32_t dx) const
    {
        if constexpr (VK == kValConst) {
            return sizeof(T) == 1 ? (cval & 0xFFu) : cval;
        } else if constexpr (VK == kValLinear31) {
            if constexpr (sizeof(T) == 1) return (row + 31u * dx) & 0xFFu;
            else return __float_as_uint((float)((row + 31u * dx) & 0xFFu));
        } else {
            const uint32_t hi = splitmix64_hi_state(row ^ dx, seed_hi);
            if constexpr (sizeof(T) == 1) return hi >> 24;
            else return __float_as_uint((float)(hi >> 8) * (1.0f / 16777216.0f));
        }
    }
};

// One unit of a uint8 grid (32 x 32 cells at (x0, y0)).  Rows come in groups
// of four, ty = 4 th + tl: word w (bytes 4w .. 4w+3) of a row holds gasket
// cells iff (w & th) == 0, and then they are the bytes b with (b & tl) == 0.
template <int VK, int MODE>
__device__ __forceinline__ void sector_unit_u8(uint8_t *__restrict__ grid, int r, uint32_t x0,
                                               uint32_t y0, uint64_t seedmix,
                                               RowValue<uint8_t, VK> rv)
{
    for (uint32_t th = 0; th < 8u; ++th) {
        uint32_t old[4][8];
        if constexpr (MODE == kStoreMerge) {
#pragma unroll
            for (int tl = 0; tl < 4; ++tl)
                ld_global_v8(grid + ((uint64_t)(y0 + 4u * th + tl) << r) + x0, old[tl]);
        }
#pragma unroll
        for (int tl = 0; tl < 4; ++tl) {
            const uint32_t y = y0 + 4u * th + (uint32_t)tl;
            uint8_t *row = grid + ((uint64_t)y << r) + x0;
            rv.set_row(seedmix, x0, y, r);
            uint32_t wv[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                uint32_t word = 0;
                if ((w & th) == 0u) {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if ((b & tl) == 0) word |= rv.bits(4u * w + b) << (8 * b);
                    if constexpr (MODE == kStoreMasked) {
                        // the gasket bytes of this word: all four, 0 and 2, 0 and 1, or 0
                        uint8_t *p = row + 4 * w;
                        if (tl == 0) *reinterpret_cast<uint32_t *>(p) = word;
                        else if (tl == 1) { p[0] = (uint8_t)word; p[2] = (uint8_t)(word >> 16); }
                        else if (tl == 2) *reinterpret_cast<uint16_t *>(p) = (uint16_t)word;
                        else p[0] = (uint8_t)word;
                    }
                }
                if constexpr (MODE == kStoreMerge) {
                    constexpr uint32_t keep_tl[4] = {0x00000000u, 0xFF00FF00u, 0xFFFF0000u,
                                                     0xFFFFFF00u};
                    const uint32_t keep = (w & th) == 0u ? keep_tl[tl] : 0xFFFFFFFFu;
                    word |= old[tl][w] & keep;
                }
                wv[w] = word;
            }
            if constexpr (MODE != kStoreMasked) st_global_v8(row, wv);
        }
    }
}

// One unit of a float32 grid (US x US cells at (x0, y0), US = 8, 16 or 32).
// Rows come in groups of eight, ty = 8 th + tl: sector sx of a row (floats
// 8 sx .. 8 sx + 7) holds gasket cells iff (sx & th) == 0, and then they are
// the floats j with (j & tl) == 0.
template <int VK, int MODE, int US>
__device__ __forceinline__ void sector_unit_f32(float *__restrict__ grid, int r, uint32_t x0,
                                                uint32_t y0, uint64_t seedmix,
                                                RowValue<float, VK> rv)
{
    constexpr uint32_t NS = US / 8;                   // sectors per row, row groups
    for (uint32_t th = 0; th < NS; ++th) {
        for (uint32_t sx = 0; sx < NS; ++sx) {
            if ((sx & th) != 0u) continue;            // uniform: no gasket cell
            const uint32_t xs = x0 + 8u * sx;
            uint32_t old[8][8];
            if constexpr (MODE == kStoreMerge) {
#pragma unroll
                for (int tl = 0; tl < 8; ++tl)
                    ld_global_v8(grid + ((uint64_t)(y0 + 8u * th + tl) << r) + xs, old[tl]);
            }
#pragma unroll
            for (int tl = 0; tl < 8; ++tl) {
                const uint32_t y = y0 + 8u * th + (uint32_t)tl;
                float *row = grid + ((uint64_t)y << r) + xs;
                rv.set_row(seedmix, xs, y, r);
                uint32_t wv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if ((j & tl) == 0) {
                        wv[j] = rv.bits((uint32_t)j);
                        if constexpr (MODE == kStoreMasked)
                            reinterpret_cast<uint32_t *>(row)[j] = wv[j];
                    } else {
                        wv[j] = MODE == kStoreMerge ? old[tl][j] : 0u;
                    }
                }
                if constexpr (MODE != kStoreMasked) st_global_v8(row, wv);
            }
        }
    }
}

template <typename T, int VK, int S, int MAP, int MODE>
__global__ void __launch_bounds__(kSectorThreads)
write_sector_kernel(T *__restrict__ grid, int r, int order, uint64_t vs, uint64_t ntiles)
{
    using SS = SectorShape<T, S>;
    constexpr int SUB = SS::SUB;
    constexpr uint32_t PER = MAP == kMapBBox ? (1u << (2 * SUB)) : (uint32_t)pow3i(SUB);
    const int lane = threadIdx.x & 31;
    const int rb = r - S;
    const uint64_t nunits = ntiles * PER;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * kSectorThreads + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * kSectorThreads) >> 5;
    const uint64_t seedmix = vs * kGoldenGamma;
    RowValue<T, VK> rv;
    rv.seed_hi = (uint32_t)(seedmix >> 32);
    rv.cval = (uint32_t)vs;
    rv.row = 0;
    LambdaLane ll;
    uint32_t W = 1;
    if constexpr (MAP != kMapBBox) {
        ll.init(lane, rb, order);
        W = pi_word(order, rb);
    }

    for (uint64_t task = warp0; task * 32 < nunits; task += nwarps) {
        const uint64_t unit = task * 32 + (uint64_t)lane;
        const uint64_t q = unit / PER;
        const uint32_t u = (uint32_t)(unit - q * PER);
        uint32_t bx = kNoUnit, by = kNoUnit;
        if constexpr (MAP == kMapBBox) {
            if (unit < nunits) {
                const uint32_t tx = (uint32_t)(q & ((1ull << rb) - 1)), tyy = (uint32_t)(q >> rb);
                if ((tx & tyy) == 0u) { bx = tx; by = tyy; }
            }
        } else {
            // the warp decodes the tiles its units span, one per reduction
            const uint64_t q_first = (task * 32) / PER;
            const uint64_t last = task * 32 + 31 < nunits ? task * 32 + 31 : nunits - 1;
            const uint64_t q_last = last / PER;
            for (uint64_t t = q_first; t <= q_last; ++t) {
                const uint32_t b = (uint32_t)t / W, a = (uint32_t)t - b * W;
                const uint2 c = ll.decode(a, b);
                if (t == q && unit < nunits) { bx = c.x; by = c.y; }
            }
        }
        // the unit inside its tile: for lambda the level-SUB gasket's units
        // (0,0), (1,0), (0,1); for the bounding box all of them, (1,1) skipped
        const uint32_t ux = MAP == kMapBBox ? (u & ((1u << SUB) - 1u)) : (u == 1u ? 1u : 0u);
        const uint32_t uy = MAP == kMapBBox ? (u >> SUB) : (u == 2u ? 1u : 0u);
        if (bx == kNoUnit || (ux & uy) != 0u) continue;
        const uint32_t x0 = (bx << S) + ux * SS::US, y0 = (by << S) + uy * SS::US;
        if constexpr (sizeof(T) == 1)
            sector_unit_u8<VK, MODE>(reinterpret_cast<uint8_t *>(grid), r, x0, y0, seedmix, rv);
        else
            sector_unit_f32<VK, MODE, SS::US>(reinterpret_cast<float *>(grid), r, x0, y0,
                                              seedmix, rv);
    }
}

template <typename T, int VK, int S, int MAP>
cudaError_t launch_write_sector(int r, T *grid, uint64_t vs, uint64_t ntiles, cudaStream_t st,
                                const LaunchCfg &cfg)
{
    using SS = SectorShape<T, S>;
    // the intra-tile variants of lambda differ only inside a tile, which
    // this kernel walks by sectors: one instance serves them all
    constexpr int M = MAP == kMapBBox ? kMapBBox : kMapLambda;
    if constexpr (!SS::OK) {
        return cudaErrorNotSupported;
    } else {
        constexpr uint64_t PER = M == kMapBBox ? (1ull << (2 * SS::SUB)) : (uint64_t)pow3i(SS::SUB);
        const uint64_t tasks = (ntiles * PER + 31) / 32;
        const uint64_t units = (tasks + kSectorThreads / 32 - 1) / (kSectorThreads / 32);
        unsigned grid_ctas = 1;
        cudaError_t e;
        if (cfg.store == kStoreMerge) {
            static std::atomic<int> occ{0};
            auto kern = write_sector_kernel<T, VK, S, M, kStoreMerge>;
            e = persistent_grid(kern, kSectorThreads, 0, units, cfg, &grid_ctas, &occ);
            if (e != cudaSuccess) return e;
            kern<<<grid_ctas, kSectorThreads, 0, st>>>(grid, r, cfg.order, vs, ntiles);
        } else if (cfg.store == kStoreMasked) {
            static std::atomic<int> occ{0};
            auto kern = write_sector_kernel<T, VK, S, M, kStoreMasked>;
            e = persistent_grid(kern, kSectorThreads, 0, units, cfg, &grid_ctas, &occ);
            if (e != cudaSuccess) return e;
            kern<<<grid_ctas, kSectorThreads, 0, st>>>(grid, r, cfg.order, vs, ntiles);
        } else {
            static std::atomic<int> occ{0};
            auto kern = write_sector_kernel<T, VK, S, M, kStoreSector>;
            e = persistent_grid(kern, kSectorThreads, 0, units, cfg, &grid_ctas, &occ);
            if (e != cudaSuccess) return e;
            kern<<<grid_ctas, kSectorThreads, 0, st>>>(grid, r, cfg.order, vs, ntiles);
        }
        return cudaGetLastError();
    }
}

}  // namespace sg
