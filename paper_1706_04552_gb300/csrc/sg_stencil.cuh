// sg_stencil.cuh -- helpers shared by the single-gasket stencil kernels
// (sg_stencil.cu) and the batched CA (sg_batch.cu): tile decoding, halo
// enumeration, guarded cell loads and the byte-parallel (SWAR) CA arithmetic.
#pragma once

#include "sg_device.cuh"
#include "sg_internal.h"

namespace sg {

constexpr int kStencilThreads = 256;
constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// Block coordinate of tile q (kNoTile past the end, and for bounding-box
// tiles with no gasket cell).  Warp-collective for the lambda map (all lanes
// pass the same q).  W = pi_word(order, rb).
template <int MAP>
__device__ __forceinline__ uint2 decode_tile(uint64_t q, uint64_t ntiles, int rb, uint32_t W,
                                             const LambdaLane &ll)
{
    uint2 c = make_uint2(kNoTile, kNoTile);
    if (q < ntiles) {
        if constexpr (MAP == kMapBBox) {
            const uint32_t bx = (uint32_t)(q & ((1ull << rb) - 1));
            const uint32_t by = (uint32_t)(q >> rb);
            if ((bx & by) == 0) c = make_uint2(bx, by);
        } else {
            const uint32_t b = (uint32_t)q / W, a = (uint32_t)q - b * W;
            c = ll.decode(a, b);
        }
    }
    return c;
}

// Fills coord[0..tpc) with the block coordinates of tiles g*tpc .. g*tpc+tpc-1.
template <int MAP>
__device__ __forceinline__ void decode_tiles(uint2 *coord, int tpc, uint64_t g,
                                             uint64_t ntiles, int rb, uint32_t W,
                                             const LambdaLane &ll)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < tpc; t += kStencilThreads / 32) {
        const uint2 c = decode_tile<MAP>(g * (uint64_t)tpc + (uint64_t)t, ntiles, rb, W, ll);
        if (lane == 0) coord[t] = c;
    }
}

// Halo slot h of a rho-tile -> tile-relative (row, col), both in [-1, rho].
// Slots: the row above (rho+2 cells), the row below (rho+2), the left column
// (rho) and the right column (rho).
template <int RHO>
__device__ __forceinline__ void halo_slot(int h, int &row, int &col)
{
    if (h < RHO + 2) { row = -1; col = h - 1; }
    else if (h < 2 * RHO + 4) { row = RHO; col = h - (RHO + 2) - 1; }
    else if (h < 3 * RHO + 4) { row = h - (2 * RHO + 4); col = -1; }
    else { row = h - (3 * RHO + 4); col = RHO; }
}

template <typename T>
__device__ __forceinline__ T load_cell(const T *__restrict__ in, int r, int64_t gx, int64_t gy)
{
    const int64_t n = (int64_t)1 << r;
    if (gx < 0 || gy < 0 || gx >= n || gy >= n) return T(0);
    if ((gx & gy) != 0) return T(0);
    return in[(gy << r) + gx];
}

// ---------------------------------------------------------------------------
// Byte-parallel (SWAR) arithmetic on 16 cells held as a uint4.
// Element i of the chunk is byte (i % 4) of word (i / 4).
// ---------------------------------------------------------------------------
// element i <- c[i-1]; element 0 <- l
__device__ __forceinline__ uint4 shift_in_left(uint4 c, uint32_t l)
{
    return make_uint4((c.x << 8) | l, __funnelshift_l(c.x, c.y, 8),
                      __funnelshift_l(c.y, c.z, 8), __funnelshift_l(c.z, c.w, 8));
}
// element i <- c[i+1]; element 15 <- r
__device__ __forceinline__ uint4 shift_in_right(uint4 c, uint32_t r)
{
    return make_uint4(__funnelshift_r(c.x, c.y, 8), __funnelshift_r(c.y, c.z, 8),
                      __funnelshift_r(c.z, c.w, 8), (c.w >> 8) | (r << 24));
}
__device__ __forceinline__ uint4 add4(uint4 a, uint4 b)
{
    return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
// 0x01 in the bytes i of a 16-cell chunk with (i & yl) == 0, yl = y mod 16
__device__ __forceinline__ uint4 member_bytes16(uint32_t yl)
{
    uint32_t w = 0x01010101u;
    if (yl & 1u) w &= 0x00FF00FFu;
    if (yl & 2u) w &= 0x0000FFFFu;
    uint4 m = make_uint4(w, w, w, w);
    if (yl & 4u) { m.y = 0u; m.w = 0u; }
    if (yl & 8u) { m.z = 0u; m.w = 0u; }
    return m;
}
// B3/S23 on bytes: alive next iff (count | self) == 3.  count <= 8, so
// t ^ 3 <= 11 and the +0x7F test below never carries between bytes.
__device__ __forceinline__ uint32_t life_rule(uint32_t count, uint32_t self, uint32_t mask)
{
    const uint32_t t = (count | self) ^ 0x03030303u;
    const uint32_t nonzero = ((t + 0x7F7F7F7Fu) & 0x80808080u) >> 7;
    return (nonzero ^ 0x01010101u) & mask;
}


// ---------------------------------------------------------------------------
// One group of CA tiles (rho >= 16), shared by the single-gasket kernel and
// the batched kernel: every tile carries its own level and buffers.
// ---------------------------------------------------------------------------
struct CaTile {
    uint32_t bx, by;          // block coordinate (kNoTile: no tile in this slot)
    int r;                    // level of the gasket the tile belongs to
    const uint8_t *in;
    uint8_t *out;
};

template <int S> struct CaGroup {
    static constexpr int RHO = 1 << S, CPR = RHO / 16, CHUNKS = RHO * CPR;
    static constexpr int TPC = CHUNKS >= kStencilThreads ? 1 : kStencilThreads / CHUNKS;
    static constexpr int P = RHO + 32;             // row pitch; interior at byte 16
    static constexpr int TILE = (RHO + 2) * P;
    static constexpr int HALO = 4 * RHO + 4;
    // Chunks are loaded and stored by 32-byte sector when a tile row spans
    // whole sectors (rho >= 32): a sector holding any gasket cell moves whole
    // (its off-gasket bytes are 0 in both buffers), so the L2 never has to
    // fill a half-written sector.  With rho = 16 a sector straddles two
    // tiles and chunks move alone.
    static constexpr uint32_t GROUP_MASK = ~(uint32_t)((RHO >= 32 ? 32 : 16) - 1);
};

// Stage every tile of the group (interior chunks of touched sectors, and the
// halo cell by cell at gasket cells only) into shared memory, then compute
// and store the next state chunk by chunk.  Called by all threads; begins
// and ends without a barrier of its own at the edges (the caller syncs
// before reusing `tiles` or `sm`).
template <int S>
__device__ __forceinline__ void ca_group_step(uint8_t *sm, const CaTile *tiles)
{
    using G = CaGroup<S>;
    constexpr int RHO = G::RHO, CPR = G::CPR, CHUNKS = G::CHUNKS, TPC = G::TPC;
    constexpr int P = G::P, TILE = G::TILE, HALO = G::HALO;
    for (int c = threadIdx.x; c < TPC * CHUNKS; c += kStencilThreads) {
        const int t = c / CHUNKS, k = c % CHUNKS, ty = k / CPR, cx = k % CPR;
        const CaTile tl = tiles[t];
        uint4 v = make_uint4(0, 0, 0, 0);
        if (tl.bx != kNoTile) {
            const uint32_t x = (tl.bx << S) + 16u * cx, y = (tl.by << S) + ty;
            if (in_gasket(x & G::GROUP_MASK, y))   // chunk in a touched sector
                v = *reinterpret_cast<const uint4 *>(tl.in + ((uint64_t)y << tl.r) + x);
        }
        *reinterpret_cast<uint4 *>(sm + t * TILE + (ty + 1) * P + 16 + 16 * cx) = v;
    }
    for (int c = threadIdx.x; c < TPC * HALO; c += kStencilThreads) {
        const int t = c / HALO, h = c % HALO;
        int row, col;
        halo_slot<RHO>(h, row, col);
        const CaTile tl = tiles[t];
        uint8_t v = 0;
        if (tl.bx != kNoTile)
            v = load_cell(tl.in, tl.r, (int64_t)(tl.bx << S) + col, (int64_t)(tl.by << S) + row);
        sm[t * TILE + (row + 1) * P + 16 + col] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < TPC * CHUNKS; c += kStencilThreads) {
        const int t = c / CHUNKS, k = c % CHUNKS, ty = k / CPR, cx = k % CPR;
        const CaTile tl = tiles[t];
        if (tl.bx == kNoTile) continue;
        const uint32_t x = (tl.bx << S) + 16u * cx, y = (tl.by << S) + ty;
        if (!in_gasket(x & G::GROUP_MASK, y)) continue;   // sector holds no gasket cell
        const uint8_t *base = sm + t * TILE + 16 + 16 * cx;
        const uint8_t *up = base + ty * P, *mid = up + P, *dn = mid + P;
        const uint4 cu = *reinterpret_cast<const uint4 *>(up);
        const uint4 cm = *reinterpret_cast<const uint4 *>(mid);
        const uint4 cd = *reinterpret_cast<const uint4 *>(dn);
        const uint4 hu = add4(add4(shift_in_left(cu, up[-1]), cu), shift_in_right(cu, up[16]));
        const uint4 hd = add4(add4(shift_in_left(cd, dn[-1]), cd), shift_in_right(cd, dn[16]));
        const uint4 hm = add4(shift_in_left(cm, mid[-1]), shift_in_right(cm, mid[16]));
        const uint4 cnt = add4(add4(hu, hd), hm);
        // x is 16-aligned: the chunk holds gasket cells iff (x & y) == 0,
        // and then bytes i with (i & (y mod 16)) == 0 are the gasket ones
        const uint4 m = in_gasket(x, y) ? member_bytes16(y & 15u) : make_uint4(0u, 0u, 0u, 0u);
        uint4 o;
        o.x = life_rule(cnt.x, cm.x, m.x);
        o.y = life_rule(cnt.y, cm.y, m.y);
        o.z = life_rule(cnt.z, cm.z, m.z);
        o.w = life_rule(cnt.w, cm.w, m.w);
        *reinterpret_cast<uint4 *>(tl.out + ((uint64_t)y << tl.r) + x) = o;
    }
}

}  // namespace sg
