// sg_compact.cuh -- the compact layout: arrays that hold only the 3^r gasket
// cells, with the tables and helpers its kernels share.
//
// Layout.  Element i (i < 3^r) of a compact array with tile side rho = 2^s
// holds cell (x, y) = (bx*rho + tx, by*rho + ty), where
//   (bx, by) is the lambda block of launch index q = i div 3^s (Theorem 1,
//            mirrored to the (x & y) == 0 orientation, in the launch's
//            walking order), and
//   (tx, ty) is the (i mod 3^s)-th cell of the level-s gasket read row by row.
// Every non-empty rho-tile holds that same level-s pattern (Section III), so
// a tile is a run of 3^s consecutive elements: the succinct blocked layout of
// Section II, with the block-space map giving the order of the blocks.
//
// Work unit.  A warp takes kUnit = 3^6 consecutive elements at a time, which
// are G = 3^(6-s) whole tiles, and works on them alone: no barrier between
// the warps of a CTA after the start.  What depends only on the position c
// inside a unit -- the cell's tile g and tile-relative coordinates and, for
// the stencils, where each neighbour's value sits among the staged values --
// is expanded once per CTA from compile-time tables into shared memory.
//
// Neighbours.  A cell's 8 (CA) or 4 (diffusion) neighbours are cells of the
// same tile or one of a fixed list of 8 / 4 cells of neighbouring tiles:
// beside a tile, the gasket pattern leaves the left neighbour only its cell
// (rho-1, 0) in contact, the tile above only (0, rho-1), the tile to the
// right (0, 0) and (0, 1), and so on.  The lists are found below by the same
// enumeration that builds the tables.
#pragma once

#include "sg_device.cuh"
#include "sg_internal.h"

namespace sg {

constexpr int kUnit = 729;            // 3^6 elements per work unit
constexpr int kUnitThreads = 256;
constexpr int kUnitWarps = kUnitThreads / 32;
constexpr uint16_t kNoCell = 0xFFFFu;
constexpr uint16_t kHaloBit = 0x8000u;
constexpr int kCaHalo = 8, kDiffHalo = 4;

template <int S> struct CompactPattern {
    static constexpr int C = pow3i(S), RHO = 1 << S, G = kUnit / C;
    uint16_t pos[C];                 // tx | ty << 8 of the e-th cell, rows top to bottom
    int8_t ca_halo[kCaHalo][4];      // (dbx, dby, lx, ly): tile offset, cell in that tile
    uint16_t ca_halo_rank[kCaHalo];  // that cell's index within its tile
    uint16_t ca_nb[C][8];            // neighbours: index in the tile, kHaloBit | h, kNoCell
    int8_t df_halo[kDiffHalo][4];
    uint16_t df_halo_rank[kDiffHalo];
    uint16_t df_nb[C][4];            // left, right, above, below (same encoding)
    uint8_t df_deg_in[C];            // gasket neighbours inside the tile
    int ca_halo_count, df_halo_count;
};

template <int S> constexpr CompactPattern<S> make_compact_pattern()
{
    using P = CompactPattern<S>;
    constexpr int R = P::RHO;
    P p{};
    uint16_t rank[R][R] = {};
    int e = 0;
    for (int y = 0; y < R; ++y)
        for (int x = 0; x < R; ++x)
            if ((x & y) == 0) {
                rank[y][x] = (uint16_t)e;
                p.pos[e] = (uint16_t)(x | (y << 8));
                ++e;
            }
    // one neighbour (dx, dy) of cell (x, y): its index in the tile, a halo
    // entry (added to the list on first sight), or kNoCell off the gasket
    auto classify = [&](int x, int y, int dx, int dy, int8_t (*halo)[4], uint16_t *hrank,
                        int &count, int cap) -> uint16_t {
        const int nx = x + dx, ny = y + dy;
        if (nx >= 0 && ny >= 0 && nx < R && ny < R)
            return (nx & ny) == 0 ? rank[ny][nx] : kNoCell;
        const int dbx = nx < 0 ? -1 : (nx >= R ? 1 : 0);
        const int dby = ny < 0 ? -1 : (ny >= R ? 1 : 0);
        const int lx = nx - dbx * R, ly = ny - dby * R;
        if ((lx & ly) != 0) return kNoCell;
        for (int h = 0; h < count; ++h)
            if (halo[h][0] == dbx && halo[h][1] == dby && halo[h][2] == lx && halo[h][3] == ly)
                return (uint16_t)(kHaloBit | h);
        if (count >= cap) return kNoCell;        // cannot happen (static_assert below)
        halo[count][0] = (int8_t)dbx;
        halo[count][1] = (int8_t)dby;
        halo[count][2] = (int8_t)lx;
        halo[count][3] = (int8_t)ly;
        hrank[count] = rank[ly][lx];
        return (uint16_t)(kHaloBit | count++);
    };
    for (int i = 0; i < P::C; ++i) {
        const int x = p.pos[i] & 0xFF, y = p.pos[i] >> 8;
        int k = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (dx != 0 || dy != 0)
                    p.ca_nb[i][k++] = classify(x, y, dx, dy, p.ca_halo, p.ca_halo_rank,
                                               p.ca_halo_count, kCaHalo);
        const int d4[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        int deg = 0;
        for (int j = 0; j < 4; ++j) {
            const uint16_t v = classify(x, y, d4[j][0], d4[j][1], p.df_halo, p.df_halo_rank,
                                        p.df_halo_count, kDiffHalo);
            p.df_nb[i][j] = v;
            deg += v < kHaloBit;
        }
        p.df_deg_in[i] = (uint8_t)deg;
    }
    return p;
}

// The tables, one per tile side (global memory; each CTA expands what it
// needs into shared memory once).
__device__ const CompactPattern<0> kCompact0 = make_compact_pattern<0>();
__device__ const CompactPattern<1> kCompact1 = make_compact_pattern<1>();
__device__ const CompactPattern<2> kCompact2 = make_compact_pattern<2>();
__device__ const CompactPattern<3> kCompact3 = make_compact_pattern<3>();
__device__ const CompactPattern<4> kCompact4 = make_compact_pattern<4>();
__device__ const CompactPattern<5> kCompact5 = make_compact_pattern<5>();
__device__ const CompactPattern<6> kCompact6 = make_compact_pattern<6>();

template <int S> __device__ __forceinline__ const CompactPattern<S> &compact_pattern()
{
    if constexpr (S == 0) return kCompact0;
    else if constexpr (S == 1) return kCompact1;
    else if constexpr (S == 2) return kCompact2;
    else if constexpr (S == 3) return kCompact3;
    else if constexpr (S == 4) return kCompact4;
    else if constexpr (S == 5) return kCompact5;
    else return kCompact6;
}

// Every tile side has the same halo sizes (checked at compile time).
template <int S> constexpr bool compact_halos_ok()
{
    constexpr CompactPattern<S> p = make_compact_pattern<S>();
    return p.ca_halo_count == kCaHalo && p.df_halo_count == kDiffHalo;
}
static_assert(compact_halos_ok<0>() && compact_halos_ok<1>() && compact_halos_ok<2>() &&
                  compact_halos_ok<3>() && compact_halos_ok<4>() && compact_halos_ok<5>() &&
                  compact_halos_ok<6>(),
              "a compact tile has 8 CA and 4 diffusion halo cells");

// Rows of a 64-tile as bits.  Row y holds its gasket cells at the columns x
// with x & y == 0: split x = 8*hi + lo, they sit in the bytes hi with
// hi & (y >> 3) == 0 and, inside each, at the bits lo with lo & (y & 7) == 0.
// In compact order the row is one run of 2^(6 - popc(y)) elements, one block
// of 2^(3 - popc(y & 7)) elements per such byte.  dep[y & 7][block] spreads
// a block onto its byte; cmp[y & 7][byte] gathers it back.
struct RowCodec {
    uint8_t dep[8][256];       // block v of a row with y & 7 = yl -> the byte
    uint8_t cmp[8][256];       // byte of such a row -> its block
    uint16_t row_start[64];    // compact index (within the tile) of row y's first cell
};

constexpr int popcount6(int v) { int n = 0; for (int i = 0; i < 6; ++i) n += (v >> i) & 1; return n; }

constexpr RowCodec make_row_codec()
{
    RowCodec t{};
    for (int yl = 0; yl < 8; ++yl)
        for (int v = 0; v < 256; ++v) {
            int d = 0, c = 0, k = 0;
            for (int lo = 0; lo < 8; ++lo)
                if ((lo & yl) == 0) {
                    if ((v >> k) & 1) d |= 1 << lo;    // bit k of the block -> column lo
                    if ((v >> lo) & 1) c |= 1 << k;    // column lo -> bit k of the block
                    ++k;
                }
            t.dep[yl][v] = (uint8_t)d;
            t.cmp[yl][v] = (uint8_t)c;
        }
    int e = 0;
    for (int y = 0; y < 64; ++y) {
        t.row_start[y] = (uint16_t)e;
        e += 1 << (6 - popcount6(y));
    }
    return t;
}

__device__ const RowCodec kRowCodec = make_row_codec();
static_assert(make_row_codec().row_start[63] == kUnit - 1, "the last row holds one cell");

// The 64 bits of `cb` from bit o on (cb holds two zero guard words).
__device__ __forceinline__ uint64_t bits_at(const uint32_t *cb, uint32_t o)
{
    const uint32_t k = o >> 5, sh = o & 31u;
    const uint32_t w0 = cb[k], w1 = cb[k + 1], w2 = cb[k + 2];
    return (uint64_t)__funnelshift_r(w0, w1, sh) | ((uint64_t)__funnelshift_r(w1, w2, sh) << 32);
}

__device__ __forceinline__ uint64_t deposit_row(const RowCodec &tc, uint64_t c, uint32_t y)
{
    const uint32_t yh = y >> 3, yl = y & 7u, nl = 8u >> __popc(yl);
    const uint32_t lmask = (1u << nl) - 1u;
    uint64_t row = 0;
    uint32_t sh = 0;
#pragma unroll
    for (uint32_t hi = 0; hi < 8; ++hi)
        if ((hi & yh) == 0u) {
            row |= (uint64_t)tc.dep[yl][(uint32_t)(c >> sh) & lmask] << (8 * hi);
            sh += nl;
        }
    return row;
}

__device__ __forceinline__ uint64_t gather_row(const RowCodec &tc, uint64_t row, uint32_t y)
{
    const uint32_t yh = y >> 3, yl = y & 7u, nl = 8u >> __popc(yl);
    uint64_t c = 0;
    uint32_t sh = 0;
#pragma unroll
    for (uint32_t hi = 0; hi < 8; ++hi)
        if ((hi & yh) == 0u) {
            c |= (uint64_t)tc.cmp[yl][(uint32_t)(row >> (8 * hi)) & 0xFFu] << sh;
            sh += nl;
        }
    return c;
}

// OR the bits of c (those of one row: its other bits are 0) into `ob` at bit o.
__device__ __forceinline__ void or_bits_at(uint32_t *ob, uint32_t o, uint64_t c)
{
    const uint32_t k = o >> 5, sh = o & 31u;
    const uint32_t lo = (uint32_t)c, hi = (uint32_t)(c >> 32);
    if (lo << sh) atomicOr(&ob[k], lo << sh);
    const uint32_t mid = sh ? (lo >> (32 - sh)) | (hi << sh) : hi;
    if (mid) atomicOr(&ob[k + 1], mid);
    if (sh && (hi >> (32 - sh))) atomicOr(&ob[k + 2], hi >> (32 - sh));
}

// Launch index of block (bx, by) at block-space level rb: the inverse of the
// lambda decode.  Undoing the mirror gives lambda_y = n_b - 1 - by; at level
// mu the coordinate bits (lambda_x, lambda_y) are (0,0), (0,1) or (1,1) for
// beta_mu = 0, 1, 2 (Eq. Delta, Eq. tau), so beta_mu is their sum.  The
// digits are then placed as the walking order deals them: interleaved, digit
// mu-1 of q is beta_mu; row-major, odd levels build omega_y and even levels
// omega_x (Eq. beta) and q = omega_y * 3^floor(rb/2) + omega_x.
__device__ __forceinline__ uint32_t lambda_index(uint32_t bx, uint32_t by, int rb, int order)
{
    const uint32_t ly = ((1u << rb) - 1u) - by;
    uint32_t q = 0, wx = 0, wy = 0;
    for (int mu = rb; mu >= 1; --mu) {
        const uint32_t beta = ((bx >> (mu - 1)) & 1u) + ((ly >> (mu - 1)) & 1u);
        if (order == kOrderInterleaved) q = q * 3u + beta;
        else if (mu & 1) wy = wy * 3u + beta;
        else wx = wx * 3u + beta;
    }
    return order == kOrderInterleaved ? q : wy * (uint32_t)pow3i(rb / 2) + wx;
}

// Cell c of a unit: its tile g within the unit and its tile-relative
// coordinates, packed as g | tx << 10 | ty << 16.
template <int S> __device__ __forceinline__ uint32_t unit_cell(int c)
{
    constexpr int C = CompactPattern<S>::C;
    const int g = c / C;
    const uint32_t pos = compact_pattern<S>().pos[c - g * C];
    return (uint32_t)g | ((pos & 0xFFu) << 10) | ((pos >> 8) << 16);
}

// The block coordinates of tiles first .. first+G-1, decoded by the calling
// warp (every lane takes part); kNoTile past the last tile.  Lane 0 writes.
template <int G>
__device__ __forceinline__ void decode_unit_tiles(uint2 *coord, uint32_t first, uint32_t ntiles,
                                                  uint32_t W, const LambdaLane &ll)
{
    const int lane = threadIdx.x & 31;
    for (int g = 0; g < G; ++g) {
        const uint32_t q = first + (uint32_t)g;
        uint2 c = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        if (q < ntiles) {
            const uint32_t b = q / W, a = q - b * W;
            c = ll.decode(a, b);
        }
        if (lane == 0) coord[g] = c;
    }
}

cudaError_t launch_compact_pack(int r, int s, int order, int elem, const void *grid,
                                void *compact, cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_compact_unpack(int r, int s, int order, int elem, const void *compact,
                                  void *grid, cudaStream_t st, const LaunchCfg &cfg);
// wide: whole aligned 16-byte stores (a destination in host memory)
cudaError_t launch_compact_write(int r, int s, int order, int elem, int vk, void *compact,
                                 uint64_t vs, cudaStream_t st, const LaunchCfg &cfg,
                                 bool wide = false);
cudaError_t launch_compact_ca(int r, int s, int order, const uint8_t *in, uint8_t *out,
                              cudaStream_t st, const LaunchCfg &cfg);
cudaError_t launch_compact_diffuse(int r, int s, int order, const float *in, float *out,
                                   float alpha, cudaStream_t st, const LaunchCfg &cfg);
// k (2 .. SG_FUSE_MAX) CA steps in one launch, rho = 64 (sg_compact_fused.cu).
cudaError_t launch_compact_ca_fused(int r, int order, const uint8_t *in, uint8_t *out, int k,
                                    cudaStream_t st, const LaunchCfg &cfg);

}  // namespace sg
