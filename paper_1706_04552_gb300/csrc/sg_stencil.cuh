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
// Tile groups staged asynchronously, shared by the single-gasket and the
// batched stencil kernels.
//
// A CTA works on groups of TPC tiles (TPC * tile chunks ~ 256 threads).  Each
// tile is staged in shared memory with a one-cell halo as whole 16-byte
// chunks: ROWS = rho + 2 rows of PC = rho/CE + 2 chunks (one halo chunk on
// each side), every chunk an asynchronous copy (cp.async) when it holds an
// in-grid gasket cell and zeros otherwise -- off-gasket cells are 0 in every
// state, so nothing else needs reading.  Two buffers alternate: the copies of
// the next group are in flight while the current group is computed.
// ---------------------------------------------------------------------------
template <typename T> struct StencilTile {
    uint32_t bx, by;          // block coordinate (kNoTile: no tile in this slot)
    int r;                    // level of the gasket the tile belongs to
    const T *in;
    T *out;
};

template <typename T, int S> struct StencilGroup {
    static constexpr int RHO = 1 << S;
    static constexpr int CE = 16 / (int)sizeof(T);           // elements per 16-byte chunk
    static constexpr int CPR = RHO / CE;                      // interior chunks per row
    static constexpr int CHUNKS = RHO * CPR;                  // interior chunks per tile
    static constexpr int TPC = CHUNKS >= kStencilThreads ? 1 : kStencilThreads / CHUNKS;
    static constexpr int PC = CPR + 2;                        // staged chunks per row
    static constexpr int ROWS = RHO + 2;
    static constexpr int P = PC * CE;                         // row pitch (elements); interior at CE
    static constexpr int TILE = ROWS * P;                     // elements per staged tile
    static constexpr int STAGED = ROWS * PC;                  // 16-byte copies per tile
    // Output chunks are stored by 32-byte sector when a tile row spans whole
    // sectors: a sector holding any gasket cell is written whole (its
    // off-gasket cells are 0 in both buffers), so the L2 never has to fill a
    // half-written sector.  Narrower rows store chunk by chunk.
    static constexpr uint32_t GROUP_MASK =
        ~(uint32_t)((RHO * (int)sizeof(T) >= 32 ? 32 / (int)sizeof(T) : CE) - 1);
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the staging copies of a group (every thread; completes at the next
// cp_async_wait + barrier).  A chunk starting at column x (a multiple of CE)
// on row y holds a gasket cell iff (x & y) == 0.
template <typename T, int S>
__device__ __forceinline__ void stage_group_async(T *sm, const StencilTile<T> *tiles)
{
    using G = StencilGroup<T, S>;
    for (int c = threadIdx.x; c < G::TPC * G::STAGED; c += kStencilThreads) {
        const int t = c / G::STAGED, k = c % G::STAGED, row = k / G::PC, cc = k % G::PC;
        const StencilTile<T> tl = tiles[t];
        T *dst = sm + t * G::TILE + row * G::P + cc * G::CE;
        bool fill = false;
        int64_t x = 0, y = 0;
        if (tl.bx != kNoTile) {
            const int64_t n = (int64_t)1 << tl.r;
            x = (int64_t)(tl.bx << S) + (int64_t)(cc - 1) * G::CE;
            y = (int64_t)(tl.by << S) + row - 1;
            fill = x >= 0 && y >= 0 && x < n && y < n && (((uint64_t)x & (uint64_t)y) == 0);
        }
        if (fill) cp_async16(dst, tl.in + (((uint64_t)y << tl.r) + (uint64_t)x));
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// The CA's next state of interior chunk k of staged tile t (buffer sm).
template <int S>
__device__ __forceinline__ void ca_chunk(const uint8_t *sm, const StencilTile<uint8_t> &tl, int t,
                                         int k)
{
    using G = StencilGroup<uint8_t, S>;
    {
        const int ty = k / G::CPR, cx = k % G::CPR;
        const uint32_t x = (tl.bx << S) + 16u * cx, y = (tl.by << S) + ty;
        if (!in_gasket(x & G::GROUP_MASK, y)) return;     // sector holds no gasket cell
        const uint8_t *up = sm + t * G::TILE + ty * G::P + 16 + 16 * cx;
        const uint8_t *mid = up + G::P, *dn = mid + G::P;
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

// The CA's next state for every interior chunk of the group's tiles.
template <int S>
__device__ __forceinline__ void ca_compute_group(const uint8_t *sm,
                                                 const StencilTile<uint8_t> *tiles)
{
    using G = StencilGroup<uint8_t, S>;
    for (int c = threadIdx.x; c < G::TPC * G::CHUNKS; c += kStencilThreads) {
        const int t = c / G::CHUNKS, k = c % G::CHUNKS;
        if (tiles[t].bx == kNoTile) continue;
        ca_chunk<S>(sm, tiles[t], t, k);
    }
}

// Diffusion: u' = u + alpha * (sum of gasket 4-neighbours - deg * u).  Off-
// gasket cells are 0, so the sum runs over the plain 4-neighbourhood.  Every
// diffusion kernel evaluates a cell through diffuse_update, so they agree bit
// for bit.
__device__ __forceinline__ float diffuse_update(float u, float l, float rr, float up, float dn,
                                                float degf, float alpha)
{
    const float sum = (l + rr) + (up + dn);
    return u + alpha * (sum - degf * u);
}

__device__ __forceinline__ float diffuse_cell(uint32_t x, uint32_t y, uint32_t n,
                                              float u, float l, float rr, float up,
                                              float dn, float alpha)
{
    if (!in_gasket(x, y)) return 0.0f;
    const int deg = (x > 0u && in_gasket(x - 1u, y)) + (x + 1u < n && in_gasket(x + 1u, y)) +
                    (y > 0u && in_gasket(x, y - 1u)) + (y + 1u < n && in_gasket(x, y + 1u));
    return diffuse_update(u, l, rr, up, dn, (float)deg, alpha);
}

// Per-chunk degrees.  Whether each cell of a 4-cell chunk is a gasket cell,
// and its gasket degree, depend only on the position: one word per chunk
// holds them (byte i = degree of cell i, or kNotCell), computed with a few
// word operations instead of four membership tests per cell.
constexpr uint32_t kNotCell = 0xFFu;
constexpr uint32_t kDeadChunk = 0xFFFFFFFFu;

// 0x01 in byte i for each set bit i of a 4-bit mask.
__device__ __forceinline__ uint32_t spread4(uint32_t m) { return (m * 0x00204081u) & 0x01010101u; }

// Bits i of 4 with (i & y) == 0: the gasket cells of a 4-cell chunk at a
// column x with (x & y) == 0, x a multiple of 4 (table by y mod 4).
__device__ __forceinline__ uint32_t member_bits4(uint32_t y) { return (0x135Fu >> (4u * (y & 3u))) & 0xFu; }

// Degree word of the chunk at (x, y), x a multiple of 4 (kDeadChunk when it
// holds no gasket cell).  In a chunk with (x & y) == 0, cell i's left and
// right neighbours inside the chunk are members iff bits i-1, i+1 of the
// row's member mask are set; across the chunk's edges, and above and below,
// the neighbour chunk is tested whole.
__device__ __forceinline__ uint32_t chunk_degrees(int x, int y, int n)
{
    if (x < 0 || y < 0 || x >= n || y >= n || (x & y) != 0) return kDeadChunk;
    const uint32_t m = member_bits4((uint32_t)y);
    const uint32_t pl = x > 0 && ((x - 1) & y) == 0;
    const uint32_t pr = x + 4 < n && ((x + 4) & y) == 0;
    const uint32_t mu = (y > 0 && (x & (y - 1)) == 0) ? member_bits4((uint32_t)(y - 1)) : 0u;
    const uint32_t md = (y + 1 < n && (x & (y + 1)) == 0) ? member_bits4((uint32_t)(y + 1)) : 0u;
    const uint32_t ml = ((m << 1) | pl) & 0xFu, mr = (m >> 1) | (pr << 3);
    const uint32_t deg = spread4(ml) + spread4(mr) + spread4(mu) + spread4(md);
    return deg | (spread4(~m & 0xFu) * kNotCell);
}

__device__ __forceinline__ float degree_cell(uint32_t word, int i, float u, float l, float rr,
                                             float up, float dn, float alpha)
{
    const uint32_t d = (word >> (8 * i)) & 0xFFu;
    // (float)d for d <= 4: the low mantissa bits of 2^23 + d, minus 2^23
    const float degf = __uint_as_float(0x4B000000u | d) - 8388608.0f;
    return d == kNotCell ? 0.0f : diffuse_update(u, l, rr, up, dn, degf, alpha);
}

template <int S>
__device__ __forceinline__ void diffuse_chunk(const float *sm, const StencilTile<float> &tl, int t,
                                              int k, float alpha)
{
    using G = StencilGroup<float, S>;
    {
        const int ty = k / G::CPR, cx = k % G::CPR;
        const uint32_t x = (tl.bx << S) + 4u * cx, y = (tl.by << S) + ty;
        if (!in_gasket(x & G::GROUP_MASK, y)) return;     // sector holds no gasket cell
        const uint32_t w = chunk_degrees((int)x, (int)y, 1 << tl.r);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (w != kDeadChunk) {
            const float *mid = sm + t * G::TILE + (ty + 1) * G::P + 4 + 4 * cx;
            const float4 cu = *reinterpret_cast<const float4 *>(mid - G::P);
            const float4 cm = *reinterpret_cast<const float4 *>(mid);
            const float4 cd = *reinterpret_cast<const float4 *>(mid + G::P);
            const float l = mid[-1], rr = mid[4];
            o.x = degree_cell(w, 0, cm.x, l, cm.y, cu.x, cd.x, alpha);
            o.y = degree_cell(w, 1, cm.y, cm.x, cm.z, cu.y, cd.y, alpha);
            o.z = degree_cell(w, 2, cm.z, cm.y, cm.w, cu.z, cd.z, alpha);
            o.w = degree_cell(w, 3, cm.w, cm.z, rr, cu.w, cd.w, alpha);
        }
        *reinterpret_cast<float4 *>(tl.out + ((uint64_t)y << tl.r) + x) = o;
    }
}

template <int S>
__device__ __forceinline__ void diffuse_compute_group(const float *sm,
                                                      const StencilTile<float> *tiles,
                                                      float alpha)
{
    using G = StencilGroup<float, S>;
    for (int c = threadIdx.x; c < G::TPC * G::CHUNKS; c += kStencilThreads) {
        const int t = c / G::CHUNKS, k = c % G::CHUNKS;
        if (tiles[t].bx == kNoTile) continue;
        diffuse_chunk<S>(sm, tiles[t], t, k, alpha);
    }
}

// Double-buffered loop over the CTA's tile groups g = blockIdx.x, + gridDim.x,
// ...: decode(g, slot) fills TPC tile descriptors (warp-collective inside),
// compute(buf, slot) produces the group's output from the staged buffer.
template <typename T, int S, class Decode, class Compute>
__device__ __forceinline__ void stencil_pipeline(T *sm, StencilTile<T> *tiles, uint64_t groups,
                                                 Decode decode, Compute compute)
{
    using G = StencilGroup<T, S>;
    uint64_t g = blockIdx.x;
    if (g >= groups) return;                      // uniform across the CTA
    int cb = 0;
    decode(g, tiles);
    __syncthreads();
    stage_group_async<T, S>(sm, tiles);
    cp_async_commit();
    for (; g < groups; g += gridDim.x) {
        const uint64_t gn = g + gridDim.x;
        const int nb = cb ^ 1;
        // slot nb was last read by the compute of the previous iteration,
        // which every thread finished before that iteration's last barrier
        if (gn < groups) decode(gn, tiles + nb * G::TPC);
        __syncthreads();
        if (gn < groups) stage_group_async<T, S>(sm + nb * G::TPC * G::TILE, tiles + nb * G::TPC);
        cp_async_commit();
        cp_async_wait<1>();                       // this thread's copies of group g landed
        __syncthreads();                          // ... and everyone else's
        compute(sm + cb * G::TPC * G::TILE, tiles + cb * G::TPC);
        __syncthreads();
        cb = nb;
    }
    cp_async_wait<0>();
}

// One warp stages one tile and its one-chunk halo into sm (cp.async, chunks
// without in-grid gasket cells zero-filled) and waits for its own copies:
// the warp-per-tile stencils need no CTA barrier.
constexpr int kWarpTileWarps = kStencilThreads / 32;

template <typename T, int S>
__device__ __forceinline__ void warp_stage(T *sm, const T *__restrict__ in, int r, int x0, int y0,
                                           int lane)
{
    using G = StencilGroup<T, S>;
    const int n = 1 << r;
    for (int i = lane; i < G::STAGED; i += 32) {
        const int row = i / G::PC, cc = i - row * G::PC;
        const int x = x0 + (cc - 1) * G::CE, y = y0 + row - 1;
        T *dst = sm + row * G::P + cc * G::CE;
        const bool fill = x >= 0 && y >= 0 && x < n && y < n && (x & y) == 0;
        if (fill) cp_async16(dst, in + (((uint64_t)y << r) + (uint64_t)x));
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
}

// Persistent grid of a kernel that takes `smem` bytes of dynamic shared
// memory.  With its static arrays that can pass the default 48 KB per CTA,
// so the dynamic limit is raised to the size used, once per device (bit d
// of `attr_devs`).
template <typename K>
inline cudaError_t dyn_smem_grid(K kern, int smem, uint64_t units, const LaunchCfg &cfg,
                                 unsigned *grid, std::atomic<int> *occ,
                                 std::atomic<uint64_t> *attr_devs)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if ((attr_devs->load(std::memory_order_acquire) & bit) == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_devs->fetch_or(bit, std::memory_order_acq_rel);
    }
    return persistent_grid(kern, kStencilThreads, (size_t)smem, units, cfg, grid, occ);
}

}  // namespace sg
