// sg_fused.cu -- k stencil steps in one launch (temporal blocking).
//
// One step of either stencil reads every tile once and writes it once, with a
// few operations per byte, so a sequence of steps is bound by HBM.  Here a
// CTA stages one rho-tile together with a halo of KH >= k rows above and
// below and HX >= k columns on either side (whole 16-byte chunks), runs the
// k steps in shared memory, and writes back only the tile itself:
//
//   * after step s a cell is exact if every cell within distance s of it was
//     staged.  Cells nearer the staged region's edge than that may be wrong
//     (their missing neighbours read as 0), but they are never written back,
//     and the tile lies KH >= k rows and HX >= k columns inside the edge;
//   * at step s only rows [s, ROWS - s) are updated: the rows outside that
//     window cannot be exact any more and nothing that is written reads them;
//   * chunks outside the grid or holding no gasket cell are staged as zeros
//     and produce zeros at every step, exactly as the single-step kernels
//     treat them (off-gasket cells are 0 in every state).
//
// The CA runs bit-sliced (one warp per tile, 32 cells per word operation).
// Diffusion at tile sides 32 and 64 runs one warp per 32 x 32 unit with the
// 9-cell gasket blocks of 4 x 4 cells held in registers (diffuse_warp_fused_
// kernel, below); at side 16 one CTA per tile on float4 chunks
// (diffuse_fused_kernel).  Either way each cell's result is the single step's,
// so k fused steps equal k single steps.  HBM moves about the tile bytes once
// in and once out per launch instead of per step.
//
// The tile coordinate comes from the lambda(omega) decode of Theorem 1 (one
// warp, redux.sync) or from the bounding-box identity map, as elsewhere.
#include "sg_bits.cuh"
#include "sg_stencil.cuh"
#include "sg_tma.cuh"

namespace sg {

template <typename T, int S, int KH> struct FusedShape {
    static constexpr int RHO = 1 << S;
    static constexpr int CE = 16 / (int)sizeof(T);            // elements per chunk
    static constexpr int HX = ((KH + CE - 1) / CE) * CE;       // halo columns per side
    static constexpr int HC = HX / CE;                         // halo chunks per side
    static constexpr int CPR = RHO / CE;                       // tile chunks per row
    static constexpr int PC = CPR + 2 * HC;                    // staged chunks per row
    static constexpr int ROWS = RHO + 2 * KH;
    static constexpr int P = PC * CE;                          // row pitch (elements)
    static constexpr int BUF = ROWS * P * (int)sizeof(T);      // bytes per state buffer
    static constexpr uint32_t GROUP_MASK = StencilGroup<T, S>::GROUP_MASK;
};

// Stage the tile at (x0, y0) with its halo into buf (every thread; complete
// after cp_async_wait<0> + barrier).
template <typename T, int S, int KH>
__device__ __forceinline__ void fused_stage(T *buf, const T *__restrict__ in, int r,
                                            int x0, int y0)
{
    using F = FusedShape<T, S, KH>;
    const int n = 1 << r;
    for (int i = threadIdx.x; i < F::ROWS * F::PC; i += kStencilThreads) {
        const int row = i / F::PC, cc = i - row * F::PC;
        const int x = x0 - F::HX + cc * F::CE, y = y0 - KH + row;
        T *dst = buf + row * F::P + cc * F::CE;
        const bool fill = x >= 0 && y >= 0 && x < n && y < n && (x & y) == 0;
        if (fill) cp_async16(dst, in + (((uint64_t)y << r) + (uint64_t)x));
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_commit();
}

// Copy the tile (rows [KH, KH + RHO), chunks [HC, HC + CPR)) to HBM, whole
// 32-byte sectors where a tile row spans them (see StencilGroup).
template <typename T, int S, int KH>
__device__ __forceinline__ void fused_store(const T *buf, T *__restrict__ out, int r,
                                            int x0, int y0)
{
    using F = FusedShape<T, S, KH>;
    for (int i = threadIdx.x; i < F::RHO * F::CPR; i += kStencilThreads) {
        const int ty = i / F::CPR, cx = i - ty * F::CPR;
        const uint32_t x = (uint32_t)x0 + (uint32_t)(cx * F::CE), y = (uint32_t)(y0 + ty);
        if (!in_gasket(x & F::GROUP_MASK, y)) continue;
        const T *src = buf + (KH + ty) * F::P + (F::HC + cx) * F::CE;
        *reinterpret_cast<uint4 *>(out + ((uint64_t)y << r) + x) =
            *reinterpret_cast<const uint4 *>(src);
    }
}

template <int S, int KH, int MAP>
__global__ void __launch_bounds__(kStencilThreads, 6)
ca_bits_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r, int order,
               uint64_t ntiles, int k)
{
    using B = BitShape<S, KH>;
    __shared__ uint32_t sm[B::WARPS][3][B::BUFW];      // two states and the mask, per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *st0 = sm[warp][0] + 1, *st1 = sm[warp][1] + 1, *mk = sm[warp][2] + 1;

    const int rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t stride = (uint64_t)gridDim.x * B::WARPS;

    for (uint64_t q = (uint64_t)blockIdx.x * B::WARPS + warp; q < ntiles; q += stride) {
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        if (c.x == kNoTile) continue;                                // uniform in the warp
        bits_tile_steps<S, KH>(st0, st1, mk, in, out, r, (int)(c.x << S), (int)(c.y << S), k,
                               lane);
    }
}

// ---------------------------------------------------------------------------
// Diffusion.  One CTA per tile.  Whether each of a chunk's four cells is a
// gasket cell, and its gasket degree, depend only on the position: they are
// worked out once per tile into one word per chunk (chunk_degrees).  The
// chunks that hold gasket cells -- a third of a 64-tile's chunks -- are
// compacted into a list while the tile is staged, and every step runs over
// that list only, so the threads of a warp all do useful work; the other
// chunks are 0 in both state buffers throughout.  The list is built in
// row-major chunk order (warp ballots and one scan), so neighbouring threads
// read neighbouring chunks.
// ---------------------------------------------------------------------------
// (at most 64 registers a thread: the unrolled chunk sweeps would take
// more; shared memory allows 3-4 resident CTAs of 64-tiles anyway)
template <int S, int KH, int MAP>
__global__ void __launch_bounds__(kStencilThreads, 4)
diffuse_fused_kernel(const float *__restrict__ in, float *__restrict__ out, int r, int order,
                     uint64_t ntiles, int k, float alpha)
{
    using F = FusedShape<float, S, KH>;
    constexpr int CH = F::ROWS * F::PC;
    constexpr int PER = (CH + kStencilThreads - 1) / kStencilThreads;
    extern __shared__ __align__(16) unsigned char fused_smem[];
    float *b0 = reinterpret_cast<float *>(fused_smem);
    float *b1 = reinterpret_cast<float *>(fused_smem + F::BUF);
    constexpr int WARPS = kStencilThreads / 32;
    __shared__ uint2 coord;
    __shared__ uint32_t live_n;
    __shared__ uint32_t warp_base[PER][WARPS];   // list position of each warp's first live chunk
    __shared__ uint16_t live_chunk[CH];          // staged chunk index (row * PC + column)
    __shared__ uint32_t live_deg[CH];            // its degree word

    const int n = 1 << r, rb = r - S;
    const int lane = threadIdx.x & 31;
    const uint32_t lanes_below = (1u << lane) - 1u;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);

    for (uint64_t q = blockIdx.x; q < ntiles; q += gridDim.x) {
        if (threadIdx.x < 32) {
            const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);
            if (threadIdx.x == 0) coord = c;
        }
        __syncthreads();                 // coord visible; last tile's buffers free
        const uint2 c = coord;
        if (c.x == kNoTile) {            // uniform: an empty bounding-box tile
            __syncthreads();
            continue;
        }
        const int x0 = (int)(c.x << S), y0 = (int)(c.y << S);
        const int warp = threadIdx.x >> 5;
        // stage the live chunks and zero the rest in both buffers; count each
        // warp's live chunks per sweep j (chunk ch = threadIdx.x + 256 j, so
        // (j, warp, lane) is row-major chunk order)
        uint32_t deg[PER], ballot[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int ch = threadIdx.x + j * kStencilThreads;
            deg[j] = kDeadChunk;
            if (ch < CH) {
                const int row = ch / F::PC, cc = ch - row * F::PC;
                const int x = x0 - F::HX + 4 * cc, y = y0 - KH + row;
                deg[j] = chunk_degrees(x, y, n);
                float *d0 = b0 + row * F::P + 4 * cc;
                if (deg[j] != kDeadChunk) {
                    cp_async16(d0, in + (((uint64_t)y << r) + (uint64_t)x));
                } else {
                    *reinterpret_cast<float4 *>(d0) = make_float4(0.f, 0.f, 0.f, 0.f);
                    *reinterpret_cast<float4 *>(b1 + (d0 - b0)) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            ballot[j] = __ballot_sync(0xFFFFFFFFu, deg[j] != kDeadChunk);
            if (lane == 0) warp_base[j][warp] = (uint32_t)__popc(ballot[j]);
        }
        cp_async_commit();
        __syncthreads();
        if (threadIdx.x == 0) {          // exclusive scan over (j, warp): row-major order
            uint32_t acc = 0;
            for (int j = 0; j < PER; ++j)
                for (int w8 = 0; w8 < WARPS; ++w8) {
                    const uint32_t cnt = warp_base[j][w8];
                    warp_base[j][w8] = acc;
                    acc += cnt;
                }
            live_n = acc;
        }
        __syncthreads();
        // the list of live chunks, in row-major order
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            if (deg[j] == kDeadChunk) continue;
            const uint32_t pos = warp_base[j][warp] + (uint32_t)__popc(ballot[j] & lanes_below);
            live_chunk[pos] = (uint16_t)(threadIdx.x + j * kStencilThreads);
            live_deg[pos] = deg[j];
        }
        cp_async_wait<0>();
        __syncthreads();
        const uint32_t nlive = live_n;
        for (int s = 1; s <= k; ++s) {
            const float *src = (s & 1) ? b0 : b1;
            float *dst = (s & 1) ? b1 : b0;
            for (uint32_t i = threadIdx.x; i < nlive; i += kStencilThreads) {
                const int ch = (int)live_chunk[i];
                const int row = ch / F::PC, cc = ch - row * F::PC;
                if (row < s || row >= F::ROWS - s) continue;
                const float *mid = src + row * F::P + 4 * cc;
                const float4 cu = *reinterpret_cast<const float4 *>(mid - F::P);
                const float4 cm = *reinterpret_cast<const float4 *>(mid);
                const float4 cd = *reinterpret_cast<const float4 *>(mid + F::P);
                // neighbours left and right of the chunk (not staged at the
                // region's edge: read inside the chunk, then use 0)
                const bool hl = cc > 0, hr = cc < F::PC - 1;
                const float lv = mid[hl ? -1 : 0], rv = mid[hr ? 4 : 3];
                const float l = hl ? lv : 0.f, rr = hr ? rv : 0.f;
                const uint32_t w = live_deg[i];
                float4 o;
                o.x = degree_cell(w, 0, cm.x, l, cm.y, cu.x, cd.x, alpha);
                o.y = degree_cell(w, 1, cm.y, cm.x, cm.z, cu.y, cd.y, alpha);
                o.z = degree_cell(w, 2, cm.z, cm.y, cm.w, cu.z, cd.z, alpha);
                o.w = degree_cell(w, 3, cm.w, cm.z, rr, cu.w, cd.w, alpha);
                *reinterpret_cast<float4 *>(dst + row * F::P + 4 * cc) = o;
            }
            __syncthreads();
        }
        fused_store<float, S, KH>((k & 1) ? b1 : b0, out, r, x0, y0);
        // the next iteration's first barrier orders these reads (and those
        // of live_n, warp_base and the lists) before the next tile rewrites them
    }
}

// ---------------------------------------------------------------------------
// Diffusion for tile sides 32 and 64: one warp per 32 x 32 unit (a 64-tile
// is its three 32-tiles that hold gasket cells), with no barrier wider than
// the warp.  The warp takes the unit with a halo of KH rows above and below
// and HX >= KH columns on either side (KH a multiple of 4) and runs the k
// steps on it.
//
// The region is cut into blocks of 4 x 4 cells (a 16-byte chunk on each of
// the 4 rows of a row group; row groups start at multiples of 4).  The cell
// (x, y) is a gasket cell iff (x & y) == 0; for a block at (X, Y), both
// multiples of 4, that is (X & Y) == 0 and (i & j) == 0 for the cell (i, j)
// inside it.  So a block either holds no gasket cell or exactly the 9 cells of
// the level-2 gasket,
//
//     j = 0:  (0,0) (1,0) (2,0) (3,0)
//     j = 1:  (0,1)       (2,1)
//     j = 2:  (0,2) (1,2)
//     j = 3:  (0,3)
//
// and of their 4-neighbours all but four lie in the block itself: the left
// and upper neighbours of (0,0) are (3,0) of the block to the left and (0,3)
// of the block above, the right neighbour of (3,0) is (0,0) of the block to
// the right, and the lower neighbour of (0,3) is (0,0) of the block below;
// every other neighbour outside the block is off the gasket.  Degrees follow:
// (0,0) has 2 plus one for each of its outside neighbours that is a gasket
// cell (its block is live), (3,0) and (0,3) have 1 plus one, and the other
// six cells have 2, 3, 2, 1, 3, 1.
//
//   * the live blocks of the region (one mask per row group: region_row_mask)
//     are listed group by group; block b belongs to lane b mod 32, which keeps
//     its 9 cell states, the 3 degrees that vary and one word with the four
//     neighbouring blocks in registers for all k steps;
//   * a step reads the four outside neighbours from three shared-memory
//     arrays in which every block publishes (0,0), (3,0) and (0,3), updates
//     the 9 cells in registers, and publishes them again after a warp barrier.
//     A missing neighbour reads the entry of every array that stays 0;
//   * only blocks whose rows meet [s, ROWS - s) are updated at step s: the
//     cells that must still be exact after step s lie in those rows, and a
//     cell is exact once every cell within distance s of it was loaded.  A
//     block on the region's edge can have the wrong degree for a neighbour
//     outside the region; no exact cell depends on it;
//   * every cell is evaluated with diffuse_update and the same operands as in
//     the single-step kernels (a neighbour off the gasket is the 0 the state
//     holds there), so k fused steps equal k single steps bit for bit.
// ---------------------------------------------------------------------------
template <int KH> struct WarpFusedShape {
    static constexpr int U = 32;                              // unit side
    static constexpr int HX = (KH + 3) / 4 * 4;               // halo columns per side
    static constexpr int HC = HX / 4;                         // halo blocks per side
    static constexpr int PC = U / 4 + 2 * HC;                 // blocks per row group
    static constexpr int ROWS = U + 2 * KH;
    static constexpr int GROUPS = ROWS / 4;                   // row groups
    // Most live blocks in any unit's region: the region meets the 3 x 3
    // neighbourhood of 32-tiles around the unit, each either empty or holding
    // the level-5 pattern, and over the 13 neighbourhoods a gasket has (the
    // same set at every block level from 3 on) the count peaks at 44, 54 and
    // 72 for KH = 4, 8, 16.  A unit with more would set kDevOverflow.
    static constexpr int MAXB = KH == 4 ? 44 : KH == 8 ? 54 : 72;
    static constexpr int SLOTS = (MAXB + 31) / 32;            // blocks per lane
    static constexpr int NB = 32 * SLOTS;
    static constexpr int ZERO = NB;                           // the entry that stays 0
    // per warp: published cells (0,0), (3,0), (0,3) of each block, the list
    // of live blocks (group << 4 | column), group masks and group starts
    static constexpr int WARP_BYTES =
        (3 * (NB + 1) * 4 + NB + GROUPS * 2 + (GROUPS + 1) + 15) / 16 * 16;
    static_assert(KH % 4 == 0 && U % 4 == 0, "row groups of 4");
    static_assert(NB < 128 && GROUPS <= 16 && PC <= 16, "block fields are 7 and 4 bits");
};

constexpr int kWarpFusedWarps = 4;                            // independent warps per CTA

// Live chunks of region row y (bit cc: the chunk at column x0 - 4*HC + 4*cc)
// for a unit at column x0 (a multiple of 32).  A chunk at column x, a
// multiple of 4, in the 32-tile at column X = x & ~31 holds a gasket cell on
// row y iff (X & y) == 0 and its index c = (x & 31) / 4 in the tile has
// (c & (y >> 2) & 7) == 0; s8 holds the c passing the second test.  Rows of
// one group of 4 have the same mask.
template <int HC>
__device__ __forceinline__ uint32_t region_row_mask(int x0, int y, int n)
{
    if (y < 0 || y >= n) return 0u;
    const uint32_t m3 = ((uint32_t)y >> 2) & 7u;
    uint32_t s8 = 0xFFu;
    if (m3 & 1u) s8 &= 0x55u;
    if (m3 & 2u) s8 &= 0x33u;
    if (m3 & 4u) s8 &= 0x0Fu;
    const uint32_t lt = (x0 >= 32 && ((x0 - 32) & y) == 0) ? (s8 >> (8 - HC)) : 0u;
    const uint32_t tt = ((x0 & y) == 0) ? s8 : 0u;
    const uint32_t rt = (x0 + 32 < n && ((x0 + 32) & y) == 0) ? (s8 & ((1u << HC) - 1u)) : 0u;
    return lt | (tt << HC) | (rt << (HC + 8));
}

// One live block in a lane's registers.
struct GasketBlock {
    float u00, u10, u20, u30, u01, u21, u02, u12, u03;   // the 9 cell states
    float d00, d30, d03;                                  // the degrees that vary
    uint32_t nb;   // blocks above (bits 0..6), below (7..13), left (14..20),
                   // right (21..27); row group (28..31)
};

template <int S, int KH, int MAP>
__global__ void __launch_bounds__(32 * kWarpFusedWarps)
diffuse_warp_fused_kernel(const float *__restrict__ in, float *__restrict__ out, int r, int order,
                          uint64_t ntiles, int k, float alpha, int *status)
{
    using F = WarpFusedShape<KH>;
    constexpr int SUB = S - 5;                                  // unit levels inside a tile
    constexpr uint32_t PER = MAP == kMapBBox ? (1u << (2 * SUB)) : (uint32_t)pow3i(SUB);
    constexpr uint32_t Z = (uint32_t)F::ZERO;
    extern __shared__ __align__(16) unsigned char wf_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *mine = wf_smem + (size_t)warp * F::WARP_BYTES;
    float *p00 = reinterpret_cast<float *>(mine);                // published (0,0)
    float *p30 = p00 + (F::NB + 1);                              // published (3,0)
    float *p03 = p30 + (F::NB + 1);                              // published (0,3)
    uint8_t *list = reinterpret_cast<uint8_t *>(p03 + (F::NB + 1));
    uint16_t *gmask = reinterpret_cast<uint16_t *>(list + F::NB);
    uint8_t *gbase = reinterpret_cast<uint8_t *>(gmask + F::GROUPS);

    const int n = 1 << r, rb = r - S;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint64_t nunits = ntiles * PER;
    if (lane == 0) { p00[Z] = 0.f; p30[Z] = 0.f; p03[Z] = 0.f; }

    const uint64_t stride = (uint64_t)gridDim.x * kWarpFusedWarps;
    for (uint64_t unit = (uint64_t)blockIdx.x * kWarpFusedWarps + warp; unit < nunits;
         unit += stride) {
        const uint64_t q = unit / PER;
        const uint32_t u = (uint32_t)(unit - q * PER);
        const uint2 c = decode_tile<MAP>(q, ntiles, rb, W, ll);     // warp-collective
        // the unit's 32-tile inside its rho-tile: for lambda the level-SUB
        // gasket's tiles (0,0), (1,0), (0,1); for the bounding box all of them,
        // the empty one skipped
        const uint32_t ux = MAP == kMapBBox ? (u & ((1u << SUB) - 1u)) : (u == 1u ? 1u : 0u);
        const uint32_t uy = MAP == kMapBBox ? (u >> SUB) : (u == 2u ? 1u : 0u);
        if (c.x == kNoTile || (ux & uy) != 0u) continue;            // uniform in the warp
        const int x0 = (int)((c.x << S) + (ux << 5)), y0 = (int)((c.y << S) + (uy << 5));
        const int gx = x0 - F::HX, gy = y0 - KH;                    // the region's corner

        // 1. live blocks group by group (lane g: group g), their positions by
        //    a warp scan, the list in shared memory
        const uint32_t m = lane < F::GROUPS ? region_row_mask<F::HC>(x0, gy + 4 * lane, n) : 0u;
        const uint32_t cnt = (uint32_t)__popc(m);
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, d);
            if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (total > (uint32_t)F::MAXB) {                            // uniform; cannot happen
            if (lane == 0) record_device_error(status, kDevOverflow);
            continue;
        }
        if (lane < F::GROUPS) {
            gmask[lane] = (uint16_t)m;
            gbase[lane] = (uint8_t)(incl - cnt);
            uint32_t mm = m, pos = incl - cnt;
            while (mm) {
                const int cc = __ffs(mm) - 1;
                mm &= mm - 1u;
                list[pos++] = (uint8_t)((lane << 4) | cc);
            }
        }
        if (lane == 0) gbase[F::GROUPS] = (uint8_t)total;
        __syncwarp();

        // 2. this lane's blocks: cells from HBM, neighbours, degrees
        GasketBlock blk[F::SLOTS];
#pragma unroll
        for (int j = 0; j < F::SLOTS; ++j) {
            const uint32_t b = 32u * j + lane;
            GasketBlock &B = blk[j];
            B = GasketBlock{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
            if (b < total) {
                const uint32_t ent = list[b];
                const int g = (int)(ent >> 4), cc = (int)(ent & 15u);
                const float *src = in + (((uint64_t)(gy + 4 * g) << r) + (uint64_t)(gx + 4 * cc));
                const float4 r0 = *reinterpret_cast<const float4 *>(src);
                const float4 r1 = *reinterpret_cast<const float4 *>(src + n);
                const float4 r2 = *reinterpret_cast<const float4 *>(src + 2 * (uint64_t)n);
                const float r3 = src[3 * (uint64_t)n];
                B.u00 = r0.x; B.u10 = r0.y; B.u20 = r0.z; B.u30 = r0.w;
                B.u01 = r1.x; B.u21 = r1.z; B.u02 = r2.x; B.u12 = r2.y; B.u03 = r3;
                const uint32_t gm = gmask[g];
                uint32_t up = Z, dn = Z;
                if (g > 0) {
                    const uint32_t mu = gmask[g - 1];
                    if ((mu >> cc) & 1u) up = gbase[g - 1] + (uint32_t)__popc(mu & ((1u << cc) - 1u));
                }
                if (g + 1 < F::GROUPS) {
                    const uint32_t md = gmask[g + 1];
                    if ((md >> cc) & 1u) dn = gbase[g + 1] + (uint32_t)__popc(md & ((1u << cc) - 1u));
                }
                const uint32_t lf = (cc > 0 && ((gm >> (cc - 1)) & 1u)) ? b - 1u : Z;
                const uint32_t rt = ((gm >> (cc + 1)) & 1u) ? b + 1u : Z;
                B.nb = up | (dn << 7) | (lf << 14) | (rt << 21) | ((uint32_t)g << 28);
                B.d00 = 2.0f + (float)(lf != Z) + (float)(up != Z);
                B.d30 = 1.0f + (float)(rt != Z);
                B.d03 = 1.0f + (float)(dn != Z);
                p00[b] = B.u00; p30[b] = B.u30; p03[b] = B.u03;
            }
        }
        __syncwarp();

        // 3. the k steps
        for (int s = 1; s <= k; ++s) {
#pragma unroll
            for (int j = 0; j < F::SLOTS; ++j) {
                GasketBlock &B = blk[j];
                const int g = (int)(B.nb >> 28);
                if (32u * j + lane >= total || 4 * g + 3 < s || 4 * g >= F::ROWS - s) continue;
                const float U = p03[B.nb & 127u], D = p00[(B.nb >> 7) & 127u];
                const float L = p30[(B.nb >> 14) & 127u], R = p00[(B.nb >> 21) & 127u];
                const float u00 = B.u00, u10 = B.u10, u20 = B.u20, u30 = B.u30;
                const float u01 = B.u01, u21 = B.u21, u02 = B.u02, u12 = B.u12, u03 = B.u03;
                // diffuse_update(u, left, right, up, down, degree, alpha)
                B.u00 = diffuse_update(u00, L, u10, U, u01, B.d00, alpha);
                B.u10 = diffuse_update(u10, u00, u20, 0.f, 0.f, 2.0f, alpha);
                B.u20 = diffuse_update(u20, u10, u30, 0.f, u21, 3.0f, alpha);
                B.u30 = diffuse_update(u30, u20, R, 0.f, 0.f, B.d30, alpha);
                B.u01 = diffuse_update(u01, 0.f, 0.f, u00, u02, 2.0f, alpha);
                B.u21 = diffuse_update(u21, 0.f, 0.f, u20, 0.f, 1.0f, alpha);
                B.u02 = diffuse_update(u02, 0.f, u12, u01, u03, 3.0f, alpha);
                B.u12 = diffuse_update(u12, u02, 0.f, 0.f, 0.f, 1.0f, alpha);
                B.u03 = diffuse_update(u03, 0.f, 0.f, u02, D, B.d03, alpha);
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < F::SLOTS; ++j) {
                const GasketBlock &B = blk[j];
                const uint32_t b = 32u * j + lane;
                const int g = (int)(B.nb >> 28);
                if (b >= total || 4 * g + 3 < s || 4 * g >= F::ROWS - s) continue;
                p00[b] = B.u00; p30[b] = B.u30; p03[b] = B.u03;
            }
            __syncwarp();
        }

        // 4. the unit's blocks out: the four rows of each block (0 at its cells
        //    off the gasket), and zeros for the other half of the 32-byte
        //    sector when that half holds no gasket cell
#pragma unroll
        for (int j = 0; j < F::SLOTS; ++j) {
            const GasketBlock &B = blk[j];
            if (32u * j + lane >= total) continue;
            const int g = (int)(B.nb >> 28);
            const int cc = (int)(list[32u * j + lane] & 15u);
            if (g < KH / 4 || g >= KH / 4 + 8 || cc < F::HC || cc >= F::HC + 8) continue;
            const int x = gx + 4 * cc;
            float *dst = out + (((uint64_t)(gy + 4 * g) << r) + (uint64_t)x);
            const uint64_t nn = (uint64_t)n;
            *reinterpret_cast<float4 *>(dst) = make_float4(B.u00, B.u10, B.u20, B.u30);
            *reinterpret_cast<float4 *>(dst + nn) = make_float4(B.u01, 0.f, B.u21, 0.f);
            *reinterpret_cast<float4 *>(dst + 2 * nn) = make_float4(B.u02, B.u12, 0.f, 0.f);
            *reinterpret_cast<float4 *>(dst + 3 * nn) = make_float4(B.u03, 0.f, 0.f, 0.f);
            const int pc = cc + (((x ^ 4) - x) >> 2);                   // the sector's other half
            if (!((gmask[g] >> pc) & 1u)) {
                float *o = out + (((uint64_t)(gy + 4 * g) << r) + (uint64_t)(x ^ 4));
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(o) = z;
                *reinterpret_cast<float4 *>(o + nn) = z;
                *reinterpret_cast<float4 *>(o + 2 * nn) = z;
                *reinterpret_cast<float4 *>(o + 3 * nn) = z;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int S, int KH, int MAP>
cudaError_t launch_ca_fused_t(int r, const uint8_t *in, uint8_t *out, int k, cudaStream_t st,
                              const LaunchCfg &cfg)
{
    using B = BitShape<S, KH>;
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    static std::atomic<int> occ{0};
    auto kern = ca_bits_kernel<S, KH, MAP>;
    unsigned grid = 1;
    cudaError_t e = persistent_grid(kern, kStencilThreads, 0, (ntiles + B::WARPS - 1) / B::WARPS,
                                    cfg, &grid, &occ);
    if (e != cudaSuccess) return e;
    kern<<<grid, kStencilThreads, 0, st>>>(in, out, r, cfg.order, ntiles, k);
    return cudaGetLastError();
}

template <int S, int KH, int MAP>
cudaError_t launch_diffuse_warp_fused_t(int r, const float *in, float *out, float alpha, int k,
                                        cudaStream_t st, const LaunchCfg &cfg)
{
    using F = WarpFusedShape<KH>;
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    constexpr uint64_t PER = MAP == kMapBBox ? (1ull << (2 * (S - 5))) : (uint64_t)pow3i(S - 5);
    constexpr int SMEM = kWarpFusedWarps * F::WARP_BYTES;
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    auto kern = diffuse_warp_fused_kernel<S, KH, MAP>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if ((attr.load(std::memory_order_acquire) & bit) == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr.fetch_or(bit, std::memory_order_acq_rel);
    }
    int *status = nullptr;
    e = device_status_ptr(&status);
    if (e != cudaSuccess) return e;
    unsigned grid = 1;
    e = persistent_grid(kern, 32 * kWarpFusedWarps, SMEM,
                        (ntiles * PER + kWarpFusedWarps - 1) / kWarpFusedWarps, cfg, &grid, &occ);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * kWarpFusedWarps, SMEM, st>>>(in, out, r, cfg.order, ntiles, k, alpha, status);
    return cudaGetLastError();
}

template <int S, int KH, int MAP>
cudaError_t launch_diffuse_fused_t(int r, const float *in, float *out, float alpha, int k,
                                   cudaStream_t st, const LaunchCfg &cfg)
{
    if constexpr (S >= 5)
        return launch_diffuse_warp_fused_t<S, KH, MAP>(r, in, out, alpha, k, st, cfg);
    using F = FusedShape<float, S, KH>;
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    auto kern = diffuse_fused_kernel<S, KH, MAP>;
    unsigned grid = 1;
    cudaError_t e = dyn_smem_grid(kern, 2 * F::BUF, ntiles, cfg, &grid, &occ, &attr);
    if (e != cudaSuccess) return e;
    kern<<<grid, kStencilThreads, 2 * F::BUF, st>>>(in, out, r, cfg.order, ntiles, k, alpha);
    return cudaGetLastError();
}

// Halo depth instance for k fused steps: the smallest of 4, 8, 16 >= k.
#define SG_FUSED_SWITCH(s, k, CALL)                                          \
    do {                                                                     \
        const int kh_ = (k) <= 4 ? 4 : (k) <= 8 ? 8 : 16;                    \
        switch ((s) * 100 + kh_) {                                           \
        case 404: return CALL(4, 4);                                         \
        case 408: return CALL(4, 8);                                         \
        case 416: return CALL(4, 16);                                        \
        case 504: return CALL(5, 4);                                         \
        case 508: return CALL(5, 8);                                         \
        case 516: return CALL(5, 16);                                        \
        case 604: return CALL(6, 4);                                         \
        case 608: return CALL(6, 8);                                         \
        case 616: return CALL(6, 16);                                        \
        default: return cudaErrorInvalidValue;                               \
        }                                                                    \
    } while (0)

cudaError_t launch_ca_fused(int r, int s, int map, const uint8_t *in, uint8_t *out, int k,
                            cudaStream_t st, const LaunchCfg &cfg)
{
    if (k < 1 || k > 16) return cudaErrorInvalidValue;
    if (map == kMapBBox) {
#define CALL(S, KH) launch_ca_fused_t<S, KH, kMapBBox>(r, in, out, k, st, cfg)
        SG_FUSED_SWITCH(s, k, CALL);
#undef CALL
    }
#define CALL(S, KH) launch_ca_fused_t<S, KH, kMapLambda>(r, in, out, k, st, cfg)
    SG_FUSED_SWITCH(s, k, CALL);
#undef CALL
}

cudaError_t launch_diffuse_fused(int r, int s, int map, const float *in, float *out,
                                 float alpha, int k, cudaStream_t st, const LaunchCfg &cfg)
{
    if (k < 1 || k > 16) return cudaErrorInvalidValue;
    if (map == kMapBBox) {
#define CALL(S, KH) launch_diffuse_fused_t<S, KH, kMapBBox>(r, in, out, alpha, k, st, cfg)
        SG_FUSED_SWITCH(s, k, CALL);
#undef CALL
    }
#define CALL(S, KH) launch_diffuse_fused_t<S, KH, kMapLambda>(r, in, out, alpha, k, st, cfg)
    SG_FUSED_SWITCH(s, k, CALL);
#undef CALL
}

}  // namespace sg
