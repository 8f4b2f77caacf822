// sg_write.cuh -- the map-and-write pass (Section IV of the paper): every
// gasket cell of a level-r grid receives v(x, y); nothing else changes,
// except under fill stores (below), which write 0 to the off-gasket cells
// of the tiles they touch.
//
// Persistent kernels serve the four maps.  A "team" (one warp, or the whole
// CTA for big tiles) owns one tile at a time and walks its share
// of the tile list with a fixed stride:
//   lambda (all three intra-tile variants): the team decodes its tile with
//     the warp-parallel lambda(omega) of Theorem 1 (LambdaLane), walking the
//     block space in the row-major or the digit-interleaved order;
//   bounding box: tile q is (q mod n_b, q div n_b), the identity map.
// Inside a tile each thread visits a fixed list of tile-relative offsets,
// which does not depend on the tile, so it is computed once and kept in
// registers:
//   sub-box (lambda, bounding box): every slot of the rho x rho tile, each
//     tested with (x & y) == 0 (Section III-D, Bounding Sub-boxes);
//   lookup table: the 3^s member slots in row-major order (Section III-D,
//     Shared Lookup Table); each thread computes its own entries once;
//   further unrolling: slot e is mapped by lambda applied at thread level
//     (Section III-D, Further Unrolling).
//
// Four ways to store:
//   scatter: each thread stores its cells directly.  Only gasket bytes may
//     change, so stores are per cell and the L2 merges them into partially
//     written 32-byte sectors, which it must fill from DRAM before writing
//     back (a read-modify-write per touched sector done by the memory system).
//   tma: a persistent team keeps STAGES-1 whole tiles in flight with 2-D
//     bulk tensor copies (cp.async.bulk.tensor, completing on mbarriers),
//     overwrites only the gasket cells of the tile in shared memory and
//     stores the tile back with a bulk tensor copy.  The read-modify-write is
//     implicit (off-gasket bytes go back as they came), whole rows of the tile
//     move, and the loads of later tiles overlap the hashing of this one.
//     Same concurrency rule as staged stores.
//   staged: the team loads the tile's touched 16-byte chunks (coalesced),
//     computes the new values into a shared-memory copy of the tile, merges
//     them into the loaded chunks under the gasket mask and stores whole
//     chunks.  Off-gasket bytes are written back with the value just read, so
//     no other kernel may write the same grid concurrently (the usual rule
//     for a read-modify-write).  Chunks of one sector are handled together
//     whenever the sector lies inside one tile, so the L2 sees whole-sector
//     writes and needs no fill.
//   fill: write-only; the tile is built in shared memory (0 at every
//     off-gasket cell, v at the gasket cells) and leaves with one bulk tensor
//     store.  Equal to the others whenever the grid is 0 off the gasket (the
//     paper's zero matrix and the stencils' invariant), and reads nothing.
#pragma once

#include "sg_device.cuh"
#include "sg_internal.h"
#include "sg_tma.cuh"
#include "sg_write_sector.cuh"

namespace sg {

constexpr int kWriteThreads = 256;

template <typename T, int S> struct WriteShape {
    static constexpr int RHO = 1 << S;
    static constexpr int SLOTS = RHO * RHO;
    static constexpr int MEMBERS = pow3i(S);
    // staged path
    static constexpr int ROW_BYTES = RHO * (int)sizeof(T);
    static constexpr int TILE_BYTES = RHO * ROW_BYTES;
    static constexpr bool STAGE_OK = ROW_BYTES >= 16;
    static constexpr int CHUNK_ELEMS = 16 / (int)sizeof(T);
    static constexpr int CPR = STAGE_OK ? ROW_BYTES / 16 : 1;       // chunks per row
    static constexpr int CHUNKS = RHO * CPR;
    static constexpr int GROUP_ELEMS = (ROW_BYTES >= 32 ? 32 : 16) / (int)sizeof(T);
};

// Team size: one warp while a tile is small, the CTA for big tiles.
template <typename T, int S, bool STAGED> struct WriteTeam {
    using WS = WriteShape<T, S>;
    static constexpr int TEAM = STAGED ? (WS::TILE_BYTES <= 1024 ? 32 : kWriteThreads)
                                       : (S >= 5 ? kWriteThreads : 32);
};

// Member slot e (0 <= e < 3^S) of a level-S tile in row-major order, the
// order of the paper's lookup table.  Row t holds 2^(S - popcount(t))
// members (the subsets of ~t), so of the rows that share the bits of t above
// bit b, those with bit b clear hold twice as many members as those with it
// set: 2 m 3^b against m 3^b, m = 2^(zero bits above b).  Walking the bits
// from the top picks the row of member e in S steps; e's rank inside the row
// then gives tx, its bits placed at the zero positions of ty.  Returns
// tx | ty << 8.
template <int S>
__device__ __forceinline__ uint32_t member_rowmajor(int e)
{
    int ty = 0, m = 1;
#pragma unroll
    for (int b = S - 1; b >= 0; --b) {
        const int clear = 2 * m * pow3i(b);     // members in the rows with bit b clear
        if (e < clear) {
            m *= 2;
        } else {
            e -= clear;
            ty |= 1 << b;
        }
    }
    int tx = 0, k = 0;
#pragma unroll
    for (int b = 0; b < S; ++b)
        if (!((ty >> b) & 1)) { tx |= ((e >> k) & 1) << b; ++k; }
    return (uint32_t)tx | ((uint32_t)ty << 8);
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

// This thread's tile-independent offsets (tx | ty << 8, or ~0u): slots of the
// sub-box, or member slots from the lookup table or the unrolled map.  A
// thread computes the table entries it visits itself, once, and keeps them in
// registers for every tile, instead of reading a table built in shared memory.
template <int S, int MAP, int TEAM, int ITERS>
__device__ __forceinline__ void intra_tile_offsets(uint32_t (&off)[ITERS], int t_in_team)
{
    constexpr int RHO = 1 << S, SLOTS = RHO * RHO, MEMBERS = pow3i(S);
    if constexpr (MAP == kMapLut) {
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int e = t_in_team + j * TEAM;
            off[j] = (e < MEMBERS) ? member_rowmajor<S>(e) : ~0u;
        }
    } else if constexpr (MAP == kMapUnroll) {
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int e = t_in_team + j * TEAM;
            off[j] = (e < MEMBERS) ? unrolled_offset<S>(e) : ~0u;
        }
    } else {
#pragma unroll
        for (int j = 0; j < ITERS; ++j) {
            const int slot = t_in_team + j * TEAM;
            off[j] = (slot < SLOTS) ? (uint32_t)((slot & (RHO - 1)) | ((slot >> S) << 8)) : ~0u;
        }
    }
}

// Tile walker: the team's sequence of tiles under a map and traversal order.
template <int MAP>
struct TileWalker {
    LambdaLane ll;
    OmegaWalker ow;
    int rb;
    __device__ __forceinline__ void init(int lane, int rb_, int order, uint64_t team,
                                         uint64_t nteams)
    {
        rb = rb_;
        if constexpr (MAP != kMapBBox) {
            ll.init(lane, rb, order);
            ow.init((uint32_t)team, (uint32_t)nteams, pi_word(order, rb));
        }
    }
    // Block coordinate of tile q (q advances by nteams between calls).
    __device__ __forceinline__ uint2 next(uint64_t q)
    {
        if constexpr (MAP == kMapBBox) {
            return make_uint2((uint32_t)(q & ((1ull << rb) - 1)), (uint32_t)(q >> rb));
        } else {
            const uint2 b = ll.decode(ow.a, ow.b);
            ow.advance();
            return b;
        }
    }
};

// ---------------------------------------------------------------------------
// Scatter stores.
// ---------------------------------------------------------------------------
template <typename T, int VK, int S, int MAP>
__global__ void __launch_bounds__(kWriteThreads)
write_scatter_kernel(T *__restrict__ grid, int r, int order, uint64_t vs, uint64_t ntiles)
{
    using WS = WriteShape<T, S>;
    constexpr int RHO = WS::RHO;
    constexpr int TEAM = WriteTeam<T, S, false>::TEAM;
    constexpr bool SUBBOX = (MAP == kMapLambda || MAP == kMapBBox);
    constexpr int NSLOT = SUBBOX ? WS::SLOTS : WS::MEMBERS;
    constexpr int ITERS = (NSLOT + TEAM - 1) / TEAM;
    constexpr int TEAMS_PER_CTA = kWriteThreads / TEAM;

    const int t_in_team = threadIdx.x % TEAM;
    const uint64_t team = (uint64_t)blockIdx.x * TEAMS_PER_CTA + threadIdx.x / TEAM;
    const uint64_t nteams = (uint64_t)gridDim.x * TEAMS_PER_CTA;
    const uint64_t seedmix = vs * kGoldenGamma;

    uint32_t off[ITERS];
    intra_tile_offsets<S, MAP, TEAM, ITERS>(off, t_in_team);
    // tile-independent parts of each cell: grid offset (ty << r | tx, masked
    // to the tile so every address stays inside it) and value-key offset;
    // slots off the gasket are dropped (in a tile holding gasket cells,
    // (x & y) == 0 iff (tx & ty) == 0; empty bounding-box tiles are skipped)
    uint32_t goff[ITERS], koff[ITERS];
#pragma unroll
    for (int j = 0; j < ITERS; ++j) {
        const uint32_t tx = off[j] & (RHO - 1), ty = (off[j] >> 8) & (RHO - 1);
        const bool keep = off[j] != ~0u && (!SUBBOX || (tx & ty) == 0u);
        goff[j] = keep ? (ty << r) | tx : ~0u;
        koff[j] = CellValue<T, VK>::offset_of(tx, ty, r);
    }
    const CellValue<T, VK> cv{seedmix, (uint32_t)vs};
    TileWalker<MAP> tw;
    tw.init(threadIdx.x & 31, r - S, order, team, nteams);

    for (uint64_t q = team; q < ntiles; q += nteams) {
        const uint2 b = tw.next(q);
        if (MAP == kMapBBox && (b.x & b.y) != 0u) continue;   // no gasket cell
        const uint32_t x0 = b.x << S, y0 = b.y << S;
        T *tile = grid + (((uint64_t)y0 << r) | x0);
        const uint32_t base = CellValue<T, VK>::base_of(x0, y0, r);
#pragma unroll
        for (int j = 0; j < ITERS; ++j)
            if (goff[j] != ~0u) tile[goff[j]] = cv(base, koff[j]);
    }
}

// ---------------------------------------------------------------------------
// Staged stores.
// ---------------------------------------------------------------------------
// Gasket mask of a 16-byte chunk starting at column xc (a multiple of the
// chunk width) on row y, as byte lanes of 0xFF (u8) or element lanes (f32).
__device__ __forceinline__ uint4 chunk_mask_u8(uint32_t xc, uint32_t y)
{
    if ((xc & y) != 0u) return make_uint4(0u, 0u, 0u, 0u);
    const uint32_t yl = y & 15u;
    uint32_t w = 0xFFFFFFFFu;
    if (yl & 1u) w &= 0x00FF00FFu;
    if (yl & 2u) w &= 0x0000FFFFu;
    uint4 m = make_uint4(w, w, w, w);
    if (yl & 4u) { m.y = 0u; m.w = 0u; }
    if (yl & 8u) { m.z = 0u; m.w = 0u; }
    return m;
}

__device__ __forceinline__ uint4 chunk_mask_f32(uint32_t xc, uint32_t y)
{
    return make_uint4(in_gasket(xc, y) ? ~0u : 0u, in_gasket(xc + 1u, y) ? ~0u : 0u,
                      in_gasket(xc + 2u, y) ? ~0u : 0u, in_gasket(xc + 3u, y) ? ~0u : 0u);
}

template <typename T>
__device__ __forceinline__ uint4 chunk_mask(uint32_t xc, uint32_t y)
{
    if constexpr (sizeof(T) == 1) return chunk_mask_u8(xc, y);
    else return chunk_mask_f32(xc, y);
}

__device__ __forceinline__ uint4 merge4(uint4 old, uint4 nw, uint4 m)
{
    return make_uint4((old.x & ~m.x) | (nw.x & m.x), (old.y & ~m.y) | (nw.y & m.y),
                      (old.z & ~m.z) | (nw.z & m.z), (old.w & ~m.w) | (nw.w & m.w));
}

template <int TEAM>
__device__ __forceinline__ void team_sync()
{
    if constexpr (TEAM == 32) __syncwarp();
    else __syncthreads();
}

template <typename T, int VK, int S, int MAP>
__global__ void __launch_bounds__(kWriteThreads)
write_staged_kernel(T *__restrict__ grid, int r, int order, uint64_t vs, uint64_t ntiles,
                    int read)
{
    using WS = WriteShape<T, S>;
    static_assert(WS::STAGE_OK, "staged stores need tile rows of at least 16 bytes");
    constexpr int RHO = WS::RHO;
    constexpr int TEAM = WriteTeam<T, S, true>::TEAM;
    constexpr bool SUBBOX = (MAP == kMapLambda || MAP == kMapBBox);
    constexpr int NSLOT = SUBBOX ? WS::SLOTS : WS::MEMBERS;
    constexpr int ITERS = (NSLOT + TEAM - 1) / TEAM;
    constexpr int CPT = (WS::CHUNKS + TEAM - 1) / TEAM;      // chunks per thread
    constexpr int TEAMS_PER_CTA = kWriteThreads / TEAM;
    __shared__ __align__(16) T tile[TEAMS_PER_CTA][WS::SLOTS];

    const int t_in_team = threadIdx.x % TEAM;
    const int team_in_cta = threadIdx.x / TEAM;
    const uint64_t team = (uint64_t)blockIdx.x * TEAMS_PER_CTA + team_in_cta;
    const uint64_t nteams = (uint64_t)gridDim.x * TEAMS_PER_CTA;
    const uint64_t seedmix = vs * kGoldenGamma;
    T *my = tile[team_in_cta];

    uint32_t off[ITERS];
    intra_tile_offsets<S, MAP, TEAM, ITERS>(off, t_in_team);
    uint32_t koff[ITERS], soff[ITERS];
#pragma unroll
    for (int j = 0; j < ITERS; ++j) {
        const uint32_t tx = off[j] & (RHO - 1), ty = (off[j] >> 8) & (RHO - 1);
        const bool keep = off[j] != ~0u && (!SUBBOX || (tx & ty) == 0u);
        koff[j] = CellValue<T, VK>::offset_of(tx, ty, r);
        soff[j] = keep ? ty * RHO + tx : ~0u;
    }
    const CellValue<T, VK> cv{seedmix, (uint32_t)vs};
    TileWalker<MAP> tw;
    tw.init(threadIdx.x & 31, r - S, order, team, nteams);

    for (uint64_t q = team; q < ntiles; q += nteams) {
        const uint2 b = tw.next(q);
        if (MAP == kMapBBox && (b.x & b.y) != 0u) continue;   // no gasket cell
        const uint32_t x0 = b.x << S, y0 = b.y << S;

        // 1. issue the loads of this thread's touched chunks
        uint4 old[CPT];
        bool act[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = t_in_team + k * TEAM;
            const int row = c / WS::CPR, cx = c % WS::CPR;
            const uint32_t xc = x0 + (uint32_t)(cx * WS::CHUNK_ELEMS), y = y0 + (uint32_t)row;
            const uint32_t xg = xc & ~(uint32_t)(WS::GROUP_ELEMS - 1);   // its sector group
            act[k] = (c < WS::CHUNKS) && in_gasket(xg, y);
            // read == 0: the fill contract, nothing read (off-gasket cells of
            // the chunks written become 0)
            old[k] = act[k] && read
                         ? *reinterpret_cast<const uint4 *>(grid + ((uint64_t)y << r) + xc)
                         : make_uint4(0u, 0u, 0u, 0u);
        }
        // 2. new values into the shared copy of the tile
        team_sync<TEAM>();        // the previous tile's merge has read `my`
        const uint32_t base = CellValue<T, VK>::base_of(x0, y0, r);
#pragma unroll
        for (int j = 0; j < ITERS; ++j)
            if (soff[j] != ~0u) my[soff[j]] = cv(base, koff[j]);
        team_sync<TEAM>();
        // 3. merge under the gasket mask and store whole chunks
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (!act[k]) continue;
            const int c = t_in_team + k * TEAM;
            const int row = c / WS::CPR, cx = c % WS::CPR;
            const uint32_t xc = x0 + (uint32_t)(cx * WS::CHUNK_ELEMS), y = y0 + (uint32_t)row;
            const uint4 nw = *reinterpret_cast<const uint4 *>(my + row * RHO + cx * WS::CHUNK_ELEMS);
            *reinterpret_cast<uint4 *>(grid + ((uint64_t)y << r) + xc) =
                merge4(old[k], nw, chunk_mask<T>(xc, y));
        }
    }
}


// ---------------------------------------------------------------------------
// TMA-pipelined stores.
// ---------------------------------------------------------------------------
constexpr int kTmaThreads = 128;

template <typename T, int S, int MAP> struct TmaShape {
    static constexpr int RHO = 1 << S;
    static constexpr bool OK = RHO * (int)sizeof(T) >= 16;
    static constexpr int TILE_BYTES = RHO * RHO * (int)sizeof(T);
    static constexpr int BUF = (TILE_BYTES + 127) / 128 * 128;      // 128-byte aligned slots
    static constexpr bool SUBBOX = (MAP == kMapLambda || MAP == kMapBBox);
    static constexpr int NSLOT = SUBBOX ? RHO * RHO : pow3i(S);
    static constexpr int TEAM = NSLOT > 96 ? kTmaThreads : 32;
    static constexpr int TEAMS = kTmaThreads / TEAM;
    static constexpr int ITERS = (NSLOT + TEAM - 1) / TEAM;
    static constexpr int STAGES = TILE_BYTES <= 1024 ? 6 : (TILE_BYTES <= 4096 ? 4 : 3);
    static constexpr size_t DSMEM = (size_t)TEAMS * STAGES * BUF + 128;
};

template <typename T, int VK, int S, int MAP>
__global__ void __launch_bounds__(kTmaThreads)
write_tma_kernel(const __grid_constant__ CUtensorMap tmap, int r, int order, uint64_t vs,
                 uint64_t ntiles, int *status)
{
    using TS = TmaShape<T, S, MAP>;
    constexpr int RHO = TS::RHO, TEAM = TS::TEAM, TEAMS = TS::TEAMS, ST = TS::STAGES;
    constexpr int ITERS = TS::ITERS;
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full[TEAMS][ST];
    __shared__ uint2 coord[TEAMS][ST];
    __shared__ int abort_team[TEAMS];

    const int tid = threadIdx.x, lane = tid & 31;
    const int tm = tid / TEAM, t = tid % TEAM;
    const bool producer_warp = t < 32;             // the team's first warp issues copies
    const uint64_t team = (uint64_t)blockIdx.x * TEAMS + tm;
    const uint64_t nteams = (uint64_t)gridDim.x * TEAMS;
    const uint64_t seedmix = vs * kGoldenGamma;
    uint8_t *dsm = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~(uintptr_t)127);
    uint8_t *buf = dsm + (size_t)tm * ST * TS::BUF;

    uint32_t off[ITERS];
    intra_tile_offsets<S, MAP, TEAM, ITERS>(off, t);
    uint32_t koff[ITERS], soff[ITERS];
#pragma unroll
    for (int j = 0; j < ITERS; ++j) {
        const uint32_t tx = off[j] & (RHO - 1), ty = (off[j] >> 8) & (RHO - 1);
        const bool keep = off[j] != ~0u && (!TS::SUBBOX || (tx & ty) == 0u);
        koff[j] = CellValue<T, VK>::offset_of(tx, ty, r);
        soff[j] = keep ? ty * RHO + tx : ~0u;
    }
    const CellValue<T, VK> cv{seedmix, (uint32_t)vs};
    if (t == 0) {
        for (int i = 0; i < ST; ++i) mbar_init(&full[tm][i], 1);
        abort_team[tm] = 0;
    }
    mbar_init_fence();
    __syncthreads();

    TileWalker<MAP> tw;
    if (producer_warp) tw.init(lane, r - S, order, team, nteams);
    const uint64_t cnt = team < ntiles ? (ntiles - team + nteams - 1) / nteams : 0;

    // issue tile k of this team into slot k % ST (warp-collective decode).
    // A bounding-box tile without gasket cells moves nothing: its slot is
    // released with a plain arrive and the consumers skip it.
    auto issue = [&](uint64_t k) {
        const uint2 b = tw.next(team + k * nteams);
        if (lane == 0) {
            const int sn = (int)(k % ST);
            coord[tm][sn] = b;
            if (MAP == kMapBBox && (b.x & b.y) != 0u) {
                mbar_arrive(&full[tm][sn]);
            } else {
                mbar_arrive_expect_tx(&full[tm][sn], (uint32_t)TS::TILE_BYTES);
                tma_load_2d(buf + sn * TS::BUF, &tmap, (int)(b.x << S), (int)(b.y << S),
                            &full[tm][sn]);
            }
        }
    };
    if (producer_warp)
        for (uint64_t k = 0; k + 1 < (uint64_t)ST && k < cnt; ++k) issue(k);

    for (uint64_t k = 0; k < cnt; ++k) {
        const int sl = (int)(k % ST);
        const bool got = mbar_wait_bounded(&full[tm][sl], (uint32_t)((k / ST) & 1));
        if (!got) {
            abort_team[tm] = 1;
            record_device_error(status, kDevTimeout);
        }
        const uint2 b = coord[tm][sl];
        const bool empty = MAP == kMapBBox && (b.x & b.y) != 0u;
        const uint32_t x0 = b.x << S, y0 = b.y << S;
        T *tile = reinterpret_cast<T *>(buf + sl * TS::BUF);
        if (got && !empty) {
            const uint32_t base = CellValue<T, VK>::base_of(x0, y0, r);
#pragma unroll
            for (int j = 0; j < ITERS; ++j)
                if (soff[j] != ~0u) tile[soff[j]] = cv(base, koff[j]);
        }
        fence_proxy_async_shared();
        team_sync<TEAM>();
        if (abort_team[tm]) {
            // a copy never completed: let the ones still in flight land (bounded)
            // before this block's shared memory goes away
            // (tiles k .. k+ST-2 were issued; tile k+ST-1 never was)
            if (t == 0)
                for (uint64_t kk = k; kk < cnt && kk + 1 < k + ST; ++kk)
                    (void)mbar_wait_bounded(&full[tm][kk % ST], (uint32_t)((kk / ST) & 1));
            break;
        }
        if (t == 0) {
            if (!empty) tma_store_2d(&tmap, (int)x0, (int)y0, tile);
            bulk_commit();              // (an empty group for an empty tile)
            bulk_wait_read<1>();        // the previous tile's slot is free again
        }
        if (producer_warp && k + ST - 1 < cnt) issue(k + ST - 1);
    }
    if (t == 0) bulk_wait_all();
}


// One element into shared memory at a shared-window address.
__device__ __forceinline__ void st_shared(uint32_t addr, uint8_t v)
{
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(addr), "r"((uint32_t)v));
}
__device__ __forceinline__ void st_shared(uint32_t addr, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

// ---------------------------------------------------------------------------
// Fill stores (write-only): the tile is built in shared memory -- 0 at every
// off-gasket cell, v(x, y) at every gasket cell -- and written back whole
// with a 2-D bulk tensor copy; nothing is read.  For grids that are 0 off
// the gasket (the paper's zero matrix, and the stencils' invariant) this is
// the same result as the preserving paths with a third of the DRAM traffic.
// Each team rotates through STAGES shared-memory slots so the hashing of
// one tile overlaps the bulk stores of the previous ones.
// ---------------------------------------------------------------------------
template <typename T, int VK, int S, int MAP>
__global__ void __launch_bounds__(kTmaThreads)
write_fill_kernel(const __grid_constant__ CUtensorMap tmap, int r, int order, uint64_t vs,
                  uint64_t ntiles)
{
    using TS = TmaShape<T, S, MAP>;
    constexpr int RHO = TS::RHO, TEAM = TS::TEAM, TEAMS = TS::TEAMS, ST = TS::STAGES;
    constexpr int ITERS = TS::ITERS;
    static_assert(ST >= 2, "the slot ring needs two slots");
    extern __shared__ uint8_t dsm_raw[];

    const int tid = threadIdx.x, lane = tid & 31;
    const int tm = tid / TEAM, t = tid % TEAM;
    const uint64_t team = (uint64_t)blockIdx.x * TEAMS + tm;
    const uint64_t nteams = (uint64_t)gridDim.x * TEAMS;
    const uint64_t seedmix = vs * kGoldenGamma;
    uint8_t *dsm = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~(uintptr_t)127);
    uint8_t *buf = dsm + (size_t)tm * ST * TS::BUF;

    // The gasket cells of a tile sit at the same tile-relative places in
    // every tile, so each slot is zeroed once here and afterwards only its
    // gasket cells are rewritten: its other cells stay 0 for the whole pass.
    for (int i = tid; i < TEAMS * ST * TS::BUF / 16; i += kTmaThreads)
        reinterpret_cast<uint4 *>(dsm)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_shared();        // the zeros are read by other teams' bulk stores too
    uint32_t off[ITERS];
    intra_tile_offsets<S, MAP, TEAM, ITERS>(off, t);
    __syncthreads();                   // every slot zeroed before any team stores
    // per-thread, tile-independent parts of each cell: value-key offset and
    // shared-memory offset (slots off the gasket are dropped: for a tile that
    // holds gasket cells, (x & y) == 0 iff (tx & ty) == 0)
    // The shared-memory address is that of the cell in slot 0 (~0u for a
    // slot that is no gasket cell); slot k is k * BUF bytes further, a
    // constant in the sweep over the slots below, which is unrolled, so a
    // cell's store needs no address arithmetic.
    const uint32_t buf_s = (uint32_t)__cvta_generic_to_shared(buf);
    uint32_t koff[ITERS], cell[ITERS];
#pragma unroll
    for (int j = 0; j < ITERS; ++j) {
        const uint32_t tx = off[j] & (RHO - 1), ty = (off[j] >> 8) & (RHO - 1);
        const bool keep = off[j] != ~0u && (!TS::SUBBOX || (tx & ty) == 0u);
        koff[j] = CellValue<T, VK>::offset_of(tx, ty, r);
        cell[j] = keep ? buf_s + (ty * RHO + tx) * (uint32_t)sizeof(T) : ~0u;
    }
    const CellValue<T, VK> cv{seedmix, (uint32_t)vs};
    TileWalker<MAP> tw;
    tw.init(lane, r - S, order, team, nteams);

    // Iteration k writes slot k % ST.  Before the barrier of iteration k the
    // issuing thread has waited (end of iteration k-1) until every store but
    // the newest ST-2 has read its slot, i.e. through the store of tile
    // k+1-ST, which is the last tile that used slot (k+1) % ST -- the slot
    // iteration k+1 writes after that barrier.  (Tiles number below 2^32:
    // fill needs rho * sizeof(T) >= 16, so r - s <= 12.)
    const uint32_t nt = (uint32_t)ntiles, stride = (uint32_t)nteams;
    uint32_t q = (uint32_t)team;
    while (q < nt) {
#pragma unroll
        for (int sl = 0; sl < ST; ++sl) {
            if (q >= nt) break;
            const uint2 b = tw.next(q);              // every warp of the team decodes
            const bool empty = MAP == kMapBBox && (b.x & b.y) != 0u;
            const uint32_t x0 = b.x << S, y0 = b.y << S;
            if (!empty) {
                const uint32_t base = CellValue<T, VK>::base_of(x0, y0, r);
#pragma unroll
                for (int j = 0; j < ITERS; ++j) {
                    // the member lists (lookup table, unrolling) fill every
                    // thread's first slots: only the last one may be empty
                    const bool full = !TS::SUBBOX && (j + 1) * TEAM <= TS::NSLOT;
                    if (full || cell[j] != ~0u)
                        st_shared(cell[j] + (uint32_t)(sl * TS::BUF), cv(base, koff[j]));
                }
                fence_proxy_async_shared();
            }
            team_sync<TEAM>();
            if (t == 0) {
                if (!empty) tma_store_2d(&tmap, (int)x0, (int)y0, buf + sl * TS::BUF);
                bulk_commit();             // one group per tile (empty for an empty tile)
                bulk_wait_read<ST - 2>();
            }
            q += stride;
        }
    }
    if (t == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int VK, int S, int MAP>
cudaError_t launch_write_tma(int r, T *grid, uint64_t vs, uint64_t ntiles, cudaStream_t st,
                             const LaunchCfg &cfg)
{
    using TS = TmaShape<T, S, MAP>;
    if constexpr (!TS::OK) {
        return cudaErrorNotSupported;
    } else {
        CUtensorMap map;
        cudaError_t e = make_grid_tensor_map(&map, grid, r, (int)sizeof(T), 1 << S);
        if (e != cudaSuccess) return e;
        int *status = nullptr;
        e = device_status_ptr(&status);
        if (e != cudaSuccess) return e;
        auto kern = write_tma_kernel<T, VK, S, MAP>;
        if (TS::DSMEM > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TS::DSMEM);
            if (e != cudaSuccess) return e;
        }
        static std::atomic<int> occ{0};
        unsigned grid_ctas = 1;
        const uint64_t units = (ntiles + TS::TEAMS - 1) / TS::TEAMS;
        e = persistent_grid(kern, kTmaThreads, TS::DSMEM, units, cfg, &grid_ctas, &occ);
        if (e != cudaSuccess) return e;
        kern<<<grid_ctas, kTmaThreads, TS::DSMEM, st>>>(map, r, cfg.order, vs, ntiles, status);
        return cudaGetLastError();
    }
}

template <typename T, int VK, int S, int MAP>
cudaError_t launch_write_fill(int r, T *grid, uint64_t vs, uint64_t ntiles, cudaStream_t st,
                              const LaunchCfg &cfg)
{
    using TS = TmaShape<T, S, MAP>;
    if constexpr (!TS::OK) {
        return cudaErrorNotSupported;
    } else {
        CUtensorMap map;
        cudaError_t e = make_grid_tensor_map(&map, grid, r, (int)sizeof(T), 1 << S);
        if (e != cudaSuccess) return e;
        auto kern = write_fill_kernel<T, VK, S, MAP>;
        if (TS::DSMEM > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TS::DSMEM);
            if (e != cudaSuccess) return e;
        }
        static std::atomic<int> occ{0};
        unsigned grid_ctas = 1;
        const uint64_t units = (ntiles + TS::TEAMS - 1) / TS::TEAMS;
        e = persistent_grid(kern, kTmaThreads, TS::DSMEM, units, cfg, &grid_ctas, &occ);
        if (e != cudaSuccess) return e;
        kern<<<grid_ctas, kTmaThreads, TS::DSMEM, st>>>(map, r, cfg.order, vs, ntiles);
        return cudaGetLastError();
    }
}

template <typename T, int VK, int S, int MAP>
cudaError_t launch_write_t(int r, T *grid, uint64_t vs, cudaStream_t st, const LaunchCfg &cfg)
{
    const int rb = r - S;
    const uint64_t ntiles = (MAP == kMapBBox) ? (1ull << (2 * rb)) : (uint64_t)pow3i(rb);
    if (cfg.store == kStoreTma) return launch_write_tma<T, VK, S, MAP>(r, grid, vs, ntiles, st, cfg);
    if (cfg.store == kStoreSector || cfg.store == kStoreMerge || cfg.store == kStoreMasked)
        return launch_write_sector<T, VK, S, MAP>(r, grid, vs, ntiles, st, cfg);
    if (cfg.store == kStoreFill) return launch_write_fill<T, VK, S, MAP>(r, grid, vs, ntiles, st, cfg);
    using WS = WriteShape<T, S>;
    bool staged = false;     // the caller resolved kStoreAuto already
    if constexpr (WS::STAGE_OK)
        staged = (cfg.store == kStoreStaged || cfg.store == kStoreFillPlain);
    unsigned grid_ctas = 1;
    cudaError_t e;
    if constexpr (WS::STAGE_OK) {
        if (staged) {
            constexpr int TEAM = WriteTeam<T, S, true>::TEAM;
            static std::atomic<int> occ{0};
            auto kern = write_staged_kernel<T, VK, S, MAP>;
            const uint64_t units = (ntiles * TEAM + kWriteThreads - 1) / kWriteThreads;
            e = persistent_grid(kern, kWriteThreads, 0, units, cfg, &grid_ctas, &occ);
            if (e != cudaSuccess) return e;
            kern<<<grid_ctas, kWriteThreads, 0, st>>>(grid, r, cfg.order, vs, ntiles,
                                                      cfg.store == kStoreStaged ? 1 : 0);
            return cudaGetLastError();
        }
    }
    if (cfg.store == kStoreStaged || cfg.store == kStoreFillPlain) return cudaErrorNotSupported;
    constexpr int TEAM = WriteTeam<T, S, false>::TEAM;
    static std::atomic<int> occ{0};
    auto kern = write_scatter_kernel<T, VK, S, MAP>;
    const uint64_t units = (ntiles * TEAM + kWriteThreads - 1) / kWriteThreads;
    e = persistent_grid(kern, kWriteThreads, 0, units, cfg, &grid_ctas, &occ);
    if (e != cudaSuccess) return e;
    kern<<<grid_ctas, kWriteThreads, 0, st>>>(grid, r, cfg.order, vs, ntiles);
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
