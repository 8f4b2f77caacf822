// sg_compact_stencil.cu -- the B3/S23 CA step and the diffusion step on
// compact arrays (layout in sg_compact.cuh).
//
// Each warp of a persistent grid takes units of 729 elements (G whole tiles)
// on its own, with a staging region of its own in shared memory:
//   1. it decodes the unit's tiles (lambda reduction of Theorem 1) and copies
//      the unit's values in (32 consecutive elements per load: whole
//      sectors);
//   2. it fetches each tile's halo: the 8 (CA) or 4 (diffusion) cells of
//      neighbouring tiles that touch it.  A neighbouring block exists when it
//      lies in the block grid and (bx & by) == 0; its launch index comes from
//      lambda_index, the inverse of the decode.  Missing neighbours read 0;
//   3. it updates the unit's elements from shared memory and stores them in
//      whole sectors.  Where each neighbour of position c sits among the
//      staged values is read from a per-CTA table expanded from the
//      compile-time tables, so a cell costs one table load and 8 (4) value
//      loads from shared memory.
// Warps never wait for one another after the table is built: the latency of
// one warp's loads is covered by the other warps of the SM.  Only gasket
// cells exist here: nothing is spent on the off-gasket 82 % of a 64-tile, and
// the state of a level-15 CA (14.3 MB) stays in L2.
//
// The CA on 64-tiles runs bit-sliced instead (compact_ca_bits_kernel below):
// the gather above spends 9 shared loads per cell and is bound by the L1 /
// shared-memory pipe, while rows of bits take the rule 64 cells at a time.
//
// The cell arithmetic is the embedded kernels' own (life rule on (count |
// self) == 3; diffusion through diffuse_update with the same grouping of the
// neighbour sum), so a compact step equals the embedded step cell for cell.
#include "sg_compact.cuh"
#include "sg_stencil.cuh"

namespace sg {

namespace {

// Staged values of a unit: its 729 elements, then G * H halo cells, then one
// zero that neighbours off the gasket point at.
template <int S, int H> struct UnitStage {
    static constexpr int G = CompactPattern<S>::G;
    static constexpr int HALO = kUnit, ZERO = kUnit + G * H, SIZE = ZERO + 1;
};

// Resolve a table entry (index in the tile / kHaloBit | h / kNoCell) of a
// cell of tile g into an index of the staged values.
template <int S, int H>
__device__ __forceinline__ uint32_t stage_slot(uint16_t v, int g)
{
    using U = UnitStage<S, H>;
    if (v == kNoCell) return (uint32_t)U::ZERO;
    if (v & kHaloBit) return (uint32_t)(U::HALO + g * H + (v & (kHaloBit - 1)));
    return (uint32_t)(g * CompactPattern<S>::C + v);
}

// The halo cell h of tile g: value of the neighbouring tile's cell, or 0
// (and *present = false) when that tile is outside the grid or empty.
template <typename T, int S>
__device__ __forceinline__ T halo_value(const T *__restrict__ in, uint2 b, int dbx, int dby,
                                        uint32_t rank, int rb, int order, bool *present)
{
    *present = false;
    if (b.x == 0xFFFFFFFFu) return T(0);
    const uint32_t nbx = b.x + (uint32_t)dbx, nby = b.y + (uint32_t)dby;   // wraps when < 0
    if ((nbx >> rb) != 0u || (nby >> rb) != 0u || (nbx & nby) != 0u) return T(0);
    *present = true;
    const uint64_t q = lambda_index(nbx, nby, rb, order);
    return in[q * (uint64_t)CompactPattern<S>::C + rank];
}

// Shared memory of a CTA: the unit table (per position, where its
// neighbours sit among the staged values), then one region per warp with the
// unit's tile coordinates, halo presence bytes and staged values.
template <typename T, int S, int H, int TABLE_BYTES> struct StencilSmem {
    static constexpr int G = CompactPattern<S>::G;
    using U = UnitStage<S, H>;
    static constexpr int COORD = 0, PRES = G * 8, VALS = ((G * 8 + G * 4) + 15) / 16 * 16;
    static constexpr int WARP = (VALS + U::SIZE * (int)sizeof(T) + 15) / 16 * 16;
    static constexpr int TABLE = TABLE_BYTES;
    static constexpr int BYTES = TABLE + kUnitWarps * WARP;
    static_assert(TABLE % 16 == 0 && WARP % 16 == 0 && VALS % 16 == 0 && PRES % 8 == 0,
                  "every region aligned for its widest element");
};

// Stage unit u into the warp's region: its values, then the halo cells of
// each of its tiles (with presence bytes when `pres` is given).  Called by
// all lanes of the warp; returns the number of elements in the unit.
template <typename T, int S, int H>
__device__ __forceinline__ uint32_t stage_unit(T *sv, uint2 *coord, uint8_t *pres,
                                               const T *__restrict__ in, uint32_t u,
                                               uint32_t total, uint32_t ntiles, uint32_t W,
                                               const LambdaLane &ll, const int8_t (*hl)[4],
                                               const uint16_t *hrank, int rb, int order)
{
    using U = UnitStage<S, H>;
    constexpr int G = U::G;
    const int lane = threadIdx.x & 31;
    decode_unit_tiles<G>(coord, u * G, ntiles, W, ll);
    const uint32_t base = u * kUnit;
    const uint32_t cnt = min((uint32_t)kUnit, total - base);
#pragma unroll 4
    for (uint32_t c = lane; c < cnt; c += 32) sv[c] = in[base + c];
    __syncwarp();                              // coord written by lane 0
    for (int h = lane; h < G * H; h += 32) {
        const int g = h / H, k = h - g * H;
        bool p;
        sv[U::HALO + h] = halo_value<T, S>(in, coord[g], hl[k][0], hl[k][1], hrank[k], rb, order,
                                           &p);
        if (pres) pres[h] = p ? 1 : 0;
    }
    if (lane == 0) sv[U::ZERO] = T(0);
    __syncwarp();
    return cnt;
}

template <int S>
__global__ void __launch_bounds__(kUnitThreads)
compact_ca_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r, int order,
                  uint32_t total)
{
    using M = StencilSmem<uint8_t, S, kCaHalo, kUnit * 16>;
    extern __shared__ __align__(16) unsigned char smem[];
    const CompactPattern<S> &pat = compact_pattern<S>();
    // per position: the staged-value index of each of its 8 neighbours
    uint4 *nbt = reinterpret_cast<uint4 *>(smem);
    for (int c = threadIdx.x; c < kUnit; c += kUnitThreads) {
        const int g = c / CompactPattern<S>::C, e = c - g * CompactPattern<S>::C;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w[k] = stage_slot<S, kCaHalo>(pat.ca_nb[e][2 * k], g) |
                   (stage_slot<S, kCaHalo>(pat.ca_nb[e][2 * k + 1], g) << 16);
        nbt[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *region = smem + M::TABLE + warp * M::WARP;
    uint2 *coord = reinterpret_cast<uint2 *>(region + M::COORD);
    uint8_t *sv = region + M::VALS;
    const int rb = r - S;
    const uint32_t ntiles = total / CompactPattern<S>::C, units = (total + kUnit - 1) / kUnit;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        __syncwarp();                          // the previous unit is finished
        const uint32_t cnt = stage_unit<uint8_t, S, kCaHalo>(
            sv, coord, nullptr, in, u, total, ntiles, W, ll, pat.ca_halo, pat.ca_halo_rank, rb,
            order);
        uint8_t *o = out + u * kUnit;
#pragma unroll 4
        for (uint32_t c = lane; c < cnt; c += 32) {
            const uint4 t = nbt[c];
            const uint32_t count = (uint32_t)sv[t.x & 0xFFFFu] + sv[t.x >> 16] +
                                   sv[t.y & 0xFFFFu] + sv[t.y >> 16] + sv[t.z & 0xFFFFu] +
                                   sv[t.z >> 16] + sv[t.w & 0xFFFFu] + sv[t.w >> 16];
            o[c] = (uint8_t)(((count | (uint32_t)sv[c]) == 3u) ? 1 : 0);
        }
    }
}

// ---------------------------------------------------------------------------
// CA, rho = 64: bit-sliced rows (the row codec of sg_compact.cuh moves a
// tile row between its compact run and a 64-bit word).  A warp takes one
// tile (729 elements) at a time:
//   1. ballots turn the 729 states (0 / 1) into 23 words of compact bits;
//   2. each lane deposits rows 2*lane and 2*lane + 1 into 64-bit row words,
//      a block at a time through dep[y & 7][block];
//   3. the B3/S23 rule runs on whole rows: horizontal 3-sums and 2-sums by
//      bitwise full adders, the rows above and below through shuffles, the
//      halo cells of the neighbouring tiles as edge bits;
//   4. the next rows are gathered back (cmp[y & 7][byte]) into compact bits
//      and stored as bytes.
// Non-member columns hold 0 in every row word and are dropped by the gather,
// so the rule can run on them freely.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t maj3(uint64_t a, uint64_t b, uint64_t c)
{
    return (a & b) | (c & (a ^ b));
}

// Horizontal sums of a row (bit x: cells x-1, x, x+1), with the cells left
// of column 0 and right of column 63 given as edge bits.
struct RowSums {
    uint64_t t0, t1;    // 3-sum L + v + R, bit planes
    uint64_t d0, d1;    // 2-sum L + R
};

__device__ __forceinline__ RowSums row_sums(uint64_t v, uint32_t left, uint32_t right)
{
    const uint64_t L = (v << 1) | (uint64_t)left, R = (v >> 1) | ((uint64_t)right << 63);
    RowSums s;
    s.t0 = L ^ v ^ R;
    s.t1 = maj3(L, v, R);
    s.d0 = L ^ R;
    s.d1 = L & R;
    return s;
}

// B3/S23 on a row from the 3-sums above and below and its own 2-sum.
__device__ __forceinline__ uint64_t life_row(uint64_t u0, uint64_t u1, uint64_t m0, uint64_t m1,
                                             uint64_t b0, uint64_t b1, uint64_t self)
{
    const uint64_t s0 = u0 ^ m0 ^ b0, k0 = maj3(u0, m0, b0);
    const uint64_t t = u1 ^ m1 ^ b1, k1 = maj3(u1, m1, b1);
    const uint64_t s1 = t ^ k0, k2 = t & k0;
    // count = s0 + 2*s1 + 4*(k1 + k2): 2 or 3 iff s1 and no carry out of bit 1
    return s1 & ~(k1 | k2) & (s0 | self);
}

__device__ __forceinline__ uint64_t shfl_up64(uint64_t v)
{
    const uint32_t lo = __shfl_up_sync(0xffffffffu, (uint32_t)v, 1);
    const uint32_t hi = __shfl_up_sync(0xffffffffu, (uint32_t)(v >> 32), 1);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

__device__ __forceinline__ uint64_t shfl_down64(uint64_t v)
{
    const uint32_t lo = __shfl_down_sync(0xffffffffu, (uint32_t)v, 1);
    const uint32_t hi = __shfl_down_sync(0xffffffffu, (uint32_t)(v >> 32), 1);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

__global__ void __launch_bounds__(kUnitThreads, 5)
compact_ca_bits_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r, int order,
                       uint32_t total)
{
    constexpr int S = 6, WORDS = (kUnit + 31) / 32;           // 23 words of compact bits
    __shared__ RowCodec tc;
    __shared__ uint32_t cbits[kUnitWarps][WORDS + 3], obits[kUnitWarps][WORDS + 3];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&kRowCodec);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&tc);
        for (int i = threadIdx.x; i < (int)(sizeof(RowCodec) / 4); i += kUnitThreads)
            dst[i] = src[i];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *cb = cbits[warp], *ob = obits[warp];
    if (lane >= WORDS && lane < WORDS + 3) cb[lane] = 0u;     // guard words
    __syncthreads();
    static_assert(sizeof(RowCodec) % 4 == 0, "copied as words");

    const CompactPattern<S> &pat = compact_pattern<S>();
    const int rb = r - S;
    const uint32_t units = total / kUnit;                     // whole tiles: r >= 6
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t y0 = 2u * lane, y1 = y0 + 1u;
    const uint32_t o0 = tc.row_start[y0], o1 = tc.row_start[y1];
    // halo cell k of lane k: its place around the tile, (ex, ey) in [-1, 64]
    int ex = 0, ey = 0;
    if (lane < kCaHalo) {
        ex = pat.ca_halo[lane][0] * 64 + pat.ca_halo[lane][2];
        ey = pat.ca_halo[lane][1] * 64 + pat.ca_halo[lane][3];
    }
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        const uint32_t bq = u / W, aq = u - bq * W;
        const uint2 b = ll.decode(aq, bq);
        const uint32_t base = u * kUnit;
        // halo cells (lanes 0..7): their loads are issued first
        uint32_t hv = 0;
        if (lane < kCaHalo) {
            bool p;
            hv = halo_value<uint8_t, S>(in, b, pat.ca_halo[lane][0], pat.ca_halo[lane][1],
                                        pat.ca_halo_rank[lane], rb, order, &p);
        }
        // 1. compact bits: lane `it` keeps word `it`
        uint32_t mine = 0;
#pragma unroll
        for (int it = 0; it < WORDS; ++it) {
            const int c = 32 * it + lane;
            const uint8_t v = c < kUnit ? in[base + c] : 0;
            const uint32_t w = __ballot_sync(0xffffffffu, v != 0);
            if (lane == it) mine = w;
        }
        const bool alive = hv != 0;
        __syncwarp();                  // the previous tile's reads of cb are done
        if (lane < WORDS) cb[lane] = mine;
        if (lane < WORDS + 3) ob[lane] = 0u;
        // edge bits and the rows above row 0 and below row 63
        const uint32_t up_body = __ballot_sync(0xffffffffu, alive && ey == -1 && ex == 0);
        const uint32_t up_right = __ballot_sync(0xffffffffu, alive && ey == -1 && ex == 64);
        const uint32_t dn_body0 = __ballot_sync(0xffffffffu, alive && ey == 64 && ex == 0);
        const uint32_t dn_body1 = __ballot_sync(0xffffffffu, alive && ey == 64 && ex == 1);
        const uint32_t dn_left = __ballot_sync(0xffffffffu, alive && ey == 64 && ex == -1);
        const uint32_t l0 = __ballot_sync(0xffffffffu, alive && ey == 0 && ex == -1);
        const uint32_t r0 = __ballot_sync(0xffffffffu, alive && ey == 0 && ex == 64);
        const uint32_t r1 = __ballot_sync(0xffffffffu, alive && ey == 1 && ex == 64);
        __syncwarp();
        // 2. rows
        const uint64_t v0 = deposit_row(tc, bits_at(cb, o0), y0);
        const uint64_t v1 = deposit_row(tc, bits_at(cb, o1), y1);
        // 3. the rule; only lane 0 has cells beside the left and right edges
        const bool first = lane == 0, last = lane == 31;
        const RowSums a = row_sums(v0, first && l0, first && r0);
        const RowSums c = row_sums(v1, 0u, first && r1);
        uint64_t u0 = shfl_up64(c.t0), u1 = shfl_up64(c.t1);       // row y0 - 1
        uint64_t b0 = shfl_down64(a.t0), b1 = shfl_down64(a.t1);   // row y1 + 1
        if (first) {
            const RowSums h = row_sums(up_body ? 1ull : 0ull, 0u, up_right != 0u);
            u0 = h.t0;
            u1 = h.t1;
        }
        if (last) {
            const RowSums h = row_sums((dn_body0 ? 1ull : 0ull) | (dn_body1 ? 2ull : 0ull),
                                       dn_left != 0u, 0u);
            b0 = h.t0;
            b1 = h.t1;
        }
        const uint64_t n0 = life_row(u0, u1, a.d0, a.d1, c.t0, c.t1, v0);
        const uint64_t n1 = life_row(a.t0, a.t1, c.d0, c.d1, b0, b1, v1);
        // 4. back to compact bits, then bytes
        or_bits_at(ob, o0, gather_row(tc, n0, y0));
        or_bits_at(ob, o1, gather_row(tc, n1, y1));
        __syncwarp();
#pragma unroll
        for (int it = 0; it < WORDS; ++it) {
            const int cc = 32 * it + lane;
            if (cc < kUnit) out[base + cc] = (uint8_t)((ob[it] >> lane) & 1u);
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kUnitThreads)
compact_diffuse_kernel(const float *__restrict__ in, float *__restrict__ out, int r, int order,
                       uint32_t total, float alpha)
{
    using M = StencilSmem<float, S, kDiffHalo, kUnit * 16>;
    extern __shared__ __align__(16) unsigned char smem[];
    const CompactPattern<S> &pat = compact_pattern<S>();
    // per position: staged-value indices of (left, right), (above, below);
    // the tile within the unit and the gasket neighbours inside the tile; and
    // which halo presence bytes count towards the degree
    uint4 *nbt = reinterpret_cast<uint4 *>(smem);
    for (int c = threadIdx.x; c < kUnit; c += kUnitThreads) {
        const int g = c / CompactPattern<S>::C, e = c - g * CompactPattern<S>::C;
        uint32_t hsel = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint16_t v = pat.df_nb[e][k];
            if (v != kNoCell && (v & kHaloBit)) hsel |= 1u << (8 * (v & 3u));
        }
        nbt[c] = make_uint4(stage_slot<S, kDiffHalo>(pat.df_nb[e][0], g) |
                                (stage_slot<S, kDiffHalo>(pat.df_nb[e][1], g) << 16),
                            stage_slot<S, kDiffHalo>(pat.df_nb[e][2], g) |
                                (stage_slot<S, kDiffHalo>(pat.df_nb[e][3], g) << 16),
                            (uint32_t)pat.df_deg_in[e] | ((uint32_t)g << 8), hsel);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *region = smem + M::TABLE + warp * M::WARP;
    uint2 *coord = reinterpret_cast<uint2 *>(region + M::COORD);
    uint8_t *pres = region + M::PRES;
    const uint32_t *presw = reinterpret_cast<const uint32_t *>(region + M::PRES);
    float *sv = reinterpret_cast<float *>(region + M::VALS);
    const int rb = r - S;
    const uint32_t ntiles = total / CompactPattern<S>::C, units = (total + kUnit - 1) / kUnit;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        __syncwarp();
        const uint32_t cnt = stage_unit<float, S, kDiffHalo>(
            sv, coord, pres, in, u, total, ntiles, W, ll, pat.df_halo, pat.df_halo_rank, rb,
            order);
        float *o = out + u * kUnit;
#pragma unroll 4
        for (uint32_t c = lane; c < cnt; c += 32) {
            const uint4 t = nbt[c];
            uint32_t deg = t.z & 0xFFu;
            if (t.w) deg += __popc(presw[t.z >> 8] & t.w);
            const float l = sv[t.x & 0xFFFFu], rr = sv[t.x >> 16];
            const float up = sv[t.y & 0xFFFFu], dn = sv[t.y >> 16];
            o[c] = diffuse_update(sv[c], l, rr, up, dn, (float)deg, alpha);
        }
    }
}

template <int S>
cudaError_t launch_ca_t(int r, int order, const uint8_t *in, uint8_t *out, cudaStream_t st,
                        const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    const uint32_t total = (uint32_t)pow3i(r);
    const uint64_t units = (total + kUnit - 1) / kUnit;
    unsigned grid = 1;
    if constexpr (S == 6) {
        auto k = compact_ca_bits_kernel;
        cudaError_t e = persistent_grid(k, kUnitThreads, 0, (units + kUnitWarps - 1) / kUnitWarps,
                                        cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kUnitThreads, 0, st>>>(in, out, r, order, total);
    } else {
        static std::atomic<uint64_t> attr{0};
        auto k = compact_ca_kernel<S>;
        constexpr int smem = StencilSmem<uint8_t, S, kCaHalo, kUnit * 16>::BYTES;
        cudaError_t e = dyn_smem_grid(k, smem, (units + kUnitWarps - 1) / kUnitWarps, cfg, &grid,
                                      &occ, &attr);
        if (e != cudaSuccess) return e;
        k<<<grid, kUnitThreads, smem, st>>>(in, out, r, order, total);
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_diffuse_t(int r, int order, const float *in, float *out, float alpha,
                             cudaStream_t st, const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    const uint32_t total = (uint32_t)pow3i(r);
    const uint64_t units = (total + kUnit - 1) / kUnit;
    unsigned grid = 1;
    auto k = compact_diffuse_kernel<S>;
    constexpr int smem = StencilSmem<float, S, kDiffHalo, kUnit * 16>::BYTES;
    cudaError_t e = dyn_smem_grid(k, smem, (units + kUnitWarps - 1) / kUnitWarps, cfg, &grid,
                                  &occ, &attr);
    if (e != cudaSuccess) return e;
    k<<<grid, kUnitThreads, smem, st>>>(in, out, r, order, total, alpha);
    return cudaGetLastError();
}

#define SG_COMPACT_S_SWITCH(s, CALL)         \
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

}  // namespace

cudaError_t launch_compact_ca(int r, int s, int order, const uint8_t *in, uint8_t *out,
                              cudaStream_t st, const LaunchCfg &cfg)
{
#define CALL(S) launch_ca_t<S>(r, order, in, out, st, cfg)
    SG_COMPACT_S_SWITCH(s, CALL)
#undef CALL
}

cudaError_t launch_compact_diffuse(int r, int s, int order, const float *in, float *out,
                                   float alpha, cudaStream_t st, const LaunchCfg &cfg)
{
#define CALL(S) launch_diffuse_t<S>(r, order, in, out, alpha, st, cfg)
    SG_COMPACT_S_SWITCH(s, CALL)
#undef CALL
}

}  // namespace sg
