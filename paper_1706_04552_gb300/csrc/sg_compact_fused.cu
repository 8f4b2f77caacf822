// sg_compact_fused.cu -- k B3/S23 steps per launch on a compact array of
// 64-tiles (layout in sg_compact.cuh), k <= SG_FUSE_MAX.
//
// One warp takes one tile at a time and runs the bit-sliced k-step routine
// of the embedded fused CA (bits_ca_step in sg_bits.cuh) on it: rows of
// bits with a halo of KH rows above and below and 16 columns either side.
// What differs is the staging.  The halo cells live in the compact runs of
// the neighbouring tiles, and a KH-step light cone reaches only part of
// them: the rows 64-KH .. 63 of the tiles above, the rows 0 .. KH-1 of the
// tiles below, and of the tile to the left only its rows 0 .. 15 (its
// columns 48 .. 63 hold gasket cells nowhere else).  Those runs are read as
// whole sectors and packed to bits by ballots; each staged 16-column chunk
// then takes its cells from them (a chunk's cells are consecutive in compact
// order) and spreads them onto its columns through the row codec.  The tile
// rows are gathered back to compact order at the end.
#include "sg_bits.cuh"
#include "sg_compact.cuh"

namespace sg {

namespace {

// The neighbour tiles s = 0 .. 8, (dtx, dty) = (s % 3 - 1, s / 3 - 1), and
// the compact elements [lo[s], hi[s]) of each that a KH-step light cone
// reaches; staged as bits from word word[s] on, each run padded to whole
// words.
template <int KH> struct HaloRuns {
    uint16_t lo[9], hi[9], word[9];
    int words;
};

template <int KH> constexpr HaloRuns<KH> make_halo_runs()
{
    const RowCodec rc = make_row_codec();
    auto start = [&](int y) { return y >= 64 ? kUnit : (int)rc.row_start[y]; };
    HaloRuns<KH> h{};
    int w = 0;
    for (int s = 0; s < 9; ++s) {
        const int dtx = s % 3 - 1, dty = s / 3 - 1;
        int y0 = dty < 0 ? 64 - KH : 0, y1 = dty > 0 ? KH : 64;
        if (dtx < 0 && y1 > 16) y1 = 16;       // left: columns 48..63 only in rows 0..15
        if (y1 < y0) y1 = y0;
        h.lo[s] = (uint16_t)start(y0);
        h.hi[s] = (uint16_t)start(y1);
        h.word[s] = (uint16_t)w;
        w += (h.hi[s] - h.lo[s] + 31) / 32;
    }
    h.words = w;
    return h;
}

template <int KH> struct HaloRunWords {
    static constexpr int value = make_halo_runs<KH>().words;
};

__device__ const HaloRuns<4> kHaloRuns4 = make_halo_runs<4>();
__device__ const HaloRuns<8> kHaloRuns8 = make_halo_runs<8>();
__device__ const HaloRuns<16> kHaloRuns16 = make_halo_runs<16>();

template <int KH> __device__ __forceinline__ const HaloRuns<KH> &halo_runs()
{
    if constexpr (KH == 4) return kHaloRuns4;
    else if constexpr (KH == 8) return kHaloRuns8;
    else return kHaloRuns16;
}

template <int KH>
__global__ void __launch_bounds__(kUnitThreads, 6)
compact_ca_fused_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int r,
                        int order, uint32_t total, int k)
{
    constexpr int S = 6;
    using B = BitShape<S, KH>;
    constexpr int HPR = 2 * B::WPR;
    constexpr int RUN_WORDS = HaloRunWords<KH>::value;
    constexpr int OUT_WORDS = (kUnit + 31) / 32;
    __shared__ RowCodec tc;
    __shared__ uint32_t sm[kUnitWarps][3][B::BUFW];           // two states and the mask
    __shared__ uint32_t runs[kUnitWarps][RUN_WORDS + 2];      // + guard words
    __shared__ uint32_t obits[kUnitWarps][OUT_WORDS + 3];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&kRowCodec);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&tc);
        for (int i = threadIdx.x; i < (int)(sizeof(RowCodec) / 4); i += kUnitThreads)
            dst[i] = src[i];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *st0 = sm[warp][0] + 1, *st1 = sm[warp][1] + 1, *mk = sm[warp][2] + 1;
    uint32_t *cb = runs[warp], *ob = obits[warp];
    if (lane < 2) cb[RUN_WORDS + lane] = 0u;
    __syncthreads();

    const HaloRuns<KH> &hr = halo_runs<KH>();
    const int rb = r - S;
    const int n = 1 << r;
    const uint32_t units = total / kUnit;                     // whole tiles: r >= 6
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        const uint32_t bq = u / W, aq = u - bq * W;
        const uint2 b = ll.decode(aq, bq);
        // launch index of neighbour tile `lane` (lanes 0..8), ~0u if it has
        // no gasket cell or lies outside the grid
        uint32_t nq = ~0u;
        if (lane < 9) {
            const uint32_t nbx = b.x + (uint32_t)(lane % 3 - 1), nby = b.y + (uint32_t)(lane / 3 - 1);
            if ((nbx >> rb) == 0u && (nby >> rb) == 0u && (nbx & nby) == 0u)
                nq = lambda_index(nbx, nby, rb, order);
        }
        __syncwarp();                  // the previous tile is finished with the buffers
        // 1. the runs as bits (whole sectors, then ballots)
        for (int s = 0; s < 9; ++s) {
            const uint32_t q = __shfl_sync(0xffffffffu, nq, s);
            const int lo = hr.lo[s], hi = hr.hi[s], w0 = hr.word[s];
            for (int e = lo; e < hi; e += 32) {
                const int c = e + lane;
                const uint8_t v = (q != ~0u && c < hi) ? in[(uint64_t)q * kUnit + c] : 0;
                const uint32_t w = __ballot_sync(0xffffffffu, v != 0);
                if (lane == 0) cb[w0 + (e - lo) / 32] = w;
            }
        }
        __syncwarp();
        // 2. staged rows: each 16-column chunk from its tile's run
        const int x0 = (int)(b.x << S), y0 = (int)(b.y << S);
        uint16_t *bh = reinterpret_cast<uint16_t *>(st0);
        uint16_t *mh = reinterpret_cast<uint16_t *>(mk);
        for (int i = lane; i < B::ROWS * HPR; i += 32) {
            const int row = i / HPR, h = i - row * HPR;
            const int x = x0 - 16 + 16 * h, y = y0 - KH + row;
            uint32_t v = 0u, m = 0u;
            if (h < B::HW && x >= 0 && y >= 0 && x < n && y < n && (x & y) == 0) {
                const int s = ((y >> S) - y0 / 64 + 1) * 3 + ((x >> S) - x0 / 64 + 1);
                const uint32_t lx = (uint32_t)x & 63u, ly = (uint32_t)y & 63u;
                const uint32_t cx = lx >> 4, n16 = 16u >> __popc(ly & 15u);
                const uint32_t rank = __popc(member_bits4(ly >> 4) & ((1u << cx) - 1u));
                const uint32_t e = tc.row_start[ly] + rank * n16;
                const uint32_t o = (uint32_t)hr.word[s] * 32u + (e - hr.lo[s]);
                const uint32_t bits = __funnelshift_r(cb[o >> 5], cb[(o >> 5) + 1], o & 31u);
                const uint32_t yl = ly & 7u, n8 = 8u >> __popc(yl), m8 = (1u << n8) - 1u;
                v = tc.dep[yl][bits & m8];
                if ((ly & 8u) == 0u) v |= (uint32_t)tc.dep[yl][(bits >> n8) & m8] << 8;
                m = member_bits16(ly & 15u);
            }
            bh[i] = (uint16_t)v;
            mh[i] = (uint16_t)m;
        }
        if (lane < OUT_WORDS + 3) ob[lane] = 0u;
        __syncwarp();
        // 3. k steps in shared memory
        for (int step = 1; step <= k; ++step) {
            bits_ca_step<S, KH>((step & 1) ? st0 : st1, (step & 1) ? st1 : st0, mk, step, lane);
            __syncwarp();
        }
        // 4. tile rows back to compact order, then bytes
        const uint32_t *fin = (k & 1) ? st1 : st0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint32_t ty = 2u * lane + j;
            const uint32_t *p = fin + (KH + ty) * B::WPR;   // columns -16 .. 79
            const uint64_t row = (uint64_t)__funnelshift_r(p[0], p[1], 16) |
                                 ((uint64_t)__funnelshift_r(p[1], p[2], 16) << 32);
            or_bits_at(ob, tc.row_start[ty], gather_row(tc, row, ty));
        }
        __syncwarp();
        const uint32_t base = u * kUnit;
#pragma unroll
        for (int it = 0; it < OUT_WORDS; ++it) {
            const int c = 32 * it + lane;
            if (c < kUnit) out[base + c] = (uint8_t)((ob[it] >> lane) & 1u);
        }
    }
}

template <int KH>
cudaError_t launch_fused_t(int r, int order, const uint8_t *in, uint8_t *out, int k,
                           cudaStream_t st, const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    const uint32_t total = (uint32_t)pow3i(r);
    const uint64_t units = total / kUnit;
    unsigned grid = 1;
    auto kern = compact_ca_fused_kernel<KH>;
    cudaError_t e = persistent_grid(kern, kUnitThreads, 0, (units + kUnitWarps - 1) / kUnitWarps,
                                    cfg, &grid, &occ);
    if (e != cudaSuccess) return e;
    kern<<<grid, kUnitThreads, 0, st>>>(in, out, r, order, total, k);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_compact_ca_fused(int r, int order, const uint8_t *in, uint8_t *out, int k,
                                    cudaStream_t st, const LaunchCfg &cfg)
{
    if (k <= 4) return launch_fused_t<4>(r, order, in, out, k, st, cfg);
    if (k <= 8) return launch_fused_t<8>(r, order, in, out, k, st, cfg);
    return launch_fused_t<16>(r, order, in, out, k, st, cfg);
}

}  // namespace sg
