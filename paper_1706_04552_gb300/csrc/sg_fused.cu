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
// The CA runs bit-sliced (one warp per tile, 32 cells per word operation);
// diffusion runs on float4 chunks with the single-step kernels' diffuse_cell
// (one CTA per tile).  Either way each cell's result is the single step's, so
// k fused steps equal k single steps.  HBM moves about the tile bytes once in
// and once out per launch instead of per step.
//
// The tile coordinate comes from the lambda(omega) decode of Theorem 1 (one
// warp, redux.sync) or from the bounding-box identity map, as elsewhere.
#include "sg_bits.cuh"
#include "sg_stencil.cuh"

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
cudaError_t launch_diffuse_fused_t(int r, const float *in, float *out, float alpha, int k,
                                   cudaStream_t st, const LaunchCfg &cfg)
{
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
