// sg_compact_io.cu -- moving between the embedded and the compact layout
// (pack, unpack) and the map-and-write pass on a compact array.
//
// Each warp of a persistent grid takes units of 729 elements (G whole tiles,
// layout in sg_compact.cuh) on its own: it decodes the unit's tiles with the
// lambda reduction of Theorem 1 into its own shared memory, then its lanes
// walk the unit's elements, 32 consecutive ones per step.  The compact side
// is therefore read or written in whole sectors; the embedded side is
// touched only at gasket cells, as the embedded write pass touches it.  The
// per-position table (tile within the unit, tile-relative coordinates) is
// expanded into shared memory once per CTA; after that barrier the warps
// never wait for one another.
#include "sg_compact.cuh"
#include "sg_stencil.cuh"

namespace sg {

namespace {

// Shared memory of a CTA: the unit table, then one region per warp.
template <int S> struct IoSmem {
    static constexpr int G = CompactPattern<S>::G;
    // every region starts on a 16-byte boundary (the per-warp arrays hold
    // 8-byte elements)
    static constexpr int TABLE = (kUnit * 4 + 15) / 16 * 16;     // unit_cell per position
    static constexpr int WARP = ((G * 8) + 15) / 16 * 16;        // per-tile words
    static constexpr int BYTES = TABLE + kUnitWarps * WARP;
    static_assert(TABLE % 16 == 0 && WARP % 16 == 0, "16-byte aligned regions");
};

template <int S>
__device__ __forceinline__ uint32_t *build_cell_table(unsigned char *smem)
{
    uint32_t *cells = reinterpret_cast<uint32_t *>(smem);
    for (int c = threadIdx.x; c < kUnit; c += kUnitThreads) cells[c] = unit_cell<S>(c);
    __syncthreads();
    return cells;
}

// MODE 0: pack (grid -> compact), 1: unpack (compact -> grid).
template <typename T, int S, int MODE>
__global__ void __launch_bounds__(kUnitThreads)
compact_move_kernel(const T *__restrict__ src, T *__restrict__ dst, int r, int order,
                    uint32_t total)
{
    using M = IoSmem<S>;
    constexpr int G = M::G;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t *cells = build_cell_table<S>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint2 *coord = reinterpret_cast<uint2 *>(smem + M::TABLE + warp * M::WARP);
    const int rb = r - S;
    const uint32_t ntiles = total / CompactPattern<S>::C, units = (total + kUnit - 1) / kUnit;
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        __syncwarp();                 // the previous unit's reads of coord are done
        decode_unit_tiles<G>(coord, u * G, ntiles, W, ll);
        __syncwarp();
        const uint32_t base = u * kUnit;
        const uint32_t cnt = min((uint32_t)kUnit, total - base);
#pragma unroll 4
        for (uint32_t c = lane; c < cnt; c += 32) {
            const uint32_t cell = cells[c];
            const uint2 b = coord[cell & 0x3FFu];
            const uint32_t x = (b.x << S) | ((cell >> 10) & 0x3Fu);
            const uint32_t y = (b.y << S) | (cell >> 16);
            const uint64_t at = ((uint64_t)y << r) | x;
            if constexpr (MODE == 0) dst[base + c] = src[at];
            else dst[at] = src[base + c];
        }
    }
}

// Byte offset of the per-warp staging buffers of the write kernel, and their
// size: a unit's values plus room to align them like their destination.
template <int S> __host__ __device__ constexpr int write_stage_offset()
{
    return IoSmem<S>::BYTES + ((kUnit * 2 + 15) / 16) * 16;
}
template <typename T> __host__ __device__ constexpr int write_stage_bytes()
{
    return (kUnit * (int)sizeof(T) + 16 + 15) / 16 * 16;
}

// WIDE: stage each unit in shared memory and store it in whole aligned
// 16-byte chunks (for a destination in host memory, across the host link);
// otherwise every lane stores its values directly (device memory, where the
// staging's extra registers cost more than the wide stores save).
template <typename T, int VK, int S, bool WIDE>
__global__ void __launch_bounds__(kUnitThreads)
compact_write_kernel(T *__restrict__ compact, int r, int order, uint32_t total, uint64_t vs)
{
    using M = IoSmem<S>;
    constexpr int G = M::G;
    constexpr int STAGE = write_stage_bytes<T>();
    extern __shared__ __align__(16) unsigned char smem[];
    // per position: the value-key offset of the cell within its tile (the
    // same in every tile), and the tile within the unit
    uint32_t *koff = reinterpret_cast<uint32_t *>(smem);
    for (int c = threadIdx.x; c < kUnit; c += kUnitThreads) {
        const uint32_t cell = unit_cell<S>(c);
        koff[c] = CellValue<T, VK>::offset_of((cell >> 10) & 0x3Fu, cell >> 16, r);
    }
    uint16_t *tile_of = reinterpret_cast<uint16_t *>(smem + M::BYTES);
    for (int c = threadIdx.x; c < kUnit; c += kUnitThreads)
        tile_of[c] = (uint16_t)(c / CompactPattern<S>::C);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *vbase = reinterpret_cast<uint32_t *>(smem + M::TABLE + warp * M::WARP);
    unsigned char *stage = smem + write_stage_offset<S>() + warp * STAGE;
    const int rb = r - S;
    const uint32_t ntiles = total / CompactPattern<S>::C, units = (total + kUnit - 1) / kUnit;
    const CellValue<T, VK> cv{vs * kGoldenGamma, (uint32_t)vs};
    LambdaLane ll;
    ll.init(lane, rb, order);
    const uint32_t W = pi_word(order, rb);
    const uint32_t nwarps = gridDim.x * kUnitWarps;
    for (uint32_t u = blockIdx.x * kUnitWarps + warp; u < units; u += nwarps) {
        __syncwarp();
        for (int g = 0; g < G; ++g) {
            const uint32_t q = u * G + (uint32_t)g;
            if (q < ntiles) {
                const uint32_t bq = q / W, aq = q - bq * W;
                const uint2 b = ll.decode(aq, bq);
                if (lane == 0) vbase[g] = CellValue<T, VK>::base_of(b.x << S, b.y << S, r);
            }
        }
        __syncwarp();
        const uint32_t base = u * kUnit;
        const uint32_t cnt = min((uint32_t)kUnit, total - base);
        if constexpr (!WIDE) {
            T *dst = compact + base;
#pragma unroll 4
            for (uint32_t c = lane; c < cnt; c += 32) {
                const uint32_t vb = G == 1 ? vbase[0] : vbase[tile_of[c]];
                dst[c] = cv(vb, koff[c]);
            }
            continue;
        }
        // the values go to shared memory at the destination's offset within
        // 16 bytes, then out as whole aligned 16-byte chunks (byte stores
        // only for the unit's ragged ends)
        unsigned char *out = reinterpret_cast<unsigned char *>(compact + base);
        const uint32_t lead = (uint32_t)(reinterpret_cast<uintptr_t>(out) & 15u);
        T *sv = reinterpret_cast<T *>(stage + lead);
#pragma unroll 4
        for (uint32_t c = lane; c < cnt; c += 32) {
            const uint32_t vb = G == 1 ? vbase[0] : vbase[tile_of[c]];
            sv[c] = cv(vb, koff[c]);
        }
        __syncwarp();
        const uint32_t nb = cnt * (uint32_t)sizeof(T);
        const uint32_t head = min((16u - lead) & 15u, nb);
        const uint32_t chunks = (nb - head) / 16u, body_end = head + 16u * chunks;
        for (uint32_t i = lane; i < head; i += 32) out[i] = stage[lead + i];
        for (uint32_t k = lane; k < chunks; k += 32)
            *reinterpret_cast<uint4 *>(out + head + 16u * k) =
                *reinterpret_cast<const uint4 *>(stage + lead + head + 16u * k);
        for (uint32_t i = body_end + lane; i < nb; i += 32) out[i] = stage[lead + i];
    }
}

template <typename T, int S, bool WIDE> constexpr int write_smem_bytes()
{
    return write_stage_offset<S>() + (WIDE ? kUnitWarps * write_stage_bytes<T>() : 0);
}

template <typename T, int S, int MODE>
cudaError_t launch_move_t(int r, int order, const T *src, T *dst, cudaStream_t st,
                          const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    const uint32_t total = (uint32_t)pow3i(r);
    const uint64_t units = (total + kUnit - 1) / kUnit;
    unsigned grid = 1;
    auto k = compact_move_kernel<T, S, MODE>;
    constexpr int smem = IoSmem<S>::BYTES;
    cudaError_t e = dyn_smem_grid(k, smem, (units + kUnitWarps - 1) / kUnitWarps, cfg, &grid,
                                  &occ, &attr);
    if (e != cudaSuccess) return e;
    k<<<grid, kUnitThreads, smem, st>>>(src, dst, r, order, total);
    return cudaGetLastError();
}

template <typename T, int VK, int S, bool WIDE>
cudaError_t launch_write_t(int r, int order, T *compact, uint64_t vs, cudaStream_t st,
                           const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    static std::atomic<uint64_t> attr{0};
    const uint32_t total = (uint32_t)pow3i(r);
    const uint64_t units = (total + kUnit - 1) / kUnit;
    unsigned grid = 1;
    auto k = compact_write_kernel<T, VK, S, WIDE>;
    constexpr int smem = write_smem_bytes<T, S, WIDE>();
    cudaError_t e = dyn_smem_grid(k, smem, (units + kUnitWarps - 1) / kUnitWarps, cfg, &grid,
                                  &occ, &attr);
    if (e != cudaSuccess) return e;
    k<<<grid, kUnitThreads, smem, st>>>(compact, r, order, total, vs);
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

template <typename T, int MODE>
cudaError_t launch_move(int r, int s, int order, const T *src, T *dst, cudaStream_t st,
                        const LaunchCfg &cfg)
{
#define CALL(S) launch_move_t<T, S, MODE>(r, order, src, dst, st, cfg)
    SG_COMPACT_S_SWITCH(s, CALL)
#undef CALL
}

template <typename T, int VK, bool WIDE>
cudaError_t launch_write_vk(int r, int s, int order, T *compact, uint64_t vs, cudaStream_t st,
                            const LaunchCfg &cfg)
{
#define CALL(S) launch_write_t<T, VK, S, WIDE>(r, order, compact, vs, st, cfg)
    SG_COMPACT_S_SWITCH(s, CALL)
#undef CALL
}

template <typename T, bool WIDE>
cudaError_t launch_write_dt(int r, int s, int order, int vk, T *compact, uint64_t vs,
                            cudaStream_t st, const LaunchCfg &cfg)
{
    switch (vk) {
    case kValConst: return launch_write_vk<T, kValConst, WIDE>(r, s, order, compact, vs, st, cfg);
    case kValLinear31:
        return launch_write_vk<T, kValLinear31, WIDE>(r, s, order, compact, vs, st, cfg);
    case kValHash: return launch_write_vk<T, kValHash, WIDE>(r, s, order, compact, vs, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_compact_pack(int r, int s, int order, int elem, const void *grid,
                                void *compact, cudaStream_t st, const LaunchCfg &cfg)
{
    if (elem == 1)
        return launch_move<uint8_t, 0>(r, s, order, (const uint8_t *)grid, (uint8_t *)compact,
                                       st, cfg);
    return launch_move<float, 0>(r, s, order, (const float *)grid, (float *)compact, st, cfg);
}

cudaError_t launch_compact_unpack(int r, int s, int order, int elem, const void *compact,
                                  void *grid, cudaStream_t st, const LaunchCfg &cfg)
{
    if (elem == 1)
        return launch_move<uint8_t, 1>(r, s, order, (const uint8_t *)compact, (uint8_t *)grid,
                                       st, cfg);
    return launch_move<float, 1>(r, s, order, (const float *)compact, (float *)grid, st, cfg);
}

cudaError_t launch_compact_write(int r, int s, int order, int elem, int vk, void *compact,
                                 uint64_t vs, cudaStream_t st, const LaunchCfg &cfg, bool wide)
{
    if (elem == 1)
        return wide ? launch_write_dt<uint8_t, true>(r, s, order, vk, (uint8_t *)compact, vs, st, cfg)
                    : launch_write_dt<uint8_t, false>(r, s, order, vk, (uint8_t *)compact, vs, st,
                                                      cfg);
    return wide ? launch_write_dt<float, true>(r, s, order, vk, (float *)compact, vs, st, cfg)
                : launch_write_dt<float, false>(r, s, order, vk, (float *)compact, vs, st, cfg);
}

}  // namespace sg
