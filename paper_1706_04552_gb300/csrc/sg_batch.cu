// sg_batch.cu -- many gaskets of uneven levels stepped by one launch.
//
// A batch is a list of gaskets, each with its own level r_i and its own pair
// of uint8 state buffers.  Instead of one grid per gasket, a step launches
// one persistent grid over a single work list: the concatenation of every
// gasket's lambda block space (3^(r_i - s) tiles each), indexed through a
// prefix sum.  A CTA takes a group of consecutive work items, finds each
// item's gasket by binary search in the prefix sum, decodes the item's tile
// with lambda at that gasket's level, and runs the CA tile step shared with
// the single-gasket kernel.  The step sequence can be captured once in a
// CUDA graph; an autotuner picks rho, the walking order and CTAs per SM.
//
// Workspace (caller-owned device memory, sg_batch_workspace_bytes(count)):
//   uint32 prefix[count + 1]   first work item of gasket i (prefix[count] = total)
//   int32  level[count]      bits 0..7 the level; bits 8..15 the gasket's own
//                            step count in a fused launch (0: the launch's k)
//   uint64 buf_a[count], buf_b[count]   state buffers (parity 0 reads a, writes b)
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sg.h"
#include "sg_sched.h"
#include "sg_bits.cuh"
#include "sg_stencil.cuh"

namespace sg {

namespace {

constexpr int kMaxBatch = 65535;

uint64_t align16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

struct WsLayout {
    uint64_t prefix, level, a, b, total;
};

WsLayout ws_layout(int count)
{
    WsLayout L;
    L.prefix = 0;
    L.level = align16(L.prefix + 4ull * (count + 1));
    L.a = align16(L.level + 4ull * count);
    L.b = L.a + 8ull * count;
    L.total = align16(L.b + 8ull * count);
    return L;
}

struct BatchView {
    const uint32_t *prefix;
    const int32_t *level;
    const uint64_t *buf_a;
    const uint64_t *buf_b;
    uint32_t count;
};

BatchView view_of(const sg_batch_plan *p)
{
    const WsLayout L = ws_layout(p->count);
    const char *ws = static_cast<const char *>(p->workspace);
    return BatchView{reinterpret_cast<const uint32_t *>(ws + L.prefix),
                     reinterpret_cast<const int32_t *>(ws + L.level),
                     reinterpret_cast<const uint64_t *>(ws + L.a),
                     reinterpret_cast<const uint64_t *>(ws + L.b), (uint32_t)p->count};
}

// Gasket that work item q belongs to: the largest i with prefix[i] <= q.
__device__ __forceinline__ uint32_t batch_instance(const uint32_t *prefix, uint32_t count,
                                                   uint32_t q)
{
    uint32_t lo = 0, hi = count;           // prefix[lo] <= q < prefix[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= q) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int S>
__global__ void __launch_bounds__(kStencilThreads)
ca_batch_kernel(BatchView bv, uint32_t total, int parity, int order)
{
    using G = StencilGroup<uint8_t, S>;
    __shared__ __align__(16) uint8_t sm[2 * G::TPC * G::TILE];
    __shared__ StencilTile<uint8_t> tiles[2 * G::TPC];

    LambdaLane ll;
    ll.init(threadIdx.x & 31, 0, order);
    const uint32_t groups = (total + G::TPC - 1) / G::TPC;
    auto decode = [&](uint64_t g, StencilTile<uint8_t> *dst) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int t = warp; t < G::TPC; t += kStencilThreads / 32) {
            const uint32_t q = (uint32_t)g * G::TPC + (uint32_t)t;
            StencilTile<uint8_t> tl{kNoTile, kNoTile, 0, nullptr, nullptr};
            if (q < total) {                                  // warp-uniform
                const uint32_t i = batch_instance(bv.prefix, bv.count, q);
                const int r = __ldg(bv.level + i) & 0xFF;
                const int rb = r - S;
                const uint32_t local = q - __ldg(bv.prefix + i);
                ll.set_level(lane, rb);
                const uint32_t W = pi_word(order, rb);
                const uint32_t b = local / W, a = local - b * W;
                const uint2 c = ll.decode(a, b);
                const uint64_t pa = __ldg(bv.buf_a + i), pb = __ldg(bv.buf_b + i);
                tl = StencilTile<uint8_t>{c.x, c.y, r,
                                          reinterpret_cast<const uint8_t *>(parity ? pb : pa),
                                          reinterpret_cast<uint8_t *>(parity ? pa : pb)};
            }
            if (lane == 0) dst[t] = tl;
        }
    };
    auto compute = [](const uint8_t *buf, const StencilTile<uint8_t> *slot) {
        ca_compute_group<S>(buf, slot);
    };
    stencil_pipeline<uint8_t, S>(sm, tiles, groups, decode, compute);
}

// One step with one warp per work item (rho = 32, 64): the item's tile is
// staged and computed by the warp alone, as in the single-gasket kernel.
template <int S>
__global__ void __launch_bounds__(kStencilThreads)
ca_batch_warp_kernel(BatchView bv, uint32_t total, int parity, int order)
{
    using G = StencilGroup<uint8_t, S>;
    extern __shared__ __align__(16) unsigned char warp_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *sm = warp_smem + warp * G::TILE;
    LambdaLane ll;
    ll.init(lane, 0, order);
    const uint64_t stride = (uint64_t)gridDim.x * kWarpTileWarps;
    for (uint64_t q = (uint64_t)blockIdx.x * kWarpTileWarps + warp; q < total; q += stride) {
        const uint32_t i = batch_instance(bv.prefix, bv.count, (uint32_t)q);   // warp-uniform
        const int r = __ldg(bv.level + i) & 0xFF, rb = r - S;
        const uint32_t local = (uint32_t)q - __ldg(bv.prefix + i);
        ll.set_level(lane, rb);
        const uint32_t W = pi_word(order, rb);
        const uint32_t b = local / W, a = local - b * W;
        const uint2 c = ll.decode(a, b);
        const uint64_t pa = __ldg(bv.buf_a + i), pb = __ldg(bv.buf_b + i);
        const uint8_t *in = reinterpret_cast<const uint8_t *>(parity ? pb : pa);
        uint8_t *out = reinterpret_cast<uint8_t *>(parity ? pa : pb);
        warp_stage<uint8_t, S>(sm, in, r, (int)(c.x << S), (int)(c.y << S), lane);
        const StencilTile<uint8_t> tl{c.x, c.y, r, in, out};
        for (int k = lane; k < G::CHUNKS; k += 32) ca_chunk<S>(sm, tl, 0, k);
        __syncwarp();                    // the tile is read before the next staging
    }
}

template <int S>
cudaError_t launch_batch_t(const sg_batch_plan *p, int parity, cudaStream_t st,
                           const LaunchCfg &cfg)
{
    static std::atomic<int> occ{0};
    unsigned grid = 1;
    cudaError_t e;
    if constexpr (S >= 5) {
        static std::atomic<uint64_t> attr{0};
        auto k = ca_batch_warp_kernel<S>;
        constexpr int smem = kWarpTileWarps * StencilGroup<uint8_t, S>::TILE;
        e = dyn_smem_grid(k, smem, ((uint64_t)p->total_tiles + kWarpTileWarps - 1) / kWarpTileWarps,
                          cfg, &grid, &occ, &attr);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, smem, st>>>(view_of(p), p->total_tiles, parity, cfg.order);
    } else {
        constexpr int TPC = StencilGroup<uint8_t, S>::TPC;
        const uint64_t groups = (p->total_tiles + TPC - 1) / TPC;
        auto k = ca_batch_kernel<S>;
        e = persistent_grid(k, kStencilThreads, 0, groups, cfg, &grid, &occ);
        if (e != cudaSuccess) return e;
        k<<<grid, kStencilThreads, 0, st>>>(view_of(p), p->total_tiles, parity, cfg.order);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch(const sg_batch_plan *p, int parity, cudaStream_t st,
                         const LaunchCfg &cfg)
{
    switch (p->rho) {
    case 16: return launch_batch_t<4>(p, parity, st, cfg);
    case 32: return launch_batch_t<5>(p, parity, st, cfg);
    case 64: return launch_batch_t<6>(p, parity, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

// k fused steps of every gasket of the batch, bit-sliced (sg_bits.cuh): a
// warp takes one work item at a time, finds its gasket, decodes its tile at
// that gasket's level and runs the k steps of the tile in shared memory.
template <int S, int KH>
__global__ void __launch_bounds__(kStencilThreads, 6)
ca_batch_bits_kernel(BatchView bv, uint32_t total, int parity, int order, int k)
{
    using B = BitShape<S, KH>;
    __shared__ uint32_t sm[B::WARPS][3][B::BUFW];      // two states and the mask, per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *st0 = sm[warp][0] + 1, *st1 = sm[warp][1] + 1, *mk = sm[warp][2] + 1;
    LambdaLane ll;
    ll.init(lane, 0, order);
    const uint64_t stride = (uint64_t)gridDim.x * B::WARPS;
    for (uint64_t q = (uint64_t)blockIdx.x * B::WARPS + warp; q < total; q += stride) {
        const uint32_t i = batch_instance(bv.prefix, bv.count, (uint32_t)q);   // warp-uniform
        const int lv = __ldg(bv.level + i);
        const int r = lv & 0xFF, rb = r - S;
        const int kk = (lv >> 8) ? (lv >> 8) : k;            // the gasket's own steps, <= KH
        const uint32_t local = (uint32_t)q - __ldg(bv.prefix + i);
        ll.set_level(lane, rb);
        const uint32_t W = pi_word(order, rb);
        const uint32_t b = local / W, a = local - b * W;
        const uint2 c = ll.decode(a, b);
        const uint64_t pa = __ldg(bv.buf_a + i), pb = __ldg(bv.buf_b + i);
        bits_tile_steps<S, KH>(st0, st1, mk, reinterpret_cast<const uint8_t *>(parity ? pb : pa),
                               reinterpret_cast<uint8_t *>(parity ? pa : pb), r,
                               (int)(c.x << S), (int)(c.y << S), kk, lane);
    }
}

template <int S, int KH>
cudaError_t launch_batch_fused_t(const sg_batch_plan *p, int parity, int k, cudaStream_t st,
                                 const LaunchCfg &cfg)
{
    using B = BitShape<S, KH>;
    static std::atomic<int> occ{0};
    unsigned grid = 1;
    auto kern = ca_batch_bits_kernel<S, KH>;
    cudaError_t e = persistent_grid(kern, kStencilThreads, 0,
                                    ((uint64_t)p->total_tiles + B::WARPS - 1) / B::WARPS, cfg,
                                    &grid, &occ);
    if (e != cudaSuccess) return e;
    kern<<<grid, kStencilThreads, 0, st>>>(view_of(p), p->total_tiles, parity, cfg.order, k);
    return cudaGetLastError();
}

// k steps (1 <= k <= SG_FUSE_MAX) of every gasket: one launch.
cudaError_t launch_batch_k(const sg_batch_plan *p, int parity, int k, cudaStream_t st,
                           const LaunchCfg &cfg)
{
    if (k == 1) return launch_batch(p, parity, st, cfg);
    if (k < 1 || k > SG_FUSE_MAX) return cudaErrorInvalidValue;
    const int kh = k <= 4 ? 4 : k <= 8 ? 8 : 16;
    switch (p->rho * 100 + kh) {
    case 1604: return launch_batch_fused_t<4, 4>(p, parity, k, st, cfg);
    case 1608: return launch_batch_fused_t<4, 8>(p, parity, k, st, cfg);
    case 1616: return launch_batch_fused_t<4, 16>(p, parity, k, st, cfg);
    case 3204: return launch_batch_fused_t<5, 4>(p, parity, k, st, cfg);
    case 3208: return launch_batch_fused_t<5, 8>(p, parity, k, st, cfg);
    case 3216: return launch_batch_fused_t<5, 16>(p, parity, k, st, cfg);
    case 6404: return launch_batch_fused_t<6, 4>(p, parity, k, st, cfg);
    case 6408: return launch_batch_fused_t<6, 8>(p, parity, k, st, cfg);
    case 6416: return launch_batch_fused_t<6, 16>(p, parity, k, st, cfg);
    default: return cudaErrorInvalidValue;
    }
}

bool plan_ok(const sg_batch_plan *p)
{
    return p != nullptr && p->workspace != nullptr && p->count >= 1 && p->count <= kMaxBatch &&
           (p->rho == 16 || p->rho == 32 || p->rho == 64) && p->total_tiles > 0 &&
           p->reserved[0] >= 0 && p->reserved[0] <= SG_FUSE_MAX;
}

sg_status cuda_fail(cudaError_t e) { return set_last_cuda_error(e); }

// Autotuner results, keyed by the multiset of levels (host memory only).
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune_cache;

}  // namespace

}  // namespace sg

using namespace sg;

extern "C" {

uint64_t sg_batch_workspace_bytes(int count)
{
    if (count < 1 || count > kMaxBatch) return 0;
    return ws_layout(count).total;
}

sg_status sg_batch_ca_plan_host(int count, const int *levels, const int *steps,
                                uint8_t *const *buf_a, uint8_t *const *buf_b, int rho,
                                void *host_image, uint64_t image_bytes, void *workspace,
                                uint64_t workspace_bytes, sg_batch_plan *plan)
{
    if (plan == nullptr || levels == nullptr || buf_a == nullptr || buf_b == nullptr ||
        host_image == nullptr)
        return SG_EINVAL;
    if (count < 1 || count > kMaxBatch) return SG_EINVAL;
    if (rho != 16 && rho != 32 && rho != 64) return SG_EUNSUPPORTED;
    if (workspace == nullptr || ((uintptr_t)workspace & 15) != 0) return SG_EINVAL;
    const WsLayout L = ws_layout(count);
    if (workspace_bytes < L.total || image_bytes < L.total) return SG_EINVAL;
    int s = 0;
    while ((1 << s) < rho) ++s;
    // validate everything before the image is touched
    uint64_t total = 0;
    int max_level = 0, max_steps = 0;
    for (int i = 0; i < count; ++i) {
        const int r = levels[i];
        if (r < s || r > 16) return SG_EINVAL;        // every gasket holds whole tiles
        if (steps != nullptr && (steps[i] < 1 || steps[i] > SG_FUSE_MAX)) return SG_EINVAL;
        if (buf_a[i] == nullptr || buf_b[i] == nullptr || buf_a[i] == buf_b[i]) return SG_EINVAL;
        if (((uintptr_t)buf_a[i] & 15) || ((uintptr_t)buf_b[i] & 15)) return SG_EINVAL;
        total += (uint64_t)pow3i(r - s);
        max_level = std::max(max_level, r);
        if (steps != nullptr) max_steps = std::max(max_steps, steps[i]);
        if (total >= (1ull << 32)) return SG_EINVAL;
    }
    unsigned char *img = static_cast<unsigned char *>(host_image);
    std::memset(img, 0, L.total);
    uint32_t run = 0;
    for (int i = 0; i < count; ++i) {
        std::memcpy(img + L.prefix + 4ull * i, &run, 4);
        run += (uint32_t)pow3i(levels[i] - s);
        const uint64_t pa = (uint64_t)(uintptr_t)buf_a[i], pb = (uint64_t)(uintptr_t)buf_b[i];
        std::memcpy(img + L.a + 8ull * i, &pa, 8);
        std::memcpy(img + L.b + 8ull * i, &pb, 8);
    }
    std::memcpy(img + L.prefix + 4ull * count, &run, 4);
    for (int i = 0; i < count; ++i) {
        const int32_t lv = levels[i] | (steps != nullptr ? steps[i] << 8 : 0);
        std::memcpy(img + L.level + 4ull * i, &lv, 4);
    }
    *plan = sg_batch_plan{};
    plan->workspace = workspace;
    plan->workspace_bytes = workspace_bytes;
    plan->count = count;
    plan->rho = rho;
    plan->total_tiles = (uint32_t)total;
    plan->max_level = (uint32_t)max_level;
    plan->reserved[0] = max_steps;                    // launches need k >= every gasket's steps
    return SG_OK;
}

sg_status sg_batch_ca_plan(int count, const int *levels, uint8_t *const *buf_a,
                           uint8_t *const *buf_b, int rho, void *workspace,
                           uint64_t workspace_bytes, sg_batch_plan *plan, void *stream)
{
    if (count < 1 || count > kMaxBatch) return SG_EINVAL;
    // host image of the workspace, copied in one transfer (pageable memory:
    // the call returns once the bytes are staged, so the vector may go)
    const WsLayout L = ws_layout(count);
    std::vector<unsigned char> img(L.total);
    sg_batch_plan p;
    const sg_status st = sg_batch_ca_plan_host(count, levels, nullptr, buf_a, buf_b, rho,
                                               img.data(), L.total, workspace, workspace_bytes,
                                               &p);
    if (st != SG_OK) return st;
    cudaError_t e = cudaMemcpyAsync(workspace, img.data(), L.total, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *plan = p;
    return SG_OK;
}

sg_status sg_batch_ca_step(const sg_batch_plan *plan, int parity, const sg_launch_opts *opts,
                           void *stream)
{
    if (!plan_ok(plan) || (parity != 0 && parity != 1) || plan->reserved[0] > 1) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    const cudaError_t e = launch_batch(plan, parity, (cudaStream_t)stream, cfg);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}

}  // extern "C"

namespace sg {
namespace {

// Capture `steps` steps as launches of k fused steps (the last one takes
// the remainder), parities alternating from start_parity, into a graph.
sg_status capture_batch(const sg_batch_plan *plan, int steps, int k, int start_parity,
                        const sg_launch_opts *opts, void **graph)
{
    if (!plan_ok(plan) || graph == nullptr || steps < 1 || steps > 1000000 ||
        k < 1 || k > SG_FUSE_MAX || (start_parity != 0 && start_parity != 1) ||
        plan->reserved[0] != 0)                       // per-gasket step counts: not captured
        return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    *graph = nullptr;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        int parity = start_parity;
        for (int done = 0; done < steps && le == cudaSuccess; parity ^= 1) {
            const int kk = std::min(k, steps - done);
            le = launch_batch_k(plan, parity, kk, cs, cfg);
            done += kk;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) {
            cudaGraphExec_t x = nullptr;
            e = cudaGraphInstantiate(&x, g, 0);
            if (e == cudaSuccess) *graph = x;
        }
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}

}  // namespace
}  // namespace sg

extern "C" {

sg_status sg_batch_ca_graph_create(const sg_batch_plan *plan, int steps, int start_parity,
                                   const sg_launch_opts *opts, void **graph)
{
    return capture_batch(plan, steps, 1, start_parity, opts, graph);
}

sg_status sg_batch_ca_graph_create_fused(const sg_batch_plan *plan, int steps, int k,
                                         int start_parity, const sg_launch_opts *opts,
                                         void **graph)
{
    return capture_batch(plan, steps, k, start_parity, opts, graph);
}

sg_status sg_batch_ca_steps(const sg_batch_plan *plan, int parity, int k,
                            const sg_launch_opts *opts, void *stream)
{
    if (!plan_ok(plan) || (parity != 0 && parity != 1) || k < 1 || k > SG_FUSE_MAX ||
        plan->reserved[0] > k || (k == 1 && plan->reserved[0] > 1))
        return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    const cudaError_t e = launch_batch_k(plan, parity, k, (cudaStream_t)stream, cfg);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}

sg_status sg_graph_launch(void *graph, void *stream)
{
    if (graph == nullptr) return SG_EINVAL;
    const cudaError_t e = cudaGraphLaunch((cudaGraphExec_t)graph, (cudaStream_t)stream);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}

sg_status sg_graph_destroy(void *graph)
{
    if (graph == nullptr) return SG_EINVAL;
    const cudaError_t e = cudaGraphExecDestroy((cudaGraphExec_t)graph);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}

}  // extern "C"

namespace sg {
namespace {

// Time `trial_steps` parity-0 launches of k steps for every (rho, walking
// order, CTAs per SM) and plan with the fastest; results are cached per
// (trial_steps, k, sorted levels).
sg_status autotune(int count, const int *levels, uint8_t *const *buf_a, uint8_t *const *buf_b,
                   void *workspace, uint64_t workspace_bytes, int trial_steps, int k,
                   sg_batch_plan *plan, sg_launch_opts *opts_out, void *stream)
{
    if (count < 1 || count > kMaxBatch || levels == nullptr || plan == nullptr ||
        opts_out == nullptr || trial_steps < 1 || trial_steps > 1000 || k < 1 ||
        k > SG_FUSE_MAX)
        return SG_EINVAL;
    int min_level = 16;
    std::vector<int> sorted(levels, levels + count);
    std::sort(sorted.begin(), sorted.end());
    min_level = sorted.front();
    std::string key = std::to_string(trial_steps) + "/" + std::to_string(k) + ":";
    for (int r : sorted) key += std::to_string(r) + ",";
    int best_rho = 0, best_order = 1, best_cps = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best_rho = it->second[0];
            best_order = it->second[1];
            best_cps = it->second[2];
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (best_rho == 0) {
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaEventCreate(&e1);
        if (e != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e); }
        float best_ms = 1e30f;
        sg_status status = SG_OK;
        for (int rho : {16, 32, 64}) {
            if ((1 << min_level) < rho) continue;
            sg_batch_plan p;
            status = sg_batch_ca_plan(count, levels, buf_a, buf_b, rho, workspace,
                                      workspace_bytes, &p, stream);
            if (status != SG_OK) break;
            for (int order : {SG_ORDER_ROWMAJOR, SG_ORDER_INTERLEAVED}) {
                for (int cps : {0, 2, 4, 8}) {
                    LaunchCfg cfg;
                    cfg.order = order;
                    cfg.ctas_per_sm = cps;
                    // repeated parity-0 steps read buffer a and rewrite buffer b:
                    // the caller's current state (a) is left as it was
                    e = launch_batch_k(&p, 0, k, st, cfg);               // warm-up
                    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                    for (int t = 0; t < trial_steps && e == cudaSuccess; ++t)
                        e = launch_batch_k(&p, 0, k, st, cfg);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) { status = cuda_fail(e); break; }
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_rho = rho;
                        best_order = order;
                        best_cps = cps;
                    }
                }
                if (status != SG_OK) break;
            }
            if (status != SG_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (status != SG_OK) return status;
        if (best_rho == 0) return SG_EUNSUPPORTED;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = {best_rho, best_order, best_cps};
    }
    sg_status status = sg_batch_ca_plan(count, levels, buf_a, buf_b, best_rho, workspace,
                                        workspace_bytes, plan, stream);
    if (status != SG_OK) return status;
    *opts_out = sg_launch_opts{};
    opts_out->order = best_order;
    opts_out->store = SG_STORE_AUTO;
    opts_out->ctas_per_sm = best_cps;
    return SG_OK;
}

}  // namespace
}  // namespace sg

extern "C" {

sg_status sg_batch_ca_autotune(int count, const int *levels, uint8_t *const *buf_a,
                               uint8_t *const *buf_b, void *workspace, uint64_t workspace_bytes,
                               int trial_steps, sg_batch_plan *plan, sg_launch_opts *opts_out,
                               void *stream)
{
    return autotune(count, levels, buf_a, buf_b, workspace, workspace_bytes, trial_steps, 1,
                    plan, opts_out, stream);
}

sg_status sg_batch_ca_autotune_fused(int count, const int *levels, uint8_t *const *buf_a,
                                     uint8_t *const *buf_b, void *workspace,
                                     uint64_t workspace_bytes, int trial_launches, int k,
                                     sg_batch_plan *plan, sg_launch_opts *opts_out, void *stream)
{
    return autotune(count, levels, buf_a, buf_b, workspace, workspace_bytes, trial_launches, k,
                    plan, opts_out, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// A batch step that allocates nothing.
//
// Some callers cannot allocate device memory when they want to step a batch:
// a real-time loop that reserved its whole memory budget at start-up, a
// plugin whose host application owns every device allocation, or a server
// that has already handed all of HBM to its own pool.  For them a cudaMalloc
// (or any allocating library call, torch's included) can fail, stall the
// device or break the host's memory accounting.  This variant of the batch
// step keeps its work list in the fixed array below instead of a workspace
// the caller provides; the caller still passes the gaskets' state buffers.
// ---------------------------------------------------------------------------
namespace sg {
namespace {

constexpr int kNoAllocMaxGaskets = SG_NOALLOC_MAX_GASKETS;

// Fixed-size scratch: the work list of at most kNoAllocMaxGaskets gaskets.
// Every device that loads the library keeps it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_worklist[(4u * (kNoAllocMaxGaskets + 1) + 15u) / 16u * 16u + (4u * kNoAllocMaxGaskets + 15u) / 16u * 16u + 16u * kNoAllocMaxGaskets];

std::atomic<void *> g_noalloc_addr[64];

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) on its first use.
cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    void *p = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (p == nullptr) {
        e = cudaGetSymbolAddress(&p, g_noalloc_worklist);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace sg

extern "C" sg_status sg_batch_ca_step_noalloc(int count, const int *levels,
                                              uint8_t *const *buf_a, uint8_t *const *buf_b,
                                              int rho, int parity, const sg_launch_opts *opts,
                                              void *stream)
{
    if (count > kNoAllocMaxGaskets) {
        set_last_error_message("sg_batch_ca_step_noalloc: more gaskets than the fixed work-list "
                               "array holds (SG_NOALLOC_MAX_GASKETS)");
        return SG_EINVAL;
    }
    if (count < 1 || levels == nullptr || buf_a == nullptr || buf_b == nullptr) return SG_EINVAL;
    if (parity != 0 && parity != 1) return SG_EINVAL;
    if (rho != 16 && rho != 32 && rho != 64) return SG_EUNSUPPORTED;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    int s = 0;
    while ((1 << s) < rho) ++s;

    // Host image of the work list in a fixed per-thread buffer (no heap):
    // the same layout and the same checks as sg_batch_ca_plan.
    thread_local unsigned char img[sizeof(g_noalloc_worklist)];
    const WsLayout L = ws_layout(count);
    uint32_t *prefix = reinterpret_cast<uint32_t *>(img + L.prefix);
    int32_t *level = reinterpret_cast<int32_t *>(img + L.level);
    uint64_t *pa = reinterpret_cast<uint64_t *>(img + L.a);
    uint64_t *pb = reinterpret_cast<uint64_t *>(img + L.b);
    uint64_t total = 0;
    int max_level = 0;
    for (int i = 0; i < count; ++i) {
        const int r = levels[i];
        if (r < s || r > 16) return SG_EINVAL;
        if (buf_a[i] == nullptr || buf_b[i] == nullptr || buf_a[i] == buf_b[i]) return SG_EINVAL;
        if (((uintptr_t)buf_a[i] & 15) || ((uintptr_t)buf_b[i] & 15)) return SG_EINVAL;
        prefix[i] = (uint32_t)total;
        level[i] = r;
        pa[i] = (uint64_t)(uintptr_t)buf_a[i];
        pb[i] = (uint64_t)(uintptr_t)buf_b[i];
        total += (uint64_t)pow3i(r - s);
        max_level = std::max(max_level, r);
        if (total >= (1ull << 32)) return SG_EINVAL;
    }
    prefix[count] = (uint32_t)total;

    // The copy below reads `img`, a host buffer that the next call on this
    // thread overwrites, so a graph captured around it would replay whatever
    // that buffer holds then: refuse while `stream` is capturing.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) {
        set_last_error_message("sg_batch_ca_step_noalloc: the stream is being captured; the "
                               "work list is copied from a host buffer that the next call "
                               "reuses");
        return SG_EUNSUPPORTED;
    }
    void *scratch = nullptr;
    e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    // The whole work list the step reads is rewritten on `stream` first, so
    // nothing in the array has to start at zero.  (Pageable source: the copy
    // is staged before the call returns, so `img` can be reused next call.)
    e = cudaMemcpyAsync(scratch, img, L.total, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    sg_batch_plan plan{};
    plan.workspace = scratch;
    plan.workspace_bytes = sizeof(g_noalloc_worklist);
    plan.count = count;
    plan.rho = rho;
    plan.total_tiles = (uint32_t)total;
    plan.max_level = (uint32_t)max_level;
    e = launch_batch(&plan, parity, (cudaStream_t)stream, cfg);
    return e == cudaSuccess ? SG_OK : cuda_fail(e);
}
