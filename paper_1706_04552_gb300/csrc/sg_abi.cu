// sg_abi.cu -- the extern "C" surface of libsg (declared in include/sg.h):
// host-side argument checks, dispatch to the kernels, the standalone lambda
// block-map kernel and the host-only launch accounting.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "sg.h"
#include "sg_device.cuh"
#include "sg_internal.h"
#include "sg_compact.cuh"
#include "sg_tma.cuh"

namespace sg {

namespace {
thread_local char g_last_error[256] = "";

constexpr int kMaxDevices = 64;
std::atomic<int> g_sm_count[kMaxDevices];

sg_status fail_cuda(cudaError_t e)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return SG_ECUDA;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int log2i(int v)
{
    int s = 0;
    while ((1 << s) < v) ++s;
    return s;
}

// Common checks of level and tile side; on success *s = log2(rho).
bool valid_level_tile(int r, int rho, int *s)
{
    if (r < 0 || r > 16) return false;
    if (!is_pow2(rho) || rho > 64) return false;
    if (rho > (1 << r)) return false;
    *s = log2i(rho);
    return true;
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// Library defaults: the measured best on GB300.
constexpr int kDefaultOrder = kOrderInterleaved;
constexpr int kDefaultWholeTileStore = kStoreStaged;

}  // namespace

// Translate sg_launch_opts (NULL = defaults) into a LaunchCfg.
bool read_launch_opts(const sg_launch_opts *o, LaunchCfg *cfg)
{
    cfg->order = kDefaultOrder;
    cfg->store = kStoreAuto;
    cfg->ctas_per_sm = 0;
    if (o == nullptr) return true;
    for (int v : o->reserved)
        if (v != 0) return false;
    if (o->order != -1) {
        if (o->order != SG_ORDER_ROWMAJOR && o->order != SG_ORDER_INTERLEAVED) return false;
        cfg->order = o->order;
    }
    if (o->store < SG_STORE_AUTO || o->store > SG_STORE_MASKED) return false;
    cfg->store = o->store;
    if (o->ctas_per_sm < 0 || o->ctas_per_sm > 64) return false;
    cfg->ctas_per_sm = o->ctas_per_sm;
    return true;
}

void set_last_error_message(const char *msg)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s", msg);
}

sg_status set_last_cuda_error(cudaError_t e)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return e == cudaErrorNotSupported ? SG_EUNSUPPORTED : SG_ECUDA;
}

namespace {

sg_status finish(cudaError_t e)
{
    if (e == cudaSuccess) return SG_OK;
    if (e == cudaErrorNotSupported) return SG_EUNSUPPORTED;
    return fail_cuda(e);
}

// One warp per launch index; lane results of the reduction are identical,
// lane 0 stores them.
__global__ void __launch_bounds__(256)
block_map_kernel(uint32_t *__restrict__ bx, uint32_t *__restrict__ by, int rb,
                 int order, uint32_t total)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    LambdaLane ll;
    ll.init(threadIdx.x & 31, rb, order);
    OmegaWalker ow;
    ow.init(warp, nwarps, pi_word(order, rb));
    for (uint32_t q = warp; q < total; q += nwarps) {
        const uint2 b = ll.decode(ow.a, ow.b);
        ow.advance();
        if ((threadIdx.x & 31) == 0) {
            bx[q] = b.x;
            by[q] = b.y;
        }
    }
}
}  // namespace

int sm_count(int *err)
{
    *err = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *err = (int)e; return 0; }
    if (dev >= 0 && dev < kMaxDevices) {
        int c = g_sm_count[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int c = 0;
    e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { *err = (int)e; return 0; }
    if (dev >= 0 && dev < kMaxDevices) g_sm_count[dev].store(c, std::memory_order_relaxed);
    return c;
}

cudaError_t launch_block_map(int rb, int order, uint32_t *bx, uint32_t *by, cudaStream_t st)
{
    const uint32_t total = (uint32_t)pow3i(rb);
    LaunchCfg cfg;
    unsigned grid = 1;
    static std::atomic<int> occ{0};
    cudaError_t e = persistent_grid(block_map_kernel, 256, 0, (total + 7) / 8, cfg, &grid, &occ);
    if (e != cudaSuccess) return e;
    block_map_kernel<<<grid, 256, 0, st>>>(bx, by, rb, order, total);
    return cudaGetLastError();
}

}  // namespace sg

using namespace sg;

extern "C" {

int sg_abi_version(void) { return SG_ABI_VERSION; }

const char *sg_status_str(sg_status s)
{
    switch (s) {
    case SG_OK: return "SG_OK";
    case SG_EINVAL: return "SG_EINVAL: invalid argument";
    case SG_ECUDA: return "SG_ECUDA: CUDA runtime error";
    case SG_ENOMEM: return "SG_ENOMEM: out of memory";
    case SG_ETIMEOUT: return "SG_ETIMEOUT: a bounded device wait gave up";
    case SG_EUNSUPPORTED: return "SG_EUNSUPPORTED: combination not provided";
    default: return "unknown sg_status";
    }
}

const char *sg_last_error_string(void) { return g_last_error; }

sg_status sg_map_write_ex(int r, int rho, sg_map map, sg_dtype dtype, void *grid,
                          sg_value_kind value_kind, uint64_t value_or_seed,
                          const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (value_kind < SG_VAL_CONST || value_kind > SG_VAL_HASH) return SG_EINVAL;
    if (grid == nullptr) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    const int elem = dtype == SG_U8 ? 1 : 4;
    if (!aligned(grid, (uintptr_t)elem)) return SG_EINVAL;
    // staged stores move whole 16-byte chunks: tile rows of >= 16 bytes and a
    // 16-byte aligned grid; AUTO falls back to per-cell stores otherwise
    const bool can_stage = rho * elem >= 16;
    if (cfg.store == SG_STORE_STAGED || cfg.store == SG_STORE_TMA ||
        cfg.store == SG_STORE_FILL) {
        if (!can_stage) return SG_EUNSUPPORTED;
        if (!aligned(grid, 16)) return SG_EINVAL;
    } else if (cfg.store == SG_STORE_SECTOR || cfg.store == SG_STORE_MERGE ||
               cfg.store == SG_STORE_MASKED) {
        // one lane per unit of whole 32-byte sectors: tile rows of >= 32 bytes
        if (rho * elem < 32) return SG_EUNSUPPORTED;
        if (!aligned(grid, 32)) return SG_EINVAL;
    } else if (cfg.store == SG_STORE_AUTO) {
        // the measured best that keeps off-gasket content: whole 32-byte
        // sectors read, merged and written back where the tile rows allow it
        if (rho * elem >= 32 && aligned(grid, 32)) cfg.store = kStoreMerge;
        else cfg.store = (can_stage && aligned(grid, 16)) ? kDefaultWholeTileStore : kStoreScatter;
    }
    if (dtype == SG_U8)
        return finish(launch_write_u8(r, s, (int)map, (int)value_kind, (uint8_t *)grid,
                                      value_or_seed, (cudaStream_t)stream, cfg));
    return finish(launch_write_f32(r, s, (int)map, (int)value_kind, (float *)grid,
                                   value_or_seed, (cudaStream_t)stream, cfg));
}

sg_status sg_map_write_mapped(int r, int rho, sg_map map, sg_dtype dtype, void *host_grid,
                              sg_value_kind value_kind, uint64_t value_or_seed,
                              const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (value_kind < SG_VAL_CONST || value_kind > SG_VAL_HASH) return SG_EINVAL;
    if (host_grid == nullptr) return SG_EINVAL;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    const int elem = dtype == SG_U8 ? 1 : 4;
    // only the paths that move data with plain loads and stores: fill runs
    // as write-only whole chunks of the staged kernel (no bulk tensor copy)
    if (cfg.store == SG_STORE_TMA) return SG_EUNSUPPORTED;
    const bool sector_mode = cfg.store == SG_STORE_SECTOR || cfg.store == SG_STORE_MERGE ||
                             cfg.store == SG_STORE_MASKED;
    if (sector_mode && rho * elem < 32) return SG_EUNSUPPORTED;   // 32-byte tile rows
    if ((cfg.store == SG_STORE_STAGED || cfg.store == SG_STORE_FILL) && rho * elem < 16)
        return SG_EUNSUPPORTED;                       // whole chunks need 16-byte tile rows
    // the pointer must be page-locked host memory mapped into the device's
    // address space; anything else is refused before a launch
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, host_grid) != cudaSuccess) {
        cudaGetLastError();                           // reset the runtime's last error
        set_last_error_message("sg_map_write_mapped: pointer attributes unavailable");
        return SG_EINVAL;
    }
    if (attr.type != cudaMemoryTypeHost || attr.devicePointer == nullptr) {
        set_last_error_message("sg_map_write_mapped: not page-locked host memory mapped "
                               "into the device");
        return SG_EINVAL;
    }
    void *grid = attr.devicePointer;
    if (!aligned(grid, (uintptr_t)elem)) return SG_EINVAL;
    if (sector_mode && !aligned(grid, 32)) return SG_EINVAL;
    const bool can_stage = rho * elem >= 16 && aligned(grid, 16);
    if ((cfg.store == SG_STORE_STAGED || cfg.store == SG_STORE_FILL) && !can_stage)
        return SG_EUNSUPPORTED;
    if (cfg.store == SG_STORE_FILL) cfg.store = kStoreFillPlain;
    // the same choice as on a device grid: 32-byte read-merge-write carries
    // over the link better than staged 16-byte chunks
    if (cfg.store == SG_STORE_AUTO)
        cfg.store = rho * elem >= 32 && aligned(grid, 32) ? kStoreMerge
                    : can_stage                            ? kStoreStaged
                                                           : kStoreScatter;
    if (dtype == SG_U8)
        return finish(launch_write_u8(r, s, (int)map, (int)value_kind, (uint8_t *)grid,
                                      value_or_seed, (cudaStream_t)stream, cfg));
    return finish(launch_write_f32(r, s, (int)map, (int)value_kind, (float *)grid,
                                   value_or_seed, (cudaStream_t)stream, cfg));
}

sg_status sg_map_write(int r, int rho, sg_map map, sg_dtype dtype, void *grid,
                       sg_value_kind value_kind, uint64_t value_or_seed, void *stream)
{
    return sg_map_write_ex(r, rho, map, dtype, grid, value_kind, value_or_seed, nullptr, stream);
}

sg_status sg_ca_step_ex(int r, int rho, sg_map map, const uint8_t *in, uint8_t *out,
                        const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (map != SG_MAP_LAMBDA && map != SG_MAP_BBOX) return SG_EUNSUPPORTED;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (!aligned(in, 16) || !aligned(out, 16)) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    return finish(launch_ca(r, s, (int)map, in, out, (cudaStream_t)stream, cfg));
}

sg_status sg_ca_step(int r, int rho, sg_map map, const uint8_t *in, uint8_t *out,
                     void *stream)
{
    return sg_ca_step_ex(r, rho, map, in, out, nullptr, stream);
}

sg_status sg_diffuse_step_ex(int r, int rho, sg_map map, const float *in, float *out,
                             float alpha, const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (map != SG_MAP_LAMBDA && map != SG_MAP_BBOX) return SG_EUNSUPPORTED;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (!aligned(in, 16) || !aligned(out, 16)) return SG_EINVAL;
    if (!(alpha == alpha) || alpha > 3.0e38f || alpha < -3.0e38f) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    return finish(launch_diffuse(r, s, (int)map, in, out, alpha, (cudaStream_t)stream, cfg));
}

sg_status sg_diffuse_step(int r, int rho, sg_map map, const float *in, float *out,
                          float alpha, void *stream)
{
    return sg_diffuse_step_ex(r, rho, map, in, out, alpha, nullptr, stream);
}

sg_status sg_ca_steps(int r, int rho, sg_map map, const uint8_t *in, uint8_t *out, int k,
                      const sg_launch_opts *opts, void *stream)
{
    if (k < 1 || k > SG_FUSE_MAX) return SG_EINVAL;
    if (k == 1) return sg_ca_step_ex(r, rho, map, in, out, opts, stream);
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (map != SG_MAP_LAMBDA && map != SG_MAP_BBOX) return SG_EUNSUPPORTED;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (!aligned(in, 16) || !aligned(out, 16)) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    if (rho < 16) return SG_EUNSUPPORTED;
    return finish(launch_ca_fused(r, s, (int)map, in, out, k, (cudaStream_t)stream, cfg));
}

sg_status sg_diffuse_steps(int r, int rho, sg_map map, const float *in, float *out,
                           float alpha, int k, const sg_launch_opts *opts, void *stream)
{
    if (k < 1 || k > SG_FUSE_MAX) return SG_EINVAL;
    if (k == 1) return sg_diffuse_step_ex(r, rho, map, in, out, alpha, opts, stream);
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    if (map < SG_MAP_LAMBDA || map > SG_MAP_LAMBDA_UNROLL) return SG_EINVAL;
    if (map != SG_MAP_LAMBDA && map != SG_MAP_BBOX) return SG_EUNSUPPORTED;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (!aligned(in, 16) || !aligned(out, 16)) return SG_EINVAL;
    if (!(alpha == alpha) || alpha > 3.0e38f || alpha < -3.0e38f) return SG_EINVAL;
    LaunchCfg cfg;
    if (!read_launch_opts(opts, &cfg)) return SG_EINVAL;
    if (rho < 16) return SG_EUNSUPPORTED;
    return finish(launch_diffuse_fused(r, s, (int)map, in, out, alpha, k,
                                       (cudaStream_t)stream, cfg));
}

sg_status sg_block_map(int rb, sg_order order, uint32_t *bx, uint32_t *by, void *stream)
{
    if (rb < 0 || rb > 16) return SG_EINVAL;
    if (order != SG_ORDER_ROWMAJOR && order != SG_ORDER_INTERLEAVED) return SG_EINVAL;
    if (bx == nullptr || by == nullptr || bx == by) return SG_EINVAL;
    if (!aligned(bx, 4) || !aligned(by, 4)) return SG_EINVAL;
    return finish(launch_block_map(rb, (int)order, bx, by, (cudaStream_t)stream));
}

namespace {
// Checks shared by the compact entries; on success *s = log2(rho).
sg_status compact_args(int r, int rho, const sg_launch_opts *opts, LaunchCfg *cfg, int *s)
{
    if (!valid_level_tile(r, rho, s)) return SG_EINVAL;
    if (!read_launch_opts(opts, cfg)) return SG_EINVAL;
    if (cfg->store != kStoreAuto) return SG_EUNSUPPORTED;
    return SG_OK;
}
}  // namespace

sg_status sg_compact_pack(int r, int rho, sg_dtype dtype, const void *grid, void *compact,
                          const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    const int elem = dtype == SG_U8 ? 1 : 4;
    if (grid == nullptr || compact == nullptr || grid == compact) return SG_EINVAL;
    if (!aligned(grid, (uintptr_t)elem) || !aligned(compact, (uintptr_t)elem)) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    return finish(launch_compact_pack(r, s, cfg.order, elem, grid, compact,
                                      (cudaStream_t)stream, cfg));
}

sg_status sg_compact_unpack(int r, int rho, sg_dtype dtype, const void *compact, void *grid,
                            const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    const int elem = dtype == SG_U8 ? 1 : 4;
    if (grid == nullptr || compact == nullptr || grid == compact) return SG_EINVAL;
    if (!aligned(grid, (uintptr_t)elem) || !aligned(compact, (uintptr_t)elem)) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    return finish(launch_compact_unpack(r, s, cfg.order, elem, compact, grid,
                                        (cudaStream_t)stream, cfg));
}

sg_status sg_compact_map_write(int r, int rho, sg_dtype dtype, void *compact,
                               sg_value_kind value_kind, uint64_t value_or_seed,
                               const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    if (value_kind < SG_VAL_CONST || value_kind > SG_VAL_HASH) return SG_EINVAL;
    const int elem = dtype == SG_U8 ? 1 : 4;
    if (compact == nullptr || !aligned(compact, (uintptr_t)elem)) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    return finish(launch_compact_write(r, s, cfg.order, elem, (int)value_kind, compact,
                                       value_or_seed, (cudaStream_t)stream, cfg));
}

sg_status sg_compact_map_write_mapped(int r, int rho, sg_dtype dtype, void *host_compact,
                                      sg_value_kind value_kind, uint64_t value_or_seed,
                                      const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (dtype != SG_U8 && dtype != SG_F32) return SG_EINVAL;
    if (value_kind < SG_VAL_CONST || value_kind > SG_VAL_HASH) return SG_EINVAL;
    if (host_compact == nullptr) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    // page-locked host memory mapped into the device's address space only
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, host_compact) != cudaSuccess) {
        cudaGetLastError();                           // reset the runtime's last error
        set_last_error_message("sg_compact_map_write_mapped: pointer attributes unavailable");
        return SG_EINVAL;
    }
    if (attr.type != cudaMemoryTypeHost || attr.devicePointer == nullptr) {
        set_last_error_message("sg_compact_map_write_mapped: not page-locked host memory "
                               "mapped into the device");
        return SG_EINVAL;
    }
    const int elem = dtype == SG_U8 ? 1 : 4;
    if (!aligned(attr.devicePointer, (uintptr_t)elem)) return SG_EINVAL;
    return finish(launch_compact_write(r, s, cfg.order, elem, (int)value_kind,
                                       attr.devicePointer, value_or_seed, (cudaStream_t)stream,
                                       cfg, /*wide=*/true));
}

sg_status sg_compact_ca_step(int r, int rho, const uint8_t *in, uint8_t *out,
                             const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    return finish(launch_compact_ca(r, s, cfg.order, in, out, (cudaStream_t)stream, cfg));
}

sg_status sg_compact_ca_steps(int r, int rho, int k, const uint8_t *in, uint8_t *out,
                              const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (k < 1 || k > SG_FUSE_MAX) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    if (k == 1) return finish(launch_compact_ca(r, s, cfg.order, in, out, (cudaStream_t)stream, cfg));
    if (rho != 64) return SG_EUNSUPPORTED;
    return finish(launch_compact_ca_fused(r, cfg.order, in, out, k, (cudaStream_t)stream, cfg));
}

sg_status sg_compact_diffuse_step(int r, int rho, const float *in, float *out, float alpha,
                                  const sg_launch_opts *opts, void *stream)
{
    int s = 0;
    LaunchCfg cfg;
    if (in == nullptr || out == nullptr || in == out) return SG_EINVAL;
    if (!aligned(in, 4) || !aligned(out, 4)) return SG_EINVAL;
    if (!(alpha == alpha) || alpha > 3.0e38f || alpha < -3.0e38f) return SG_EINVAL;
    const sg_status st = compact_args(r, rho, opts, &cfg, &s);
    if (st != SG_OK) return st;
    return finish(launch_compact_diffuse(r, s, cfg.order, in, out, alpha, (cudaStream_t)stream,
                                         cfg));
}

sg_status sg_device_status(void *stream)
{
    int status = 0;
    cudaError_t e = read_device_status(&status, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e);
    if (status == kDevOk) return SG_OK;
    if (status == kDevOverflow) {
        set_last_error_message("sg_device_status: a fused diffusion unit had more live chunks "
                               "than its bound; that unit was not written");
        return SG_EUNSUPPORTED;
    }
    return SG_ETIMEOUT;
}

sg_status sg_wait_selftest(int blocks, int arrive, uint64_t limit_ns, void *stream)
{
    if (blocks < 1 || blocks > 1024) return SG_EINVAL;
    if (limit_ns < 1000 || limit_ns > kWaitLimitNs) return SG_EINVAL;
    return finish(launch_wait_selftest(blocks, arrive != 0, limit_ns, (cudaStream_t)stream));
}

sg_status sg_launch_stats(int r, int rho, sg_map map, uint64_t *launched, uint64_t *useful)
{
    int s = 0;
    if (!valid_level_tile(r, rho, &s)) return SG_EINVAL;
    uint64_t l;
    const uint64_t cells = (uint64_t)pow3i(r);
    switch (map) {
    case SG_MAP_LAMBDA: l = (uint64_t)pow3i(r - s) << (2 * s); break;
    case SG_MAP_BBOX: l = 1ull << (2 * r); break;
    case SG_MAP_LAMBDA_LUT:
    case SG_MAP_LAMBDA_UNROLL: l = cells; break;
    default: return SG_EINVAL;
    }
    if (launched) *launched = l;
    if (useful) *useful = cells;
    return SG_OK;
}

}  // extern "C"
