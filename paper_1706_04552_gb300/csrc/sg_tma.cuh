// sg_tma.cuh -- thin inline-PTX wrappers for the Blackwell bulk-copy engine
// (TMA) and shared-memory mbarriers, plus bounded waits.
//
// Every wait here is bounded by wall time (%globaltimer): a wait that has
// not completed after kWaitLimitNs reports failure instead of spinning on,
// and the caller records SG_ETIMEOUT in the device status word.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace sg {

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

// Device status word (one per device, defined in sg_tma.cu): 0 = fine,
// otherwise the first error a kernel recorded.  Kernels receive its address;
// sg_device_status() reads and clears it.
enum : int { kDevOk = 0, kDevTimeout = 1,
              // a fused diffusion unit listed more live chunks than its
              // register slots hold (a bound checked on the host; the unit is
              // skipped rather than run wrong)
              kDevOverflow = 2 };

__device__ __forceinline__ void record_device_error(int *status, int code)
{
    atomicCAS(status, kDevOk, code);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make barrier initialisation visible to the bulk-copy engine.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of `bar` to complete; false after `limit_ns`.
// Two bounds: the wall clock, and a count of polls that cannot finish in
// less than about half the limit (a poll takes at least one issue cycle,
// under 1 ns at the maximum SM clock), so the loop ends even if the timer
// were to stall.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    const uint64_t max_rounds = limit_ns / 32 + 1;   // 64 polls a round
    for (uint64_t round = 0; round < max_rounds; ++round) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// 2-D tiled bulk copy global -> shared, completing on `bar` (complete_tx).
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// 2-D tiled bulk copy shared -> global, tracked by the bulk async-group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y,
                                             const void *smem_src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_addr(smem_src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// All but the newest N committed bulk groups have finished reading shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// All committed bulk groups have completed (their writes are performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Order this thread's generic-proxy shared-memory writes before later
// bulk-copy (async-proxy) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Host: 2-D tensor map over a row-major n x n grid with rho x rho boxes.
cudaError_t make_grid_tensor_map(CUtensorMap *map, void *grid, int r, int elem_bytes, int rho);

// Host: the same with box_w x box_h boxes (box_w elements along a row).
cudaError_t make_box_tensor_map(CUtensorMap *map, void *grid, int r, int elem_bytes, int box_w,
                                int box_h);

// Host: device address of the current device's status word (cached per device).
cudaError_t device_status_ptr(int **ptr);

// Host: read the current device's status word into *status and clear it
// (synchronises `st`).
cudaError_t read_device_status(int *status, cudaStream_t st);

// Host: launch the bounded-wait self-test (sg_wait_selftest) on `st`.
cudaError_t launch_wait_selftest(int blocks, int arrive, uint64_t limit_ns, cudaStream_t st);

}  // namespace sg
