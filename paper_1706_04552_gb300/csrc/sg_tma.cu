// sg_tma.cu -- host-side tensor-map encoding and the device status word.
#include <cudaTypedefs.h>

#include <atomic>

#include "sg_tma.cuh"

namespace sg {

namespace {
__device__ int g_device_status = 0;

constexpr int kMaxDevices = 64;
std::atomic<int *> g_status_ptr[kMaxDevices];
std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};

cudaError_t encode_fn(PFN_cuTensorMapEncodeTiled_v12000 *out)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = g_encode.load(std::memory_order_acquire);
    if (fn == nullptr) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || p == nullptr) return cudaErrorNotSupported;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        g_encode.store(fn, std::memory_order_release);
    }
    *out = fn;
    return cudaSuccess;
}
}  // namespace

cudaError_t make_grid_tensor_map(CUtensorMap *map, void *grid, int r, int elem_bytes, int rho)
{
    return make_box_tensor_map(map, grid, r, elem_bytes, rho, rho);
}

cudaError_t make_box_tensor_map(CUtensorMap *map, void *grid, int r, int elem_bytes, int box_w,
                                int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    cudaError_t e = encode_fn(&fn);
    if (e != cudaSuccess) return e;
    const cuuint64_t n = 1ull << r;
    const cuuint64_t dims[2] = {n, n};
    const cuuint64_t strides[1] = {n * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt =
        elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult res = fn(map, dt, 2, grid, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t device_status_ptr(int **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int *p = g_status_ptr[dev].load(std::memory_order_acquire);
    if (p == nullptr) {
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_device_status);
        if (e != cudaSuccess) return e;
        g_status_ptr[dev].store(p, std::memory_order_release);
    }
    *ptr = p;
    return cudaSuccess;
}

namespace {
// Every block waits on an mbarrier of its own that expects one arrival.  With
// `arrive` thread 0 makes it, so the phase completes; without it nothing ever
// arrives, each wait gives up after limit_ns and the block records kDevTimeout.
__global__ void __launch_bounds__(128) wait_selftest_kernel(int *status, int arrive,
                                                            uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) record_device_error(status, kDevTimeout);
    __syncthreads();
}
}  // namespace

cudaError_t launch_wait_selftest(int blocks, int arrive, uint64_t limit_ns, cudaStream_t st)
{
    int *status = nullptr;
    cudaError_t e = device_status_ptr(&status);
    if (e != cudaSuccess) return e;
    wait_selftest_kernel<<<blocks, 128, 0, st>>>(status, arrive, limit_ns);
    return cudaGetLastError();
}

cudaError_t read_device_status(int *status, cudaStream_t st)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(status, g_device_status, sizeof(int), 0,
                                              cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (*status != 0)
        e = cudaMemcpyToSymbolAsync(g_device_status, &zero, sizeof(int), 0,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace sg
