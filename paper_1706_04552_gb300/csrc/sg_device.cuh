// sg_device.cuh -- device building blocks shared by the libsg kernels:
// the warp-parallel lambda(omega) block decode (Theorem 1), per-cell values,
// and launch-geometry helpers.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sg {

constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ constexpr int pow3i(int k) { return k == 0 ? 1 : 3 * pow3i(k - 1); }

// ---------------------------------------------------------------------------
// lambda(omega), Theorem 1, decoded by one warp.
//
// Lane l (l < 16) owns level mu = l + 1.  Eq. beta reads omega_y at odd mu
// (even l) and omega_x at even mu (odd l), digit ceil(mu/2)-1 = l/2 in base
// 3; Eq. Delta turns the digit into the offset weights (Dx, Dy) =
// (beta/2, beta - beta/2); Eq. tau scales them by 2^(mu-1); Eq. lambda sums
// the tau over all levels, which one warp reduction (redux.sync) does: the
// x part is packed in the low 16 bits and the y part in the high 16 bits of
// one word, and since every tau is a distinct power of two no carry crosses
// between lanes or halves.  The result is mirrored into the (x & y) == 0
// orientation: by = n_b - 1 - lambda_y.
//
// The per-lane divisor 3^(l/2) is replaced by a fixed-point reciprocal
// m = ceil(2^32 / 3^k): for w < 3^8 and 3^k <= 3^7, floor(w * m / 2^32) is
// exactly floor(w / 3^k) because w * (m * 3^k - 2^32) < 2^32.
// ---------------------------------------------------------------------------
struct LambdaLane {
    uint64_t recip;    // ceil(2^32 / 3^(l/2))
    uint32_t shift;    // mu - 1
    uint32_t reads_y;  // 1 at odd mu
    uint32_t active;   // mu <= rb
    uint32_t nb_m1;    // n_b - 1

    __device__ __forceinline__ void init(int lane, int rb)
    {
        const int l = lane & 15;
        uint64_t p = 1;
        for (int i = 0; i < (l >> 1); ++i) p *= 3;
        recip = ((1ull << 32) + p - 1) / p;
        shift = (uint32_t)l;
        reads_y = (l & 1) == 0;
        active = (lane < 16) && (l < rb);
        nb_m1 = (1u << rb) - 1u;
    }

    // Every lane of the warp must call this with the same (wx, wy).
    __device__ __forceinline__ uint2 decode(uint32_t wx, uint32_t wy) const
    {
        const uint32_t w = reads_y ? wy : wx;
        const uint32_t d = (uint32_t)(((uint64_t)w * recip) >> 32);
        const uint32_t beta = d - 3u * ((d * 0xAAABu) >> 17);   // d mod 3, d < 2^16
        const uint32_t dx = beta >> 1, dy = beta - dx;
        const uint32_t tau = active ? ((dx << shift) | (dy << (shift + 16))) : 0u;
        const uint32_t sum = __reduce_add_sync(0xffffffffu, tau);
        return make_uint2(sum & 0xFFFFu, nb_m1 - (sum >> 16));
    }
};

// The parallel space Pi is walked row by row: q -> omega = (q mod W, q div W)
// with W = 3^floor(rb/2).  A persistent loop advances q by a fixed stride, so
// omega is stepped incrementally instead of divided every time.
struct OmegaWalker {
    uint32_t wx, wy, W, step_x, step_y;

    __device__ __forceinline__ void init(uint32_t q0, uint32_t stride, uint32_t W_)
    {
        W = W_;
        wy = q0 / W;
        wx = q0 - wy * W;
        step_y = stride / W;
        step_x = stride - step_y * W;
    }
    __device__ __forceinline__ void advance()
    {
        wx += step_x;
        wy += step_y;
        if (wx >= W) { wx -= W; wy += 1; }
    }
};

// ---------------------------------------------------------------------------
// Values written by the map-and-write pass.
// ---------------------------------------------------------------------------
enum : int { kValConst = 0, kValLinear31 = 1, kValHash = 2 };

// SplitMix64 output for generator state s (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t s)
{
    uint64_t z = s + kGoldenGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T> struct Value;

template <> struct Value<uint8_t> {
    template <int VK>
    static __device__ __forceinline__ uint8_t at(uint32_t x, uint32_t y, int r,
                                                 uint64_t vs, uint64_t seedmix)
    {
        if (VK == kValConst) return (uint8_t)vs;
        if (VK == kValLinear31) return (uint8_t)((x * 31u + y) & 0xFFu);
        const uint64_t key = ((uint64_t)y << r) | x;
        return (uint8_t)(splitmix64(seedmix ^ key) >> 56);
    }
};

template <> struct Value<float> {
    template <int VK>
    static __device__ __forceinline__ float at(uint32_t x, uint32_t y, int r,
                                               uint64_t vs, uint64_t seedmix)
    {
        if (VK == kValConst) return __uint_as_float((uint32_t)vs);
        if (VK == kValLinear31) return (float)((x * 31u + y) & 0xFFu);
        const uint64_t key = ((uint64_t)y << r) | x;
        // a 24-bit integer scaled by 2^-24: exact in float
        return (float)(uint32_t)(splitmix64(seedmix ^ key) >> 40) * (1.0f / 16777216.0f);
    }
};

__device__ __forceinline__ bool in_gasket(uint32_t x, uint32_t y) { return (x & y) == 0u; }

}  // namespace sg
