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
// Lane l (l < 16) owns level mu = l + 1.  Eq. beta takes, at level mu, the
// base-3 digit ceil(mu/2)-1 of omega_y (odd mu) or omega_x (even mu); Eq.
// Delta turns the digit into the offset weights (Dx, Dy) = (beta/2,
// beta - beta/2); Eq. tau scales them by 2^(mu-1); Eq. lambda sums the tau
// over all levels, which one warp reduction (redux.sync) does: the x part is
// packed in the low 16 bits and the y part in the high 16 bits of one word,
// and since every tau is a distinct power of two no carry crosses between
// lanes or halves.  The result is mirrored into the (x & y) == 0
// orientation: by = n_b - 1 - lambda_y.
//
// The warp is handed two base-3 words (a, b), each below 3^8, and lane l
// reads one digit of one of them:
//   kOrderRowMajor:    (a, b) = (omega_x, omega_y), the paper's Pi walked row
//                      by row; lane l reads digit l/2 of b (l even) or a.
//   kOrderInterleaved: (a, b) = (q mod 3^8, q div 3^8) for launch index q, and
//                      omega is q with its base-3 digits dealt alternately to
//                      omega_y (even positions) and omega_x (odd positions);
//                      lane l then reads digit l mod 8 of a (l < 8) or b.
// Both give beta_mu = the digit Eq. beta names; the second walks Pi so that
// consecutive launch indices are neighbouring tiles (finest level fastest).
//
// The per-lane divisor 3^k (k <= 7) is replaced by a fixed-point reciprocal
// m = ceil(2^32 / 3^k): for w < 3^8, floor(w * m / 2^32) is exactly
// floor(w / 3^k) because w * (m * 3^k - 2^32) < 2^32.  For k = 0, m = 2^32
// does not fit a word; that lane keeps m = 0 and adds w itself.  This is the
// published method of division by an invariant integer through a multiply by
// a rounded-up reciprocal (Granlund and Montgomery, "Division by Invariant
// Integers using Multiplication", PLDI 1994); the inequality above is its
// exactness condition for this dividend range, and the host tests check it.
// ---------------------------------------------------------------------------
enum : int { kOrderRowMajor = 0, kOrderInterleaved = 1 };

constexpr uint32_t kPow3_8 = 6561;   // 3^8: the interleaved order's word size

__host__ __device__ inline uint32_t pi_word(int order, int rb)
{
    // the divisor that splits a launch index q into the two words (a, b)
    return order == kOrderInterleaved ? kPow3_8 : (uint32_t)pow3i(rb / 2);
}

// ceil(2^32 / 3^k) for k = 1..7 (k = 0 handled apart, see above)
__host__ __device__ constexpr uint32_t recip3(int k)
{
    return k == 1 ? 1431655766u : k == 2 ? 477218589u : k == 3 ? 159072863u
         : k == 4 ? 53024288u : k == 5 ? 17674763u : k == 6 ? 5891588u
         : k == 7 ? 1963863u : 0u;
}

struct LambdaLane {
    uint32_t recip;    // ceil(2^32 / 3^digit), 0 for digit 0
    uint32_t keep_w;   // all ones for digit 0 (quotient = w), else 0
    uint32_t shift;    // mu - 1
    uint32_t reads_b;  // this lane's digit comes from word b
    uint32_t active;   // mu <= rb
    uint32_t nb_m1;    // n_b - 1

    __device__ __forceinline__ void init(int lane, int rb, int order)
    {
        const int l = lane & 15;
        const int digit = order == kOrderInterleaved ? (l & 7) : (l >> 1);
        // select from the table with compile-time indices (no local memory)
        recip = 0u;
#pragma unroll
        for (int i = 1; i < 8; ++i)
            if (digit == i) recip = recip3(i);
        keep_w = digit == 0 ? 0xFFFFFFFFu : 0u;
        shift = (uint32_t)l;
        reads_b = order == kOrderInterleaved ? (l >= 8) : ((l & 1) == 0);
        active = (lane < 16) && (l < rb);
        nb_m1 = (1u << rb) - 1u;
    }

    // Re-aim the lane at another block-space level (the digit constants
    // depend only on the walking order): used by batches of gaskets.
    __device__ __forceinline__ void set_level(int lane, int rb)
    {
        const int l = lane & 15;
        active = (lane < 16) && (l < rb);
        nb_m1 = (1u << rb) - 1u;
    }

    // Every lane of the warp must call this with the same (a, b).
    __device__ __forceinline__ uint2 decode(uint32_t a, uint32_t b) const
    {
        const uint32_t w = reads_b ? b : a;
        const uint32_t d = __umulhi(w, recip) + (w & keep_w);
        // d mod 3 for d < 2^16: 0xAAAB = ceil(2^17 / 3), the same
        // rounded-up-reciprocal division (exact: d * (3 * 0xAAAB - 2^17) < 2^17)
        const uint32_t beta = d - 3u * ((d * 0xAAABu) >> 17);
        const uint32_t dx = beta >> 1, dy = beta - dx;
        const uint32_t tau = active ? ((dx << shift) | (dy << (shift + 16))) : 0u;
        const uint32_t sum = __reduce_add_sync(0xffffffffu, tau);
        return make_uint2(sum & 0xFFFFu, nb_m1 - (sum >> 16));
    }
};

// A persistent loop advances the launch index q by a fixed stride; the two
// words (a, b) = (q mod W, q div W) are stepped incrementally instead of
// divided every time.
struct OmegaWalker {
    uint32_t a, b, W, step_a, step_b;

    __device__ __forceinline__ void init(uint32_t q0, uint32_t stride, uint32_t W_)
    {
        W = W_;
        b = q0 / W;
        a = q0 - b * W;
        step_b = stride / W;
        step_a = stride - step_b * W;
    }
    __device__ __forceinline__ void advance()
    {
        a += step_a;
        b += step_b;
        if (a >= W) { a -= W; b += 1; }
    }
};

// ---------------------------------------------------------------------------
// Values written by the map-and-write pass.
// ---------------------------------------------------------------------------
enum : int { kValConst = 0, kValLinear31 = 1, kValHash = 2 };

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): for generator state s,
// z = s + gamma; z = (z ^ (z >> 30)) * M1; z = (z ^ (z >> 27)) * M2;
// output z ^ (z >> 31).
//
// splitmix64_hi_state: the high 32 bits of the output for the state
// seedmix ^ key, key below 2^32, given as its halves (s_lo, s_hi).  The
// written values use only bits 40..63 of the output (u8: h >> 56; f32:
// h >> 40), and the finaliser's last step h = z ^ (z >> 31) leaves bits
// 33..63 of z unchanged, so h >> 32 agrees with z >> 32 in every bit used
// (bits 40..63); that step is skipped.  The rest is the same 64-bit
// arithmetic written on 32-bit halves: the state's high half is the
// constant high half of seedmix, each 64-bit shift is one funnel shift per
// half, and the second product needs only its high half.
__device__ __forceinline__ uint32_t splitmix64_hi_state(uint32_t s_lo, uint32_t s_hi)
{
    constexpr uint32_t G_LO = (uint32_t)kGoldenGamma, G_HI = (uint32_t)(kGoldenGamma >> 32);
    constexpr uint64_t M1 = 0xBF58476D1CE4E5B9ull, M2 = 0x94D049BB133111EBull;
    constexpr uint32_t M1_LO = (uint32_t)M1, M1_HI = (uint32_t)(M1 >> 32);
    constexpr uint32_t M2_LO = (uint32_t)M2, M2_HI = (uint32_t)(M2 >> 32);
    // z = s + gamma: the high half is one of two values (carry or not), and
    // so is the high half after the first xor-shift; both pairs depend only
    // on the seed and are computed once per thread
    const uint32_t zh0 = s_hi + G_HI, zh1 = zh0 + 1u;
    const uint32_t th0 = zh0 ^ (zh0 >> 30), th1 = zh1 ^ (zh1 >> 30);
    const uint32_t z_lo = s_lo + G_LO;
    const bool carry = z_lo < s_lo;
    const uint32_t z_hi = carry ? zh1 : zh0;
    // z ^= z >> 30
    const uint32_t t_lo = z_lo ^ __funnelshift_r(z_lo, z_hi, 30);
    const uint32_t t_hi = carry ? th1 : th0;
    // z *= M1 (mod 2^64)
    const uint64_t p = (uint64_t)t_lo * M1_LO;
    const uint32_t y_lo = (uint32_t)p;
    const uint32_t y_hi = (uint32_t)(p >> 32) + t_lo * M1_HI + t_hi * M1_LO;
    // z ^= z >> 27
    const uint32_t w_lo = y_lo ^ __funnelshift_r(y_lo, y_hi, 27);
    const uint32_t w_hi = y_hi ^ (y_hi >> 27);
    // high half of z * M2 (mod 2^64)
    return __umulhi(w_lo, M2_LO) + w_lo * M2_HI + w_hi * M2_LO;
}

// Value of the cell whose linear index (row-major, pitch n = 2^r) is
// base + koff, for r <= 16 (so the index, which is also the hash key y*n + x,
// fits in 32 bits).  The write kernels split the index into a per-tile base
// ((y0 << r) | x0, x0 and y0 multiples of rho) and a per-thread offset that
// is the same for every tile ((ty << r) | tx, tx and ty below rho).  Their
// bits are disjoint, so base + koff = base ^ koff, and the hash state
// seedmix ^ key is (seedmix ^ base) ^ koff: one xor per cell after a per-tile
// xor.  For the linear value the split is the same with x*31 + y in place of
// the index (an add there: those bits overlap).
template <typename T, int VK> struct CellValue {
    uint64_t seedmix;      // seed * gamma
    uint32_t cval;         // the constant's bits

    __device__ __forceinline__ static uint32_t base_of(uint32_t x0, uint32_t y0, int r)
    {
        return VK == kValLinear31 ? x0 * 31u + y0 : (y0 << r) | x0;
    }
    __device__ __forceinline__ static uint32_t offset_of(uint32_t tx, uint32_t ty, int r)
    {
        return VK == kValLinear31 ? tx * 31u + ty : (ty << r) | tx;
    }
    __device__ __forceinline__ T operator()(uint32_t base, uint32_t koff) const
    {
        if constexpr (VK == kValConst) {
            if constexpr (sizeof(T) == 1) return (T)cval;
            else return __uint_as_float(cval);
        } else if constexpr (VK == kValLinear31) {
            return (T)((base + koff) & 0xFFu);
        } else {
            // bits 32..63 of the hash; (seedmix ^ base) is the same for the
            // whole tile, so it is computed once per tile
            const uint32_t hi = splitmix64_hi_state(((uint32_t)seedmix ^ base) ^ koff,
                                                    (uint32_t)(seedmix >> 32));
            if constexpr (sizeof(T) == 1) return (T)(hi >> 24);
            else return (float)(hi >> 8) * (1.0f / 16777216.0f);
        }
    }
};

__device__ __forceinline__ bool in_gasket(uint32_t x, uint32_t y) { return (x & y) == 0u; }

}  // namespace sg
