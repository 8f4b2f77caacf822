// sg_bits.cuh -- the bit-sliced B3/S23 CA on one staged tile, shared by the
// fused single-gasket kernel (sg_fused.cu) and the fused batch kernel
// (sg_batch.cu).
#pragma once

#include "sg_stencil.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// CA, bit-sliced.  In shared memory a staged row is a string of bits, one
// cell per bit (bit j of a row = column x0 - 16 + j: a 16-cell halo on each
// side, then padding to whole 32-bit words), and the B3/S23 rule runs on 32
// cells at a time: the eight neighbour planes (the rows above and below and
// the row itself, shifted by one column either way with funnel shifts) are
// summed by a tree of bitwise full adders, and the bits of the count decide
// the next state.  One warp owns one tile at a time, so the steps need only
// __syncwarp.  States are 0/1 bytes in HBM: 16-byte chunks are packed to 16
// bits when staged and unpacked when stored.
// ---------------------------------------------------------------------------
template <int S, int KH> struct BitShape {
    static constexpr int RHO = 1 << S;
    static constexpr int HW = RHO / 16 + 2;          // staged 16-cell half-words per row
    static constexpr int WPR = (HW + 1) / 2;         // 32-bit words per row
    static constexpr int ROWS = RHO + 2 * KH;
    static constexpr int WORDS = ROWS * WPR;
    // a buffer holds one pad word before and after the rows, so that a
    // row's neighbour words can be read at fixed offsets -1 / +1 (the pads'
    // contents are never used: edge words are masked off)
    static constexpr int BUFW = WORDS + 2;
    static constexpr int WARPS = kStencilThreads / 32;
    static constexpr uint32_t GROUP_MASK = StencilGroup<uint8_t, S>::GROUP_MASK;
};

// Bit i of the result = byte i of a chunk of 0/1 bytes.
__device__ __forceinline__ uint32_t pack16(uint4 c)
{
    // byte j of a word sits at bit 8j; two shifted ORs bring it to bit j
    auto nib = [](uint32_t w) {
        w |= w >> 7;
        w |= w >> 14;
        return w & 0xFu;
    };
    return nib(c.x) | (nib(c.y) << 4) | (nib(c.z) << 8) | (nib(c.w) << 12);
}

// Byte i of the result = bit i of b (0/1 bytes).
__device__ __forceinline__ uint4 unpack16(uint32_t b)
{
    // nib * (1 + 2^7 + 2^14 + 2^21) puts bit j of the nibble at bit 8j; the
    // four shifted copies do not overlap, so no carry disturbs them
    auto bytes = [](uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; };
    return make_uint4(bytes(b & 0xFu), bytes((b >> 4) & 0xFu), bytes((b >> 8) & 0xFu),
                      bytes((b >> 12) & 0xFu));
}

// Bits i of 16 with (i & yl) == 0 (yl = y mod 16): the gasket cells of a
// 16-cell chunk at a column x with (x & y) == 0, x a multiple of 16.
__device__ __forceinline__ uint32_t member_bits16(uint32_t yl)
{
    uint32_t m = 0xFFFFu;
    if (yl & 1u) m &= 0x5555u;
    if (yl & 2u) m &= 0x3333u;
    if (yl & 4u) m &= 0x0F0Fu;
    if (yl & 8u) m &= 0x00FFu;
    return m;
}

__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &sum,
                                         uint32_t &carry)
{
    sum = a ^ b ^ c;
    carry = (a & b) | (c & (a ^ b));
}

// Stage the tile at (x0, y0) with its halo as bits, and the gasket mask of
// every staged bit (0 off the grid, off the gasket and in padding).
template <int S, int KH>
__device__ __forceinline__ void bits_stage(uint32_t *bits, uint32_t *mask,
                                           const uint8_t *__restrict__ in, int r, int x0, int y0,
                                           int lane)
{
    using B = BitShape<S, KH>;
    constexpr int HPR = 2 * B::WPR;                  // half-words per row, padding included
    const int n = 1 << r;
    uint16_t *bh = reinterpret_cast<uint16_t *>(bits);
    uint16_t *mh = reinterpret_cast<uint16_t *>(mask);
#pragma unroll 4
    for (int i = lane; i < B::ROWS * HPR; i += 32) {
        const int row = i / HPR, h = i - row * HPR;
        const int x = x0 - 16 + 16 * h, y = y0 - KH + row;
        uint32_t v = 0u, m = 0u;
        if (h < B::HW && x >= 0 && y >= 0 && x < n && y < n && (x & y) == 0) {
            v = pack16(__ldg(reinterpret_cast<const uint4 *>(in + (((uint64_t)y << r) +
                                                                    (uint64_t)x))));
            m = member_bits16((uint32_t)y & 15u);
        }
        bh[i] = (uint16_t)v;
        mh[i] = (uint16_t)m;
    }
}

// Word w of a staged row and its left and right neighbour planes (bit j <-
// bit j-1 and bit j <- bit j+1).  p points at the word; its neighbours are
// read at p[-1] and p[+1].  At the row's ends those reads land in the
// previous or next row (or in a pad word), so the outermost staged column on
// each side takes a wrong neighbour.  That costs nothing: the staged halo is
// 16 columns wide and a wrong value moves one column per step, so after
// k <= 16 steps it has reached at most the column next to the tile -- the
// light cone that already limits every halo cell (their own neighbours
// outside the staged window are not there either).
struct BitRow {
    uint32_t v, l, r;
};
__device__ __forceinline__ BitRow bit_row(const uint32_t *p)
{
    const uint32_t v = p[0];
    return BitRow{v, __funnelshift_l(p[-1], v, 1), __funnelshift_r(v, p[1], 1)};
}

// One step over the window rows [s, ROWS - s): src -> dst.  The lanes form
// G = 32 / WPR groups; lane (g, w) updates word w of a run of consecutive
// rows, carrying down the run each row's horizontal sums: the 3-cell sum
// (l + v + r) serves the rows above and below it, the 2-cell sum (l + r) the
// row itself, so a row costs one full adder, one half adder and the merge:
//   count = up3 + mid2 + dn3 = s0 + 2 s1 + 4 (t1 + t2).
//
// For 64-tiles (three words a row) each lane instead takes whole rows, a run
// of about three: it loads a row's three words once, forms their neighbour
// planes in registers (the row's outermost bits take a 0 neighbour, as the
// light cone allows), and its loads fall on distinct banks (the lanes' rows
// are three rows, nine words, apart).  The adder tree is the same.
struct BitRow3 {
    uint32_t s[3], c[3];    // 3-cell sums (l + v + r) of each word: sum and carry
    uint32_t v[3], l[3], r[3];
};
__device__ __forceinline__ void bit_row3(const uint32_t *p, BitRow3 &o)
{
    const uint32_t v0 = p[0], v1 = p[1], v2 = p[2];
    o.v[0] = v0; o.v[1] = v1; o.v[2] = v2;
    o.l[0] = v0 << 1;
    o.l[1] = __funnelshift_l(v0, v1, 1);
    o.l[2] = __funnelshift_l(v1, v2, 1);
    o.r[0] = __funnelshift_r(v0, v1, 1);
    o.r[1] = __funnelshift_r(v1, v2, 1);
    o.r[2] = v2 >> 1;
#pragma unroll
    for (int w = 0; w < 3; ++w) full_add(o.l[w], o.v[w], o.r[w], o.s[w], o.c[w]);
}

template <int S, int KH>
__device__ __forceinline__ void bits_ca_step(const uint32_t *src, uint32_t *dst,
                                             const uint32_t *mask, int s, int lane)
{
    using B = BitShape<S, KH>;
    if constexpr (B::WPR == 3) {
        const int rows = B::ROWS - 2 * s, run = (rows + 31) / 32;
        const int first = s + lane * run;
        const int last = min(first + run, B::ROWS - s);
        if (first >= last) return;
        BitRow3 u, m, d;
        bit_row3(src + (first - 1) * 3, u);
        bit_row3(src + first * 3, m);
        for (int row = first; row < last; ++row) {
            bit_row3(src + (row + 1) * 3, d);
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                const uint32_t ms2 = m.l[w] ^ m.r[w], mc2 = m.l[w] & m.r[w];
                uint32_t s0, c1, t0, t1;
                full_add(u.s[w], ms2, d.s[w], s0, c1);
                full_add(u.c[w], mc2, d.c[w], t0, t1);
                const uint32_t s1 = t0 ^ c1, t2 = t0 & c1;
                dst[row * 3 + w] = (s0 | m.v[w]) & s1 & ~(t1 | t2) & mask[row * 3 + w];
            }
            u = m;
            m = d;
        }
        return;
    }
    constexpr int G = 32 / B::WPR;
    const int g = lane / B::WPR, w = lane - g * B::WPR;
    if (g >= G) return;                               // idle lanes (32 not a multiple of WPR)
    const int rows = B::ROWS - 2 * s, run = (rows + G - 1) / G;
    const int first = s + g * run;
    const int last = min(first + run, B::ROWS - s);
    if (first >= last) return;
    const uint32_t *p = src + (first - 1) * B::WPR + w;
    const BitRow u = bit_row(p);
    uint32_t us, uc;                                  // 3-sum of the row above
    full_add(u.l, u.v, u.r, us, uc);
    p += B::WPR;
    BitRow m = bit_row(p);
    uint32_t ms3, mc3;                                // 3-sum of the current row
    full_add(m.l, m.v, m.r, ms3, mc3);
    const uint32_t *pk = mask + first * B::WPR + w;
    uint32_t *po = dst + first * B::WPR + w;
#pragma unroll 2
    for (int row = first; row < last; ++row) {
        p += B::WPR;
        const BitRow d = bit_row(p);
        uint32_t ds3, dc3;
        full_add(d.l, d.v, d.r, ds3, dc3);
        const uint32_t ms2 = m.l ^ m.r, mc2 = m.l & m.r;   // 2-sum of the current row
        uint32_t s0, c1, t0, t1;
        full_add(us, ms2, ds3, s0, c1);
        full_add(uc, mc2, dc3, t0, t1);
        const uint32_t s1 = t0 ^ c1, t2 = t0 & c1;
        // alive next iff count is 3, or count is 2 and alive: s1 set, no
        // weight-4 bit, and s0 or the cell itself
        *po = (s0 | m.v) & s1 & ~(t1 | t2) & *pk;
        po += B::WPR;
        pk += B::WPR;
        us = ms3;
        uc = mc3;
        m = d;
        ms3 = ds3;
        mc3 = dc3;
    }
}

// Unpack the tile rows (rows [KH, KH + RHO), half-words 1 .. RHO/16) to HBM,
// whole 32-byte sectors where a tile row spans them.
template <int S, int KH>
__device__ __forceinline__ void bits_store(const uint32_t *bits, uint8_t *__restrict__ out,
                                           int r, int x0, int y0, int lane)
{
    using B = BitShape<S, KH>;
    constexpr int CPR = B::RHO / 16, HPR = 2 * B::WPR;
    const uint16_t *bh = reinterpret_cast<const uint16_t *>(bits);
    for (int i = lane; i < B::RHO * CPR; i += 32) {
        const int ty = i / CPR, cx = i - ty * CPR;
        const uint32_t x = (uint32_t)(x0 + 16 * cx), y = (uint32_t)(y0 + ty);
        if (!in_gasket(x & B::GROUP_MASK, y)) continue;
        const uint32_t v = bh[(KH + ty) * HPR + 1 + cx];
        *reinterpret_cast<uint4 *>(out + ((uint64_t)y << r) + x) = unpack16(v);
    }
}

// k steps of one tile by one warp: stage (tile + halo, from `in`), step in
// shared memory, store the tile to `out`.  st0 / st1 / mk: the warp's two
// state buffers and mask buffer, each pointing one word into a buffer of
// BitShape<S, KH>::BUFW words (the pads).
template <int S, int KH>
__device__ __forceinline__ void bits_tile_steps(uint32_t *st0, uint32_t *st1, uint32_t *mk,
                                                const uint8_t *__restrict__ in,
                                                uint8_t *__restrict__ out, int r, int x0, int y0,
                                                int k, int lane)
{
    bits_stage<S, KH>(st0, mk, in, r, x0, y0, lane);
    __syncwarp();
    for (int s = 1; s <= k; ++s) {
        bits_ca_step<S, KH>((s & 1) ? st0 : st1, (s & 1) ? st1 : st0, mk, s, lane);
        __syncwarp();
    }
    bits_store<S, KH>((k & 1) ? st1 : st0, out, r, x0, y0, lane);
    __syncwarp();                        // the buffers are read before the next staging
}

}  // namespace sg
