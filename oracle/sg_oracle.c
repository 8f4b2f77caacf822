/*
 * sg_oracle.c -- CPU oracle for the embedded Sierpinski-gasket hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  The product
 * library never links, loads or calls anything in this directory, and this
 * file shares no code, header, table or constant generator with it.
 *
 * Paper: C. A. Navarro, B. Bustos, R. Vega, N. Hitschfeld, "Block-space GPU
 * Mapping for Embedded Sierpinski Gasket Fractals" (arXiv:1706.04552).
 *
 * Conventions (the paper's readings are listed in the design notes):
 *   n = 2^r, cells (x, y) with x the column, y the row, row-major storage,
 *   index y*n + x.  The gasket G_r is the set of cells with (x & y) == 0.
 *   The paper draws the same gasket mirrored vertically (origin top-left, y
 *   growing downwards, membership x & (n-1-y) == 0, Section III-D); its
 *   lambda map is computed here in the paper's orientation and mirrored.
 *
 * Every function is single-threaded straight-line C: loops over the whole
 * grid (or a rectangular region of it) in the order the definition reads.
 * Floating point is double.  Nothing is blocked, fused or reordered.
 *
 * Parity status: every function below is pinned by the CPU tests (closed
 * forms, brute force, published test vectors, hand-worked cases, and
 * independent library formulations); none is "parity unpinned".
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define OR_U8 0
#define OR_F32 1
#define OR_VAL_CONST 0
#define OR_VAL_LINEAR31 1
#define OR_VAL_HASH 2
#define OR_MAP_LAMBDA 0
#define OR_MAP_BBOX 1
#define OR_MAP_LAMBDA_LUT 2
#define OR_MAP_LAMBDA_UNROLL 3

/* ------------------------------------------------------------------------ */
/* Membership                                                                */
/* ------------------------------------------------------------------------ */

/* Gasket membership, bitwise closed form (the embedded layout of Section I,
 * in the orientation (x & y) == 0). */
int or_member(uint64_t x, uint64_t y) { return (x & y) == 0; }

/* Gasket membership in the paper's own orientation, Section III-D (Bounding
 * Sub-boxes): a cell is inside iff x & (n - 1 - y) == 0. */
int or_member_paper(int r, uint64_t x, uint64_t y)
{
    uint64_t n = (uint64_t)1 << r;
    return (x & (n - 1 - y)) == 0;
}

/* Gasket of level r built by the recursive construction of Section I and
 * Section III-A: level 0 is one cell, level k+1 is three copies of level k at
 * half scale.  In the (x & y) == 0 orientation the copies sit at offsets
 * (0,0), (2^k,0) and (0,2^k).  bm is an n*n byte map, set to 1 on members. */
void or_gasket_recursive(int r, uint8_t *bm)
{
    uint64_t n = (uint64_t)1 << r;
    memset(bm, 0, (size_t)(n * n));
    bm[0] = 1;
    for (int k = 0; k < r; ++k) {
        uint64_t h = (uint64_t)1 << k;
        for (uint64_t y = 0; y < h; ++y)
            for (uint64_t x = 0; x < h; ++x)
                if (bm[y * n + x]) {
                    bm[y * n + (x + h)] = 1;   /* copy to the right */
                    bm[(y + h) * n + x] = 1;   /* copy below        */
                }
    }
}

/* Volume of the level-r gasket by brute force over the whole n x n box
 * (Section III-A: the volume is 3^r). */
uint64_t or_count_members(int r)
{
    uint64_t n = (uint64_t)1 << r, c = 0;
    for (uint64_t y = 0; y < n; ++y)
        for (uint64_t x = 0; x < n; ++x)
            c += (uint64_t)or_member(x, y);
    return c;
}

/* ------------------------------------------------------------------------ */
/* The block-space map lambda(omega), Theorem 1                              */
/* ------------------------------------------------------------------------ */

static uint64_t ipow3(int k)
{
    uint64_t p = 1;
    for (int i = 0; i < k; ++i) p *= 3;
    return p;
}

/* Extent of the parallel space Pi: omega_x < 3^floor(rb/2), omega_y <
 * 3^ceil(rb/2).  (The helper beta reads omega_x at even levels and omega_y
 * at odd levels, so these are the digit counts it consumes.) */
void or_pi_extent(int rb, uint64_t *wx_extent, uint64_t *wy_extent)
{
    *wx_extent = ipow3(rb / 2);
    *wy_extent = ipow3((rb + 1) / 2);
}

/* lambda(omega) exactly as Theorem 1 states it, in the paper's orientation.
 * For every level mu = 1..rb:
 *   beta_mu  = floor((omega_x*((mu+1) mod 2) + omega_y*(mu mod 2)) /
 *                    3^(ceil(mu/2)-1)) mod 3                (Eq. beta)
 *   Dx = floor(beta/2),  Dy = beta - floor(beta/2)            (Eq. Delta)
 *   tau_x = Dx * 2^(mu-1), tau_y = Dy * 2^(mu-1)              (Eq. tau)
 * and lambda = (sum of tau_x, sum of tau_y)                   (Eq. lambda). */
void or_lambda_paper(int rb, uint64_t wx, uint64_t wy, uint64_t *lx, uint64_t *ly)
{
    uint64_t sx = 0, sy = 0;
    for (int mu = 1; mu <= rb; ++mu) {
        uint64_t operand = wx * (uint64_t)((mu + 1) % 2) + wy * (uint64_t)(mu % 2);
        uint64_t divisor = ipow3((mu + 1) / 2 - 1);       /* 3^(ceil(mu/2)-1) */
        uint64_t beta = (operand / divisor) % 3;
        uint64_t dx = beta / 2;
        uint64_t dy = beta - beta / 2;
        uint64_t tau_x = dx * ((uint64_t)1 << (mu - 1));
        uint64_t tau_y = dy * ((uint64_t)1 << (mu - 1));
        sx += tau_x;
        sy += tau_y;
    }
    *lx = sx;
    *ly = sy;
}

/* The point omega of Pi that launch index q names, for two walking orders.
 *   order 0 (row-major): omega = (q mod Wx, q div Wx), the paper's 2-D grid
 *     read row by row.
 *   order 1 (interleaved): the base-3 digits of q, least significant first,
 *     are dealt alternately to omega_y (digits 0, 2, 4, ...) and omega_x
 *     (digits 1, 3, 5, ...). */
void or_omega_of_index(int rb, int order, uint64_t q, uint64_t *wx, uint64_t *wy)
{
    if (order == 0) {
        uint64_t wxe, wye;
        or_pi_extent(rb, &wxe, &wye);
        *wx = q % wxe;
        *wy = q / wxe;
        return;
    }
    uint64_t x = 0, y = 0, px = 1, py = 1;
    for (int d = 0; d < rb; ++d) {
        uint64_t digit = q % 3;
        q /= 3;
        if (d % 2 == 0) { y += digit * py; py *= 3; }
        else            { x += digit * px; px *= 3; }
    }
    *wx = x;
    *wy = y;
}

/* Block coordinate of launch index q in the (x & y) == 0 orientation: the
 * paper's lambda of omega(q), mirrored vertically: by = n_b - 1 - lambda_y. */
void or_block_of_index(int rb, int order, uint64_t q, uint64_t *bx, uint64_t *by)
{
    uint64_t wx, wy, lx, ly;
    or_omega_of_index(rb, order, q, &wx, &wy);
    or_lambda_paper(rb, wx, wy, &lx, &ly);
    *bx = lx;
    *by = (((uint64_t)1 << rb) - 1) - ly;
}

/* All 3^rb block coordinates in launch order (the map the GPU decodes). */
void or_block_map(int rb, int order, uint32_t *bx, uint32_t *by)
{
    uint64_t total = ipow3(rb);
    for (uint64_t q = 0; q < total; ++q) {
        uint64_t a, b;
        or_block_of_index(rb, order, q, &a, &b);
        bx[q] = (uint32_t)a;
        by[q] = (uint32_t)b;
    }
}

/* Thread-slot accounting for one pass (Lemma 1, Theorem 2, Section III-D).
 * launched = cell slots the map's threads examine, one per thread in the
 * paper's model; useful = gasket cells.  Counted by walking the blocks the
 * map launches and the slots inside each, not by a closed form.
 *   lambda, bounding sub-boxes: every block is a full rho x rho sub-box;
 *   lambda, lookup table / further unrolling: only member slots are mapped;
 *   bounding box: every block of the n_b x n_b box, every slot. */
void or_launch_counts(int r, int s, int map, uint64_t *launched, uint64_t *useful)
{
    int rb = r - s;
    uint64_t rho = (uint64_t)1 << s, nb = (uint64_t)1 << rb;
    uint64_t l = 0, u = 0;
    if (map == OR_MAP_BBOX) {
        for (uint64_t by = 0; by < nb; ++by)
            for (uint64_t bx = 0; bx < nb; ++bx)
                for (uint64_t ty = 0; ty < rho; ++ty)
                    for (uint64_t tx = 0; tx < rho; ++tx) {
                        ++l;
                        u += (uint64_t)or_member(bx * rho + tx, by * rho + ty);
                    }
    } else {
        uint64_t blocks = ipow3(rb);
        for (uint64_t q = 0; q < blocks; ++q) {
            uint64_t bx, by;
            or_block_of_index(rb, 0, q, &bx, &by);
            for (uint64_t ty = 0; ty < rho; ++ty)
                for (uint64_t tx = 0; tx < rho; ++tx) {
                    int m = or_member(bx * rho + tx, by * rho + ty);
                    l += (map == OR_MAP_LAMBDA) ? 1u : (uint64_t)m;
                    u += (uint64_t)m;
                }
        }
    }
    *launched = l;
    *useful = u;
}

/* ------------------------------------------------------------------------ */
/* Values written by the map-and-write pass                                  */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the output produced by a generator whose state
 * is `state` -- advance the state by the golden gamma, then apply the
 * Mix13 finaliser. */
uint64_t or_splitmix64_next(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Per-cell hash: key = y*n + x, state = seed*gamma XOR key, h = SplitMix64
 * output of that state. */
uint64_t or_cell_hash(int r, uint64_t x, uint64_t y, uint64_t seed)
{
    uint64_t n = (uint64_t)1 << r;
    uint64_t key = y * n + x;
    return or_splitmix64_next((seed * 0x9E3779B97F4A7C15ULL) ^ key);
}

static uint8_t value_u8(int r, uint64_t x, uint64_t y, int vk, uint64_t vs)
{
    if (vk == OR_VAL_CONST) return (uint8_t)(vs & 0xFF);
    if (vk == OR_VAL_LINEAR31) return (uint8_t)((x * 31 + y) & 0xFF);
    return (uint8_t)(or_cell_hash(r, x, y, vs) >> 56);
}

static float value_f32(int r, uint64_t x, uint64_t y, int vk, uint64_t vs)
{
    if (vk == OR_VAL_CONST) {
        uint32_t bits = (uint32_t)(vs & 0xFFFFFFFFu);
        float f;
        memcpy(&f, &bits, sizeof f);
        return f;
    }
    if (vk == OR_VAL_LINEAR31) return (float)((x * 31 + y) & 0xFF);
    /* top 24 bits of the hash scaled by 2^-24: exact in float and double */
    double u = (double)(or_cell_hash(r, x, y, vs) >> 40) / 16777216.0;
    return (float)u;
}

/* Map-and-write pass of Section IV: every gasket cell receives v(x, y),
 * every other cell keeps its previous content.  Brute-force scan of the rows
 * [y0, y1) of the level-r grid; `band` holds those rows (pitch n elements). */
void or_map_write_rows(int r, int dtype, void *band, uint64_t y0, uint64_t y1,
                       int vk, uint64_t vs)
{
    uint64_t n = (uint64_t)1 << r;
    for (uint64_t y = y0; y < y1; ++y)
        for (uint64_t x = 0; x < n; ++x) {
            if (!or_member(x, y)) continue;
            uint64_t i = (y - y0) * n + x;
            if (dtype == OR_U8)
                ((uint8_t *)band)[i] = value_u8(r, x, y, vk, vs);
            else
                ((float *)band)[i] = value_f32(r, x, y, vk, vs);
        }
}

/* ------------------------------------------------------------------------ */
/* Per-cell stencils on the embedded gasket                                  */
/* ------------------------------------------------------------------------ */
/*
 * Both step functions update a rectangular region [x0, x0+w) x [y0, y0+h)
 * of the level-r grid, given the previous state of that same region (pitch
 * w).  Cells outside the region are read as 0, and region cells outside the
 * grid stay 0.  When the region is the whole
 * grid this is exactly the definition (neighbours outside the grid are
 * absent); on a smaller region a cell whose neighbourhood of radius t stays
 * inside the region is exact after t steps.
 */

static int in_grid(int64_t v, uint64_t n) { return v >= 0 && (uint64_t)v < n; }

/* Gasket-restricted Life-like B3/S23 step: a gasket cell is alive next iff
 * exactly 3 of its 8 in-grid gasket neighbours are alive, or it is alive and
 * exactly 2 are.  Cells off the gasket are 0.  Alive means state 1. */
void or_ca_step_region(int r, int64_t x0, int64_t y0, int64_t w, int64_t h,
                       const uint8_t *in, uint8_t *out)
{
    uint64_t n = (uint64_t)1 << r;
    for (int64_t j = 0; j < h; ++j)
        for (int64_t i = 0; i < w; ++i) {
            int64_t x = x0 + i, y = y0 + j;
            uint8_t next = 0;
            if (in_grid(x, n) && in_grid(y, n) && or_member((uint64_t)x, (uint64_t)y)) {
                int count = 0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0) continue;
                        int64_t nx = x + dx, ny = y + dy;
                        if (!in_grid(nx, n) || !in_grid(ny, n)) continue;
                        if (!or_member((uint64_t)nx, (uint64_t)ny)) continue;
                        int64_t li = nx - x0, lj = ny - y0;
                        if (li < 0 || li >= w || lj < 0 || lj >= h) continue;
                        if (in[lj * w + li] == 1) ++count;
                    }
                int alive = in[j * w + i] == 1;
                next = (uint8_t)((count == 3 || (alive && count == 2)) ? 1 : 0);
            }
            out[j * w + i] = next;
        }
}

/* Explicit diffusion step over the 4-neighbourhood restricted to the gasket:
 * N = in-grid 4-neighbours that are gasket cells, deg = |N|,
 * u' = u + alpha * (sum_{j in N} u_j - deg * u).  Off-gasket cells are 0.
 * deg depends only on the geometry, so it counts neighbours outside the
 * region too; only their values are unknown (read as 0). */
void or_diffuse_step_region(int r, int64_t x0, int64_t y0, int64_t w, int64_t h,
                            const double *in, double *out, double alpha)
{
    static const int dxs[4] = {-1, 1, 0, 0};
    static const int dys[4] = {0, 0, -1, 1};
    uint64_t n = (uint64_t)1 << r;
    for (int64_t j = 0; j < h; ++j)
        for (int64_t i = 0; i < w; ++i) {
            int64_t x = x0 + i, y = y0 + j;
            double next = 0.0;
            if (in_grid(x, n) && in_grid(y, n) && or_member((uint64_t)x, (uint64_t)y)) {
                double u = in[j * w + i], sum = 0.0;
                int deg = 0;
                for (int k = 0; k < 4; ++k) {
                    int64_t nx = x + dxs[k], ny = y + dys[k];
                    if (!in_grid(nx, n) || !in_grid(ny, n)) continue;
                    if (!or_member((uint64_t)nx, (uint64_t)ny)) continue;
                    ++deg;
                    int64_t li = nx - x0, lj = ny - y0;
                    if (li >= 0 && li < w && lj >= 0 && lj < h) sum += in[lj * w + li];
                }
                next = u + alpha * (sum - (double)deg * u);
            }
            out[j * w + i] = next;
        }
}

/* Expected content of listed cells after the map-and-write pass, for
 * checking a full-size grid at sampled cells: v(x, y) at gasket cells, the
 * cell's previous content (passed in `before`) elsewhere. */
void or_write_expected_at(int r, int dtype, int vk, uint64_t vs, uint64_t count,
                          const uint64_t *xs, const uint64_t *ys,
                          const void *before, void *out)
{
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t x = xs[i], y = ys[i];
        if (dtype == OR_U8)
            ((uint8_t *)out)[i] = or_member(x, y) ? value_u8(r, x, y, vk, vs)
                                                  : ((const uint8_t *)before)[i];
        else
            ((float *)out)[i] = or_member(x, y) ? value_f32(r, x, y, vk, vs)
                                                : ((const float *)before)[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Compact storage: the succinct blocked layout (Section II) with the        */
/* block-space map as its block order                                        */
/* ------------------------------------------------------------------------ */

/* The cell held by every element of a compact array at level r with tile
 * side 2^s, written to xs[i], ys[i] for i < 3^r:
 *   q = i div 3^s and e = i mod 3^s;
 *   (bx, by) = the block of launch index q (or_block_of_index, level r - s);
 *   (tx, ty) = the e-th cell of the level-s gasket {(tx & ty) == 0} when its
 *              2^s x 2^s square is read row by row;
 *   x = bx * 2^s + tx, y = by * 2^s + ty.
 * Every non-empty tile holds the same level-s pattern, so the tiles become
 * runs of 3^s consecutive elements in launch order.  The level-s cells are
 * listed once by scanning the square (rows top to bottom, each row left to
 * right) and keeping the members. */
void or_compact_cells(int r, int s, int order, uint64_t *xs, uint64_t *ys)
{
    uint64_t rho = (uint64_t)1 << s, per_tile = ipow3(s);
    uint64_t tiles = ipow3(r - s);
    uint64_t ltx[729], lty[729];          /* s <= 6: at most 3^6 cells */
    uint64_t m = 0;
    for (uint64_t ty = 0; ty < rho; ++ty)
        for (uint64_t tx = 0; tx < rho; ++tx)
            if (or_member(tx, ty)) { ltx[m] = tx; lty[m] = ty; ++m; }
    for (uint64_t q = 0; q < tiles; ++q) {
        uint64_t bx, by;
        or_block_of_index(r - s, order, q, &bx, &by);
        for (uint64_t e = 0; e < per_tile; ++e) {
            xs[q * per_tile + e] = bx * rho + ltx[e];
            ys[q * per_tile + e] = by * rho + lty[e];
        }
    }
}
