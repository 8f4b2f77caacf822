"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
the volume 3^r (Section III-A, Lemma 1), Lucas's theorem (Pascal's triangle
mod 2 built by the addition recurrence), the packing orthotope of Lemma 2,
lambda being a bijection onto the non-empty tiles (Theorem 1), hand-worked
fixtures, published SplitMix64 vectors, Conway's Life computed by a 2-D
convolution, and the graph Laplacian of the gasket built with scipy.sparse.
"""
import math

import numpy as np
import pytest

from conftest import read_golden_rows


# ---------------------------------------------------------------- membership

@pytest.mark.parametrize("r", range(0, 13))
def test_volume_is_3_pow_r(orc, r):
    # Section III-A: V = k^r with k = 3 for the gasket
    assert orc.count_members(r) == 3 ** r


def test_volume_level16_brute_force(orc):
    # Lemma 1 at the largest level the paper ran (n = 2^16): 4.3e9 tests
    assert orc.count_members(16) == 3 ** 16 == 43046721


def test_hausdorff_exponent(orc):
    # Lemma 1: 3^r = n^H with H = log2 3
    for r in range(1, 13):
        n = 2 ** r
        assert math.isclose(orc.count_members(r), n ** math.log2(3), rel_tol=1e-9)


@pytest.mark.parametrize("r", range(0, 11))
def test_recursion_equals_bitwise(orc, r):
    # the 3-copy construction and the closed form (x & y) == 0 agree
    assert np.array_equal(orc.gasket_recursive(r), orc.member_grid(r))


def _pascal_mod2(n: int) -> np.ndarray:
    # P[y][x] = C(x+y, x) mod 2 by the addition recurrence
    # P[y][x] = P[y-1][x] + P[y][x-1], P[0][.] = P[.][0] = 1
    p = np.zeros((n, n), dtype=np.uint8)
    p[0, :] = 1
    for y in range(1, n):
        p[y] = np.bitwise_xor.accumulate(p[y - 1])
    return p


@pytest.mark.parametrize("r", [0, 1, 2, 5, 8, 10])
def test_lucas_pascal_mod2(orc, r):
    # Lucas: C(x+y, x) is odd iff adding x and y makes no carry iff x & y == 0
    assert np.array_equal(_pascal_mod2(1 << r), orc.member_grid(r))
    assert np.array_equal(_pascal_mod2(1 << r), orc.gasket_recursive(r))


def test_paper_orientation_is_vertical_mirror(orc):
    # Section III-D tests x & (n-1-y) == 0 with y pointing down
    for r in range(0, 6):
        n = 1 << r
        for y in range(n):
            for x in range(n):
                assert orc.member_paper(r, x, y) == orc.member(x, n - 1 - y)


# ------------------------------------------------------------------- lambda

@pytest.mark.parametrize("rb", range(0, 13))
def test_pi_extent_lemma2(orc, rb):
    # Lemma 2: the level-rb gasket packs into 3^ceil(rb/2) x 3^floor(rb/2)
    wx, wy = orc.pi_extent(rb)
    assert sorted((wx, wy)) == sorted((3 ** ((rb + 1) // 2), 3 ** (rb // 2)))
    assert wx * wy == 3 ** rb


def test_lambda_hand_worked_rb2(orc):
    rows = read_golden_rows("lambda_rb2.txt")
    assert len(rows) == 9
    for wx, wy, lx, ly in rows:
        assert orc.lambda_paper(2, int(wx), int(wy)) == (int(lx), int(ly))


def test_lambda_rb1_is_the_three_cells(orc):
    # Pi is 1 x 3 at rb = 1; the paper-orientation gasket is (0,0),(0,1),(1,1)
    got = [orc.lambda_paper(1, 0, wy) for wy in range(3)]
    assert got == [(0, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("rb", range(0, 13))
def test_lambda_is_a_bijection_onto_the_block_gasket(orc, rb):
    # Theorem 1: every omega of Pi maps to a distinct member of the level-rb
    # gasket (paper orientation) and all 3^rb members are reached
    wx_e, wy_e = orc.pi_extent(rb)
    nb = 1 << rb
    if rb <= 6:
        seen = set()
        for wy in range(wy_e):
            for wx in range(wx_e):
                lx, ly = orc.lambda_paper(rb, wx, wy)
                assert orc.member_paper(rb, lx, ly)
                seen.add((lx, ly))
        assert len(seen) == 3 ** rb
    bx, by = orc.block_map(rb)
    assert len(bx) == 3 ** rb
    assert np.all((bx & by) == 0) and np.all(bx < nb) and np.all(by < nb)
    keys = by.astype(np.int64) * nb + bx
    assert len(np.unique(keys)) == 3 ** rb


@pytest.mark.parametrize("rb", [0, 1, 2, 5, 8, 11])
def test_interleaved_order_is_a_bijection_of_pi(orc, rb):
    # dealing q's base-3 digits alternately to omega_y and omega_x visits
    # every omega of Pi once, so both walking orders launch the same tiles
    wx_e, wy_e = orc.pi_extent(rb)
    seen = set()
    for q in range(3 ** rb):
        wx, wy = orc.omega_of_index(rb, q, orc.ORDER_INTERLEAVED)
        assert wx < wx_e and wy < wy_e
        seen.add((wx, wy))
    assert len(seen) == 3 ** rb
    a = orc.block_map(rb, orc.ORDER_ROWMAJOR)
    b = orc.block_map(rb, orc.ORDER_INTERLEAVED)
    ka = set(zip(a[0].tolist(), a[1].tolist()))
    kb = set(zip(b[0].tolist(), b[1].tolist()))
    assert ka == kb and len(kb) == 3 ** rb


def test_interleaved_order_hand_worked():
    # rb = 2: q = 3*d1 + d0, omega_y = d0, omega_x = d1; with the rb = 2 table
    # q = 5 (d0 = 2, d1 = 1): omega = (1, 2) -> lambda = (1, 3)
    # rb = 4: q = 63 = 2*27 + 1*9 + 0*3 + 0 has digits d0..d3 = 0, 0, 1, 2, so
    # omega_y = d0 + 3*d2 = 3 and omega_x = d1 + 3*d3 = 6
    import oracle
    assert oracle.omega_of_index(2, 5, oracle.ORDER_INTERLEAVED) == (1, 2)
    assert oracle.omega_of_index(4, 63, oracle.ORDER_INTERLEAVED) == (6, 3)
    lx, ly = oracle.lambda_paper(2, 1, 2)
    assert (lx, ly) == (1, 3)
    assert oracle.block_of_index(2, 5, oracle.ORDER_INTERLEAVED) == (1, 0)


@pytest.mark.parametrize("r,s", [(4, 1), (6, 2), (8, 3), (9, 4), (10, 4),
                                 (10, 5), (10, 6), (12, 4)])
def test_lambda_tiles_are_exactly_the_nonempty_tiles(orc, r, s):
    # the block-space gasket of side n_b = n / rho is the set of rho-tiles
    # that hold at least one cell, and each holds the level-s gasket (3^s cells)
    rho, rb = 1 << s, r - s
    nb = 1 << rb
    g = orc.member_grid(r).reshape(nb, rho, nb, rho)
    per_tile = g.sum(axis=(1, 3))                     # [by, bx]
    nonempty = set(zip(*np.nonzero(per_tile)))
    bx, by = orc.block_map(rb)
    assert set(zip(by.tolist(), bx.tolist())) == {(int(a), int(b)) for a, b in nonempty}
    assert np.all(per_tile[by, bx] == 3 ** s)


@pytest.mark.parametrize("r,s", [(6, 2), (8, 3), (10, 4), (10, 5)])
def test_launch_counts(orc, r, s):
    # Theorem 2 / Lemma 1: lambda launches 3^(r-s) blocks of rho^2 slots,
    # the bounding box n^2 slots; both find the same 3^r useful cells
    lam, useful = orc.launch_counts(r, s, orc.MAP_LAMBDA)
    bb, useful_bb = orc.launch_counts(r, s, orc.MAP_BBOX)
    lut, useful_lut = orc.launch_counts(r, s, orc.MAP_LAMBDA_LUT)
    assert useful == useful_bb == useful_lut == 3 ** r
    assert lam == 3 ** (r - s) * 4 ** s
    assert bb == 4 ** r
    assert lut == 3 ** r
    # O(n^H): lambda's slots stay within the constant (4/3)^s of n^log2(3)
    assert lam <= (4 / 3) ** s * (2 ** r) ** math.log2(3) * (1 + 1e-9)


# ------------------------------------------------------------ values / hash

def test_splitmix64_published_vectors(orc):
    gamma = 0x9E3779B97F4A7C15
    for seed, k, out in read_golden_rows("splitmix64_vectors.txt"):
        state = (int(seed) + int(k) * gamma) % 2**64
        assert orc.splitmix64_next(state) == int(out)


def test_cell_hash_definition(orc):
    # key = y*n + x, state = seed*gamma ^ key: the cell whose key is 1234567
    # at n = 2^16 (x = 54919, y = 18) with seed 0 is the generator seeded
    # with 1234567, whose first output is published
    assert 18 * 65536 + 54919 == 1234567
    assert orc.cell_hash(16, 54919, 18, 0) == 6457827717110365317
    assert orc.cell_hash(5, 0, 0, 0) == 0xE220A8397B1DCDAF


def _written_mask(orc, r, dtype, vk, value):
    n = 1 << r
    a = np.full((n, n), 0xA5 if dtype == np.uint8 else -7.0, dtype=dtype)
    b = np.full((n, n), 0x5A if dtype == np.uint8 else -9.0, dtype=dtype)
    orc.map_write(r, a, vk, value)
    orc.map_write(r, b, vk, value)
    return a, a == b


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
@pytest.mark.parametrize("r", [0, 1, 3, 7, 10])
def test_write_touches_exactly_the_gasket(orc, r, dtype):
    # Section IV: the pass writes every gasket cell and nothing else
    n = 1 << r
    a, written = _written_mask(orc, r, dtype, orc.VAL_HASH, 1)
    assert int(written.sum()) == 3 ** r
    ys, xs = np.nonzero(written)
    assert np.all((xs & ys) == 0)


def test_write_values_hand_cases(orc):
    r = 5
    n = 1 << r
    g = np.zeros((n, n), dtype=np.uint8)
    orc.map_write(r, g, orc.VAL_LINEAR31, 0)
    assert g[0, 3] == 93                       # 3*31 + 0
    assert g[3, 0] == 3                        # 0*31 + 3
    assert g[2, 5] == 157                      # 5*31 + 2
    assert g[2, 9] == (9 * 31 + 2) - 256       # wraps to 25
    assert g[1, 1] == 0                        # off the gasket: untouched
    h = np.zeros((n, n), dtype=np.uint8)
    orc.map_write(r, h, orc.VAL_HASH, 0)
    assert h[0, 0] == 0xE2                     # top byte of 0xE220A839...
    f = np.zeros((n, n), dtype=np.float32)
    orc.map_write(r, f, orc.VAL_HASH, 0)
    assert f[0, 0] == np.float32(0xE220A8 / 2**24)
    c = np.zeros((n, n), dtype=np.float32)
    orc.map_write(r, c, orc.VAL_CONST, int(np.float32(2.5).view(np.uint32)))
    assert c.sum() == 2.5 * 3 ** r


def test_write_band_equals_rows_of_full(orc):
    r, n = 9, 512
    full = np.zeros((n, n), dtype=np.float32)
    orc.map_write(r, full, orc.VAL_HASH, 3)
    band = np.zeros((100, n), dtype=np.float32)
    orc.map_write(r, band, orc.VAL_HASH, 3, y0=200, y1=300)
    assert np.array_equal(band, full[200:300])


# ----------------------------------------------------------------------- CA

def _life_by_convolution(state: np.ndarray, mask: np.ndarray) -> np.ndarray:
    from scipy.signal import convolve2d
    k = np.ones((3, 3), dtype=np.int64)
    k[1, 1] = 0
    count = convolve2d(state.astype(np.int64), k, mode="same", boundary="fill",
                       fillvalue=0)
    nxt = (count == 3) | ((state == 1) & (count == 2))
    return (nxt & (mask == 1)).astype(np.uint8)


@pytest.mark.parametrize("r,p,seed", [(3, 0.5, 0), (6, 0.5, 0), (8, 0.3, 0),
                                      (9, 0.5, 7)])
def test_ca_equals_masked_life(orc, r, p, seed):
    # with 0 off the gasket, the gasket-restricted rule is plain Life with a
    # zero (non-wrapping) border, masked to the gasket
    from paper_1706_04552_gb300 import inputs
    mask = orc.member_grid(r)
    s = inputs.ca_seed_grid(r, p, seed)
    for _ in range(6):
        ref = _life_by_convolution(s, mask)
        s = orc.ca_step(r, s)
        assert np.array_equal(s, ref)


def test_ca_hand_cases(orc):
    for r in (0, 1, 4):
        n = 1 << r
        dead = np.zeros((n, n), dtype=np.uint8)
        assert not orc.ca_step(r, dead).any()
    full = orc.member_grid(1)                     # all 3 cells alive
    assert np.array_equal(orc.ca_step(1, full), full)
    rows = read_golden_rows("ca_r2_hand.txt")
    i_in = rows.index(["in"])
    i_out = rows.index(["out"])
    a = np.array(rows[i_in + 1:i_out], dtype=np.uint8)
    b = np.array(rows[i_out + 1:], dtype=np.uint8)
    assert np.array_equal(orc.ca_step(2, a), b)
    assert np.array_equal(orc.ca_step(2, b), b)   # still life


def test_ca_region_light_cone(orc):
    # a region of radius >= t around a cell reproduces that cell after t steps
    from paper_1706_04552_gb300 import inputs
    r, t = 8, 6
    n = 1 << r
    s_full = orc.ca_steps(r, inputs.ca_seed_grid(r, 0.4, 5), t)
    rng = np.random.default_rng(1)
    xs, ys = inputs.gasket_cells(r)
    for i in rng.choice(len(xs), 25, replace=False):
        x, y = int(xs[i]), int(ys[i])
        R = t + 1
        x0, y0 = x - R, y - R
        win = inputs.ca_seed_region(r, 0.4, 5, x0, y0, 2 * R + 1, 2 * R + 1)
        win = orc.ca_steps(r, win, t, x0, y0)
        assert win[R, R] == s_full[y, x]
    assert n == 256


# ---------------------------------------------------------------- diffusion

def test_diffusion_hand_r1(orc):
    u = np.zeros((2, 2))
    u[0, 0] = 1.0
    for step, a, b, c in read_golden_rows("diffusion_r1_hand.txt"):
        if int(step) > 0:
            u = orc.diffuse_step(1, u, 0.2)
        assert math.isclose(u[0, 0], float(a), abs_tol=1e-15)
        assert math.isclose(u[0, 1], float(b), abs_tol=1e-15)
        assert math.isclose(u[1, 0], float(c), abs_tol=1e-15)
        assert u[1, 1] == 0.0


@pytest.mark.parametrize("r", [2, 5, 8])
def test_diffusion_matches_sparse_laplacian(orc, r):
    # u' = (I - alpha L) u with L = D - A the graph Laplacian of the gasket's
    # 4-neighbour graph, assembled with scipy.sparse
    import scipy.sparse as sp
    from paper_1706_04552_gb300 import inputs
    n = 1 << r
    xs, ys = inputs.gasket_cells(r)
    idx = -np.ones((n, n), dtype=np.int64)
    idx[ys, xs] = np.arange(len(xs))
    rows, cols = [], []
    for dx, dy in ((1, 0), (0, 1)):
        nx, ny = xs + dx, ys + dy
        ok = (nx < n) & (ny < n)
        ok[ok] &= idx[ny[ok], nx[ok]] >= 0
        a, b = idx[ys[ok], xs[ok]], idx[ny[ok], nx[ok]]
        rows += [a, b]
        cols += [b, a]
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(xs),) * 2)
    L = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    u0 = inputs.uniform_grid(r, 0).astype(np.float64)
    v = u0[ys, xs]
    u = u0
    for _ in range(5):
        v = v - 0.2 * (L @ v)
        u = orc.diffuse_step(r, u, 0.2)
        assert np.max(np.abs(u[ys, xs] - v)) < 1e-14
    off = np.ones((n, n), dtype=bool)
    off[ys, xs] = False
    assert not u[off].any()


@pytest.mark.parametrize("r", [4, 7, 9])
def test_diffusion_invariants(orc, r):
    from paper_1706_04552_gb300 import inputs
    u = inputs.uniform_grid(r, 0).astype(np.float64)
    mask = orc.member_grid(r).astype(bool)
    total, lo, hi = u.sum(), u[mask].min(), u[mask].max()
    for _ in range(20):
        u = orc.diffuse_step(r, u, 0.2)
        # each edge exchanges 0.2*(u_j - u_i) symmetrically: mass conserved
        assert abs(u.sum() - total) <= 1e-12 * total
        # convex update (weights 1 - 0.2*deg >= 0.2): no new extrema
        assert u[mask].min() >= lo - 1e-15 and u[mask].max() <= hi + 1e-15
    c = np.where(mask, 0.75, 0.0)
    assert np.array_equal(orc.diffuse_step(r, c, 0.2), c)


def test_diffusion_region_light_cone(orc):
    from paper_1706_04552_gb300 import inputs
    r, t = 8, 7
    full = orc.diffuse_steps(r, inputs.uniform_grid(r, 2), t)
    xs, ys = inputs.gasket_cells(r)
    rng = np.random.default_rng(3)
    for i in rng.choice(len(xs), 25, replace=False):
        x, y = int(xs[i]), int(ys[i])
        R = t + 1
        win = inputs.uniform_region(r, 2, x - R, y - R, 2 * R + 1, 2 * R + 1)
        win = orc.diffuse_steps(r, win, t, 0.2, x - R, y - R)
        assert win[R, R] == full[y, x]


def test_write_expected_at_matches_full_pass(orc):
    # the sampled form agrees with the brute-force pass cell by cell
    r, n = 8, 256
    rng = np.random.default_rng(0)
    before = rng.integers(0, 256, (n, n), dtype=np.uint8)
    full = before.copy()
    orc.map_write(r, full, orc.VAL_HASH, 9)
    ys, xs = np.divmod(np.arange(n * n), n)
    got = orc.write_expected_at(r, np.uint8, orc.VAL_HASH, 9, xs, ys, before.ravel())
    assert np.array_equal(got, full.ravel())


# --------------------------------------------------------------------------
# Compact storage
# --------------------------------------------------------------------------

def test_compact_layout_hand_worked(orc):
    rows = read_golden_rows("compact_hand.txt")
    cases = {}
    for r, s, order, i, x, y in rows:
        cases.setdefault((int(r), int(s), int(order)), []).append((int(i), int(x), int(y)))
    assert len(rows) == 9 + 9 + 27
    for (r, s, order), cells in cases.items():
        xs, ys = orc.compact_cells(r, s, order)
        assert len(xs) == 3 ** r == len(cells)
        for i, x, y in cells:
            assert (int(xs[i]), int(ys[i])) == (x, y), (r, s, order, i)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("r", range(0, 10))
def test_compact_layout_is_a_bijection_onto_the_gasket(orc, r, order):
    # every element holds a distinct gasket cell and all 3^r cells appear
    n = 1 << r
    for s in range(0, min(r, 6) + 1):
        xs, ys = orc.compact_cells(r, s, order)
        assert len(xs) == 3 ** r
        assert not np.any(xs & ys)
        assert xs.max(initial=0) < n and ys.max(initial=0) < n
        assert len(np.unique(ys * n + xs)) == 3 ** r


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("r,s", [(3, 1), (6, 2), (8, 4), (9, 6), (10, 5)])
def test_compact_tiles_are_runs_in_launch_order(orc, r, s, order):
    # element block q*3^s .. (q+1)*3^s - 1 lies in tile q of the block map,
    # and inside it the cells come row by row, left to right
    xs, ys = orc.compact_cells(r, s, order)
    bx, by = orc.block_map(r - s, order)
    c = 3 ** s
    tx = (xs.reshape(-1, c) & ((1 << s) - 1)).astype(np.int64)
    ty = (ys.reshape(-1, c) & ((1 << s) - 1)).astype(np.int64)
    assert np.array_equal(xs.reshape(-1, c) >> np.uint64(s), np.repeat(bx[:, None], c, 1))
    assert np.array_equal(ys.reshape(-1, c) >> np.uint64(s), np.repeat(by[:, None], c, 1))
    key = ty * (1 << s) + tx
    assert np.all(np.diff(key, axis=1) > 0)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("r", [0, 1, 3, 6])
def test_compact_single_tile_is_the_row_major_member_list(orc, r, order):
    # with one tile (s = r) the compact order is the gasket read row by row,
    # which numpy's nonzero gives for the membership mask
    xs, ys = orc.compact_cells(r, r, order)
    ny, nx = np.nonzero(orc.member_grid(r))
    assert np.array_equal(xs, nx.astype(np.uint64)) and np.array_equal(ys, ny.astype(np.uint64))


@pytest.mark.parametrize("order", [0, 1])
def test_compact_unit_tiles_follow_the_block_map(orc, order):
    # with 1 x 1 tiles (s = 0) element q is block q itself
    for r in range(0, 8):
        xs, ys = orc.compact_cells(r, 0, order)
        bx, by = orc.block_map(r, order)
        assert np.array_equal(xs, bx.astype(np.uint64)) and np.array_equal(ys, by.astype(np.uint64))


def test_compact_pack_unpack_round_trip(orc):
    r, s, n = 7, 3, 128
    rng = np.random.default_rng(4)
    g = rng.integers(0, 256, (n, n), dtype=np.uint8)
    c = orc.compact_pack(r, s, g)
    assert c.shape == (3 ** r,)
    back = orc.compact_unpack(r, s, c, np.zeros_like(g))
    mask = orc.member_grid(r).astype(bool)
    assert np.array_equal(back, np.where(mask, g, 0))
    assert np.array_equal(orc.compact_pack(r, s, back), c)


def test_compact_steps_are_the_embedded_steps(orc):
    # the compact CA and diffusion steps stand for the embedded ones: same
    # multiset of cell values, placed by the layout
    r, s, n = 6, 2, 64
    from paper_1706_04552_gb300 import inputs
    g = inputs.ca_seed_grid(r, 0.4, 3)
    c = orc.compact_pack(r, s, g)
    want = orc.ca_step(r, g)
    got = orc.compact_unpack(r, s, orc.compact_ca_step(r, s, c), np.zeros_like(g))
    assert np.array_equal(got, want)
    u = inputs.uniform_grid(r, 3)
    cu = orc.compact_pack(r, s, u)
    want = orc.diffuse_step(r, u, 0.2)
    got = orc.compact_unpack(r, s, orc.compact_diffuse_step(r, s, cu, 0.2),
                             np.zeros((n, n)))
    assert np.array_equal(got, want)
    # the total over the gasket is conserved in the compact form too
    assert abs(orc.compact_diffuse_step(r, s, cu).sum() - cu.astype(np.float64).sum()) < 1e-9
