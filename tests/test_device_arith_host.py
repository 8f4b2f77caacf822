"""Host-side emulation of the device arithmetic, checked against the oracle.

The kernels decode lambda with per-lane fixed-point reciprocals, a 16-bit
mod-3 trick, a packed (x, y) reduction and an incremental walk of the launch
index; they build the lookup table with a row-major rank and map unrolled
slots with thread-level lambda.  These tests restate that integer
arithmetic in numpy exactly as the kernels do it and check it against the
oracle for every block index up to level 14, and every rho, so that the
index arithmetic is shown in range before the kernels run."""
import os
import re

import numpy as np
import pytest

import oracle

ORDERS = {0: "rowmajor", 1: "interleaved"}
HEADER = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1706_04552_gb300", "csrc",
                      "sg_device.cuh")


def _recip_table():
    """The reciprocals recip3(k) as the device header writes them."""
    with open(HEADER) as f:
        body = re.search(r"constexpr uint32_t recip3\(int k\)\s*\{(.*?)\}", f.read(),
                         re.S).group(1)
    tab = [0] * 8
    for k, v in re.findall(r"k == (\d) \? (\d+)u", body):
        tab[int(k)] = int(v)
    return tab


def test_reciprocal_table_is_exact_for_every_word():
    # entry k = ceil(2^32 / 3^k) (0 for k = 0, whose lane adds w instead), and
    # the high word of w * entry (+ w for k = 0) is floor(w / 3^k) for every
    # base-3 word w < 3^8
    tab = _recip_table()
    assert len(tab) == 8 and tab[0] == 0
    w = np.arange(3 ** 8, dtype=np.uint64)
    for k in range(8):
        if k:
            assert tab[k] == -(-(1 << 32) // 3 ** k) and tab[k] < (1 << 32)
        d = ((w * np.uint64(tab[k])) >> np.uint64(32)) + (w if k == 0 else 0)
        assert np.array_equal(d, w // np.uint64(3 ** k)), k


def _pi_word(order, rb):
    return 6561 if order == 1 else 3 ** (rb // 2)


def _decode(q, rb, order):
    """LambdaLane::decode over all lanes for launch indices q (uint64)."""
    W = np.uint64(_pi_word(order, rb))
    b = q // W
    a = q - b * W
    acc = np.zeros(len(q), dtype=np.uint64)
    tab = _recip_table()
    for lane in range(32):
        l = lane & 15
        digit = (l & 7) if order == 1 else (l >> 1)
        p = 3 ** digit
        recip = np.uint64(tab[digit])
        keep_w = np.uint64(0xFFFFFFFF if digit == 0 else 0)
        reads_b = (l >= 8) if order == 1 else (l & 1) == 0
        active = lane < 16 and l < rb
        w = b if reads_b else a
        assert np.all(w < 6561)                          # the reciprocal's range
        d = ((w * recip) >> np.uint64(32)) + (w & keep_w)
        assert np.all(d < 65536)                         # the mod-3 trick's range
        beta = d - np.uint64(3) * ((d * np.uint64(0xAAAB)) >> np.uint64(17))
        assert np.all(beta == (w // np.uint64(p)) % np.uint64(3))
        dx = beta >> np.uint64(1)
        dy = beta - dx
        if active:
            acc += (dx << np.uint64(l)) | (dy << np.uint64(l + 16))
    acc &= np.uint64(0xFFFFFFFF)
    bx = acc & np.uint64(0xFFFF)
    by = np.uint64((1 << rb) - 1) - (acc >> np.uint64(16))
    return bx.astype(np.uint32), by.astype(np.uint32)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("rb", list(range(0, 13)) + [14])
def test_lambda_decode_arithmetic_matches_oracle(rb, order):
    q = np.arange(3 ** rb, dtype=np.uint64)
    bx, by = _decode(q, rb, order)
    ebx, eby = oracle.block_map(rb, order)
    assert np.array_equal(bx, ebx) and np.array_equal(by, eby)
    assert np.all(bx < (1 << rb)) and np.all(by < (1 << rb))


@pytest.mark.parametrize("stride", [1, 7, 152 * 8, 9728, 12161])
def test_incremental_walk_of_the_launch_index(stride):
    # OmegaWalker: (a, b) = (q mod W, q div W) stepped by a fixed stride
    for W in (1, 3, 27, 243, 6561):
        for q0 in (0, 1, stride - 1, 5000):
            a, b = q0 % W, q0 // W
            sb, sa = stride // W, stride % W
            q = q0
            for _ in range(200):
                assert (a, b) == (q % W, q // W)
                a += sa
                b += sb
                if a >= W:
                    a -= W
                    b += 1
                q += stride


def _member_rowmajor(S, e):
    """member_rowmajor<S>(e): row by the halves' member counts, then tx by
    placing e's bits at the zero bits of ty."""
    ty, m = 0, 1
    for b in range(S - 1, -1, -1):
        clear = 2 * m * 3 ** b
        if e < clear:
            m *= 2
        else:
            e -= clear
            ty |= 1 << b
    tx = k = 0
    for b in range(S):
        if not (ty >> b) & 1:
            tx |= ((e >> k) & 1) << b
            k += 1
    return tx, ty


def _unrolled(S, e):
    WS = 3 ** (S // 2)
    wx, wy = e % WS, e // WS
    lx = ly = 0
    for mu in range(1, S + 1):
        w = wy if mu & 1 else wx
        for _ in range((mu + 1) // 2 - 1):
            w //= 3
        beta = w % 3
        dx = beta >> 1
        lx += dx << (mu - 1)
        ly += (beta - dx) << (mu - 1)
    return lx, (1 << S) - 1 - ly


@pytest.mark.parametrize("S", range(0, 7))
def test_lookup_table_entries_and_unrolled_slots(S):
    R = 1 << S
    # the table entries, in row-major order: every member exactly once
    members = [(tx, ty) for ty in range(R) for tx in range(R) if tx & ty == 0]
    assert [_member_rowmajor(S, e) for e in range(3 ** S)] == members
    cells = {_unrolled(S, e) for e in range(3 ** S)}
    assert len(cells) == 3 ** S
    assert all(x & y == 0 and 0 <= x < R and 0 <= y < R for x, y in cells)


# ------------------------------------------------------------------------
# The bit-sliced fused CA (sg_ca_steps), restated word for word in numpy:
# staging packs 16-byte chunks of 0/1 bytes to 16 bits, each step sums the
# eight neighbour planes with full adders, and the store unpacks bits back
# to bytes.  Run over every tile of a small gasket, it must reproduce k
# steps of the oracle.  (The kernel walks each word down a run of rows and
# carries the row sums along; the arithmetic per row is the one below.)
# ------------------------------------------------------------------------
_M32 = 0xFFFFFFFF


def _pack16(chunk):
    v = 0
    for j, w in enumerate(chunk.view("<u4")):
        w = int(w)
        w |= w >> 7
        w |= w >> 14
        v |= (w & 0xF) << (4 * j)
    return v


def _unpack16(b):
    out = []
    for j in range(4):
        nib = (b >> (4 * j)) & 0xF
        out.append(((nib * 0x00204081) & 0x01010101) & _M32)
    return np.array(out, dtype="<u4").view(np.uint8)


def _member_bits16(yl):
    m = 0xFFFF
    for bit, keep in ((1, 0x5555), (2, 0x3333), (4, 0x0F0F), (8, 0x00FF)):
        if yl & bit:
            m &= keep
    return m


def _full_add(a, b, c):
    return a ^ b ^ c, (a & b) | (c & (a ^ b))


def _bits_ca(r, S, KH, k, state):
    rho, n = 1 << S, 1 << r
    HW = rho // 16 + 2
    WPR = (HW + 1) // 2
    HPR, ROWS = 2 * WPR, rho + 2 * KH
    gmask = ~((32 if rho >= 32 else 16) - 1)
    out = np.zeros_like(state)
    bxs, bys = oracle.block_map(r - S, 1)
    for tbx, tby in zip(bxs.tolist(), bys.tolist()):
        x0, y0 = tbx << S, tby << S
        half = np.zeros((ROWS, HPR), dtype=np.uint64)
        mhalf = np.zeros((ROWS, HPR), dtype=np.uint64)
        for row in range(ROWS):
            for h in range(HPR):
                x, y = x0 - 16 + 16 * h, y0 - KH + row
                if h < HW and 0 <= x < n and 0 <= y < n and (x & y) == 0:
                    half[row, h] = _pack16(np.ascontiguousarray(state[y, x:x + 16]))
                    mhalf[row, h] = _member_bits16(y & 15)
        cur = half[:, 0::2] | (half[:, 1::2] << np.uint64(16))
        mask = mhalf[:, 0::2] | (mhalf[:, 1::2] << np.uint64(16))
        z = np.zeros(1, dtype=np.uint64)
        one, s31 = np.uint64(1), np.uint64(31)
        m32 = np.uint64(_M32)
        for s in range(1, k + 1):
            nxt = cur.copy()
            for row in range(s, ROWS - s):
                a, b, c = cur[row - 1], cur[row], cur[row + 1]
                planes = []
                for v in (a, b, c):
                    vl = np.concatenate([z, v[:-1]])
                    vr = np.concatenate([v[1:], z])
                    planes.append((((v << one) | (vl >> s31)) & m32,
                                   (v >> one) | ((vr << s31) & m32)))
                (aL, aR), (bL, bR), (cL, cR) = planes
                us, uc = _full_add(aL, a, aR)          # 3-sum of the row above
                ds, dc = _full_add(cL, c, cR)          # 3-sum of the row below
                ms, mc = bL ^ bR, bL & bR              # 2-sum of the row itself
                s0, c1 = _full_add(us, ms, ds)
                t0, t1 = _full_add(uc, mc, dc)
                s1, t2 = t0 ^ c1, t0 & c1
                nxt[row] = (s0 | b) & s1 & (~(t1 | t2) & m32) & mask[row]
            cur = nxt
        for ty in range(rho):
            for cx in range(rho // 16):
                x, y = x0 + 16 * cx, y0 + ty
                if ((x & gmask) & y) != 0:
                    continue
                h = 1 + cx
                bits = (int(cur[KH + ty, h // 2]) >> (16 * (h % 2))) & 0xFFFF
                out[y, x:x + 16] = _unpack16(bits)
    return out


@pytest.mark.parametrize("r,S,KH,k", [(6, 4, 4, 3), (7, 5, 8, 7), (8, 6, 16, 16),
                                      (6, 4, 16, 13)])
def test_bit_sliced_ca_restated_matches_oracle(r, S, KH, k):
    from paper_1706_04552_gb300 import inputs
    s0 = inputs.ca_seed_grid(r, 0.45, 21 + r)
    want = oracle.ca_steps(r, s0, k)
    assert np.array_equal(_bits_ca(r, S, KH, k, s0), want)


def test_pack_and_unpack_are_inverse_on_every_pattern():
    for b in range(1 << 16):
        chunk = _unpack16(b)
        assert set(chunk.tolist()) <= {0, 1}
        assert _pack16(chunk) == b


# ------------------------------------------------------------------------
# The fused diffusion's per-chunk degree word, restated: byte i = number of
# in-grid gasket 4-neighbours of cell (x + i, y), or 0xFF off the gasket;
# 0xFFFFFFFF for a chunk with no gasket cell.  Checked against brute force
# for every 4-cell chunk of the grid and its one-chunk border.
# ------------------------------------------------------------------------
def _spread4(m):
    return (m * 0x00204081) & 0x01010101


def _member_bits4(y):
    return (0x135F >> (4 * (y & 3))) & 0xF


def _chunk_degrees(x, y, n):
    if x < 0 or y < 0 or x >= n or y >= n or (x & y) != 0:
        return 0xFFFFFFFF
    m = _member_bits4(y)
    pl = int(x > 0 and ((x - 1) & y) == 0)
    pr = int(x + 4 < n and ((x + 4) & y) == 0)
    mu = _member_bits4(y - 1) if (y > 0 and (x & (y - 1)) == 0) else 0
    md = _member_bits4(y + 1) if (y + 1 < n and (x & (y + 1)) == 0) else 0
    ml, mr = ((m << 1) | pl) & 0xF, (m >> 1) | (pr << 3)
    deg = _spread4(ml) + _spread4(mr) + _spread4(mu) + _spread4(md)
    return (deg | (_spread4(~m & 0xF) * 0xFF)) & 0xFFFFFFFF


@pytest.mark.parametrize("r", [2, 3, 6])
def test_chunk_degree_words_match_brute_force(r):
    n = 1 << r
    mem = oracle.member_grid(r).astype(bool)

    def member(x, y):
        return 0 <= x < n and 0 <= y < n and bool(mem[y, x])
    for y in range(-1, n + 1):
        for x in range(-4, n + 4, 4):
            word = _chunk_degrees(x, y, n)
            if not any(member(x + i, y) for i in range(4)):
                assert word == 0xFFFFFFFF, (x, y)
                continue
            for i in range(4):
                b = (word >> (8 * i)) & 0xFF
                if not member(x + i, y):
                    assert b == 0xFF, (x, y, i)
                else:
                    d = sum(member(x + i + dx, y + dy)
                            for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)))
                    assert b == d, (x, y, i)


# ------------------------------------------------------------------------
# The write kernels' hash: SplitMix64's high word computed on 32-bit halves
# (splitmix64_hi), restated operation for operation and checked against the
# 64-bit SplitMix64 of the input module on the bits the values use.
# ------------------------------------------------------------------------
def _splitmix64_hi(seedmix, key):
    m = np.uint64(0xFFFFFFFF)
    g = 0x9E3779B97F4A7C15
    m1, m2 = 0xBF58476D1CE4E5B9, 0x94D049BB133111EB
    u = lambda v: np.uint64(v)
    key = key.astype(np.uint64)
    s_lo = (u(seedmix) & m) ^ key
    s_hi = u(seedmix) >> u(32)
    zh0 = (s_hi + u(g >> 32)) & m             # the two values of the high half
    zh1 = (zh0 + u(1)) & m
    th0, th1 = zh0 ^ (zh0 >> u(30)), zh1 ^ (zh1 >> u(30))
    z_lo = (s_lo + u(g & 0xFFFFFFFF)) & m
    carry = z_lo < s_lo
    z_hi = np.where(carry, zh1, zh0)

    def fshr(lo, hi, n):                      # __funnelshift_r(lo, hi, n)
        return ((lo >> u(n)) | (hi << u(32 - n))) & m
    t_lo = z_lo ^ fshr(z_lo, z_hi, 30)
    t_hi = np.where(carry, th1, th0)
    p = t_lo * u(m1 & 0xFFFFFFFF)             # < 2^64: exact in uint64
    y_lo = p & m
    y_hi = ((p >> u(32)) + ((t_lo * u(m1 >> 32)) & m) + ((t_hi * u(m1 & 0xFFFFFFFF)) & m)) & m
    w_lo = y_lo ^ fshr(y_lo, y_hi, 27)
    w_hi = y_hi ^ (y_hi >> u(27))
    umulhi = (w_lo * u(m2 & 0xFFFFFFFF)) >> u(32)
    return (umulhi + ((w_lo * u(m2 >> 32)) & m) + ((w_hi * u(m2 & 0xFFFFFFFF)) & m)) & m


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 12345, 2**63 + 7])
def test_hash_high_word_matches_splitmix64(seed):
    from paper_1706_04552_gb300 import inputs
    rng = np.random.default_rng(seed % 1000)
    keys = np.concatenate([np.arange(4096, dtype=np.uint64),
                           rng.integers(0, 2**32, 200_000, dtype=np.uint64),
                           np.array([2**32 - 1, 2**31, 2**31 - 1], dtype=np.uint64)])
    with np.errstate(over="ignore"):
        seedmix = (seed * 0x9E3779B97F4A7C15) & (2**64 - 1)
        h = inputs.splitmix64_next(np.uint64(seedmix) ^ keys)
    hi = _splitmix64_hi(seedmix, keys)
    assert np.array_equal(hi >> np.uint64(24), h >> np.uint64(56))   # u8 values
    assert np.array_equal(hi >> np.uint64(8), h >> np.uint64(40))    # f32 values


@pytest.mark.parametrize("r,S", [(6, 4), (10, 5), (16, 6), (16, 4)])
def test_tile_base_and_offset_bits_are_disjoint(r, S):
    # key = base + koff with base = (y0 << r) | x0 and koff = (ty << r) | tx:
    # the kernels xor the two instead of adding them
    rng = np.random.default_rng(r * 10 + S)
    nb = 1 << (r - S)
    bx = rng.integers(0, nb, 5000, dtype=np.uint64)
    by = rng.integers(0, nb, 5000, dtype=np.uint64)
    tx = rng.integers(0, 1 << S, 5000, dtype=np.uint64)
    ty = rng.integers(0, 1 << S, 5000, dtype=np.uint64)
    rs, ss = np.uint64(r), np.uint64(S)
    base = ((by << ss) << rs) | (bx << ss)
    koff = (ty << rs) | tx
    assert np.array_equal(base + koff, base ^ koff)
    assert np.all(base + koff < np.uint64(1 << (2 * r)))


# --------------------------------------------------------------------------
# Compact layout: the bit-sliced CA step on 64-tiles (compact_ca_bits_kernel)
# --------------------------------------------------------------------------
M64 = (1 << 64) - 1


def _row_codec():
    """dep / cmp / row_start as make_row_codec builds them."""
    dep = [[0] * 256 for _ in range(8)]
    cmp_ = [[0] * 256 for _ in range(8)]
    for yl in range(8):
        for v in range(256):
            d = c = k = 0
            for lo in range(8):
                if lo & yl == 0:
                    if (v >> k) & 1:
                        d |= 1 << lo
                    if (v >> lo) & 1:
                        c |= 1 << k
                    k += 1
            dep[yl][v], cmp_[yl][v] = d, c
    starts, e = [], 0
    for y in range(64):
        starts.append(e)
        e += 1 << (6 - bin(y).count("1"))
    return dep, cmp_, starts


def _halo_list64():
    """The CA halo cells of a 64-tile in the order make_compact_pattern
    discovers them: cells row by row, neighbours by (dy, dx)."""
    R, halo = 64, []
    for y in range(R):
        for x in range(R):
            if x & y:
                continue
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    nx, ny = x + dx, y + dy
                    if 0 <= nx < R and 0 <= ny < R:
                        continue
                    dbx = -1 if nx < 0 else (1 if nx >= R else 0)
                    dby = -1 if ny < 0 else (1 if ny >= R else 0)
                    lx, ly = nx - dbx * R, ny - dby * R
                    if lx & ly == 0 and (dbx, dby, lx, ly) not in halo:
                        halo.append((dbx, dby, lx, ly))
    return halo


def _lambda_index(bx, by, rb, order):
    """Launch index of a block: the inverse of the decode, as lambda_index."""
    ly = ((1 << rb) - 1) - by
    q = wx = wy = 0
    for mu in range(rb, 0, -1):
        beta = ((bx >> (mu - 1)) & 1) + ((ly >> (mu - 1)) & 1)
        if order == 1:
            q = q * 3 + beta
        elif mu & 1:
            wy = wy * 3 + beta
        else:
            wx = wx * 3 + beta
    return q if order == 1 else wy * 3 ** (rb // 2) + wx


def _compact_bits_ca_tile(state, u, bx, by, rb, order, tabs, halo):
    """One tile of compact_ca_bits_kernel, word operation by word operation."""
    dep, cmp_, starts = tabs
    base = u * 729
    words = [0] * 26
    for c in range(729):
        if state[base + c]:
            words[c >> 5] |= 1 << (c & 31)
    alive = {}
    for k, (dbx, dby, lx, ly) in enumerate(halo):
        nbx, nby = bx + dbx, by + dby
        ok = 0 <= nbx < (1 << rb) and 0 <= nby < (1 << rb) and (nbx & nby) == 0
        v = state[_lambda_index(nbx, nby, rb, order) * 729 + starts[ly] +
                  _rank_in_row(lx, ly)] if ok else 0
        alive[(dbx * 64 + lx, dby * 64 + ly)] = bool(v)

    def bits_at(o):
        k, sh = o >> 5, o & 31
        w0, w1, w2 = words[k], words[k + 1], words[k + 2]
        lo = ((w0 | (w1 << 32)) >> sh) & 0xFFFFFFFF
        hi = ((w1 | (w2 << 32)) >> sh) & 0xFFFFFFFF
        return lo | (hi << 32)

    def deposit(c, y):
        yh, yl = y >> 3, y & 7
        nl = 8 >> bin(yl).count("1")
        row, sh = 0, 0
        for hi in range(8):
            if hi & yh == 0:
                row |= dep[yl][(c >> sh) & ((1 << nl) - 1)] << (8 * hi)
                sh += nl
        return row

    def gather(row, y):
        yh, yl = y >> 3, y & 7
        nl = 8 >> bin(yl).count("1")
        c, sh = 0, 0
        for hi in range(8):
            if hi & yh == 0:
                c |= cmp_[yl][(row >> (8 * hi)) & 0xFF] << sh
                sh += nl
        return c

    def maj(a, b, c):
        return (a & b) | (c & (a ^ b))

    def sums(v, left, right):
        L = ((v << 1) | left) & M64
        R = (v >> 1) | (right << 63)
        return (L ^ v ^ R, maj(L, v, R), L ^ R, L & R)

    rows = [deposit(bits_at(starts[y]), y) for y in range(64)]
    edge_l = {y: int(alive.get((-1, y), False)) for y in range(-1, 65)}
    edge_r = {y: int(alive.get((64, y), False)) for y in range(-1, 65)}
    above = sum(1 << x for x in range(64) if alive.get((x, -1), False))
    below = sum(1 << x for x in range(64) if alive.get((x, 64), False))
    ext = {-1: above, 64: below}
    ext.update(enumerate(rows))
    s = {y: sums(ext[y], edge_l[y], edge_r[y]) for y in range(-1, 65)}
    out = [0] * 729
    for y in range(64):
        u0, u1 = s[y - 1][0], s[y - 1][1]
        m0, m1 = s[y][2], s[y][3]
        b0, b1 = s[y + 1][0], s[y + 1][1]
        s0, k0 = u0 ^ m0 ^ b0, maj(u0, m0, b0)
        t, k1 = u1 ^ m1 ^ b1, maj(u1, m1, b1)
        s1, k2 = t ^ k0, t & k0
        nxt = s1 & ~(k1 | k2) & (s0 | rows[y]) & M64
        c = gather(nxt, y)
        for i in range(1 << (6 - bin(y).count("1"))):
            out[starts[y] + i] = (c >> i) & 1
    return out


def _rank_in_row(lx, ly):
    """Rank of member lx among the members of row ly of a 64-tile."""
    return sum(1 for x in range(lx) if x & ly == 0)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("r", [6, 7, 8])
def test_compact_bit_sliced_ca_restated_matches_oracle(r, order):
    from paper_1706_04552_gb300 import inputs
    s0 = inputs.ca_seed_grid(r, 0.45, 30 + r)
    packed = oracle.compact_pack(r, 6, s0, order)
    want = oracle.compact_ca_step(r, 6, packed, order)
    rb = r - 6
    bx, by = oracle.block_map(rb, order)
    tabs, halo = _row_codec(), _halo_list64()
    assert len(halo) == 8 and tabs[2][63] == 728
    got = []
    for u in range(3 ** rb):
        got += _compact_bits_ca_tile(packed, u, int(bx[u]), int(by[u]), rb, order, tabs, halo)
    assert np.array_equal(np.array(got, dtype=np.uint8), want)


def _halo_runs(KH):
    """make_halo_runs: the runs of the 9 neighbour tiles a KH-step light cone
    reaches, and their word offsets."""
    _, _, starts = _row_codec()

    def start(y):
        return 729 if y >= 64 else starts[y]
    lo, hi, word, w = [], [], [], 0
    for s in range(9):
        dtx, dty = s % 3 - 1, s // 3 - 1
        y0 = 64 - KH if dty < 0 else 0
        y1 = KH if dty > 0 else 64
        if dtx < 0 and y1 > 16:
            y1 = 16
        y1 = max(y1, y0)
        lo.append(start(y0))
        hi.append(start(y1))
        word.append(w)
        w += (hi[-1] - lo[-1] + 31) // 32
    return lo, hi, word, w


def _member_bits4(y):
    return (0x135F >> (4 * (y & 3))) & 0xF


@pytest.mark.parametrize("KH", [4, 8, 16])
@pytest.mark.parametrize("order", [0, 1])
def test_compact_fused_staging_restated_matches_the_grid(KH, order):
    # compact_ca_fused_kernel's staging: runs of the neighbour tiles packed to
    # bits, then every staged 16-column chunk deposited through the row codec,
    # must give the chunk's bits read straight off the embedded grid
    from paper_1706_04552_gb300 import inputs
    r = 8
    n = 1 << r
    grid = inputs.ca_seed_grid(r, 0.5, 70 + KH)
    packed = oracle.compact_pack(r, 6, grid, order)
    rb = r - 6
    bx_all, by_all = oracle.block_map(rb, order)
    dep, _, starts = _row_codec()
    lo, hi, word, nwords = _halo_runs(KH)
    for u in range(3 ** rb):
        bx, by = int(bx_all[u]), int(by_all[u])
        cb = [0] * (nwords + 2)
        for s in range(9):
            nbx, nby = bx + s % 3 - 1, by + s // 3 - 1
            ok = 0 <= nbx < (1 << rb) and 0 <= nby < (1 << rb) and (nbx & nby) == 0
            q = _lambda_index(nbx, nby, rb, order) if ok else None
            for e in range(lo[s], hi[s]):
                if q is not None and packed[q * 729 + e]:
                    bit = (e - lo[s])
                    cb[word[s] + bit // 32] |= 1 << (bit % 32)
        x0, y0 = bx * 64, by * 64
        for row in range(64 + 2 * KH):
            for h in range(6):
                x, y = x0 - 16 + 16 * h, y0 - KH + row
                want = 0
                if 0 <= x < n and 0 <= y < n and (x & y) == 0:
                    for lo16 in range(16):
                        if grid[y, x + lo16]:
                            want |= 1 << lo16
                    s = ((y >> 6) - by + 1) * 3 + ((x >> 6) - bx + 1)
                    lx, ly = x & 63, y & 63
                    cx, n16 = lx >> 4, 16 >> bin(ly & 15).count("1")
                    rank = bin(_member_bits4(ly >> 4) & ((1 << cx) - 1)).count("1")
                    e = starts[ly] + rank * n16
                    assert lo[s] <= e and e + n16 <= hi[s], (u, row, h)
                    o = word[s] * 32 + (e - lo[s])
                    bits = ((cb[o >> 5] | (cb[(o >> 5) + 1] << 32)) >> (o & 31)) & 0xFFFFFFFF
                    yl = ly & 7
                    n8 = 8 >> bin(yl).count("1")
                    m8 = (1 << n8) - 1
                    got = dep[yl][bits & m8]
                    if (ly & 8) == 0:
                        got |= dep[yl][(bits >> n8) & m8] << 8
                    assert got == want, (u, row, h, got, want)
                elif 0 <= x < n and 0 <= y < n:
                    assert not grid[y, x:x + 16].any()


# --------------------------------------------------------------------------
# Compact layout: the compile-time neighbour tables (make_compact_pattern)
# --------------------------------------------------------------------------
HOST_SRC = os.path.join(os.path.dirname(__file__), "host_src", "dump_compact_tables.cu")


@pytest.fixture(scope="module")
def compact_tables(tmp_path_factory):
    """The tables as the library's header computes them, printed by a host
    program built with nvcc from that header (skipped without nvcc)."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path_factory.mktemp("ct") / "dump_ct")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                    "-I", os.path.join(root, "include"),
                    "-I", os.path.join(root, "paper_1706_04552_gb300", "csrc"),
                    HOST_SRC, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    t = {}
    for line in out.splitlines():
        kind, *vals = line.split()
        t.setdefault(kind, []).append(tuple(int(v) for v in vals))
    return t


@pytest.mark.parametrize("S", range(0, 7))
def test_compact_neighbour_tables_match_brute_force(compact_tables, S):
    R = 1 << S
    members = [(x, y) for y in range(R) for x in range(R) if x & y == 0]
    rank = {c: i for i, c in enumerate(members)}
    pos = {e: (x, y) for s, e, x, y in compact_tables["pos"] if s == S}
    assert [pos[e] for e in range(len(members))] == members
    ca_halo = {h: v for s, h, *v in compact_tables["cahalo"] if s == S}
    df_halo = {h: v for s, h, *v in compact_tables["dfhalo"] if s == S}
    assert len(ca_halo) == 8 and len(df_halo) == 4

    def expect(x, y, dx, dy, halo):
        nx, ny = x + dx, y + dy
        if 0 <= nx < R and 0 <= ny < R:
            return rank[(nx, ny)] if nx & ny == 0 else 0xFFFF
        dbx = -1 if nx < 0 else (1 if nx >= R else 0)
        dby = -1 if ny < 0 else (1 if ny >= R else 0)
        lx, ly = nx - dbx * R, ny - dby * R
        if lx & ly:
            return 0xFFFF
        hs = [h for h, v in halo.items() if v[:4] == [dbx, dby, lx, ly]]
        assert len(hs) == 1 and halo[hs[0]][4] == rank[(lx, ly)]
        return 0x8000 | hs[0]

    ca = {(e, k): v for s, e, k, v in compact_tables["ca"] if s == S}
    df = {(e, k): v for s, e, k, v in compact_tables["df"] if s == S}
    deg = {e: v for s, e, v in compact_tables["deg"] if s == S}
    d8 = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
    d4 = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    used_ca, used_df = set(), set()
    for e, (x, y) in enumerate(members):
        for k, (dx, dy) in enumerate(d8):
            v = expect(x, y, dx, dy, ca_halo)
            assert ca[(e, k)] == v, (S, e, k)
            if v != 0xFFFF and v & 0x8000:
                used_ca.add(v & 0x7FFF)
        inside = 0
        for k, (dx, dy) in enumerate(d4):
            v = expect(x, y, dx, dy, df_halo)
            assert df[(e, k)] == v, (S, e, k)
            if v != 0xFFFF and v & 0x8000:
                used_df.add(v & 0x7FFF)
            inside += v < 0x8000
        assert deg[e] == inside
    assert used_ca == set(range(8)) and used_df == set(range(4))


@pytest.mark.parametrize("order", [0, 1])
def test_inverse_lambda_restated_inverts_the_block_map(order):
    # lambda_index (the compact kernels' halo lookup) read back into base-3
    # digits gives every block's launch index, at every level up to 11
    for rb in range(0, 12):
        bx, by = oracle.block_map(rb, order)
        for q in range(3 ** rb):
            assert _lambda_index(int(bx[q]), int(by[q]), rb, order) == q, (rb, q)


# ---------------------------------------------------------------------------
# The warp-per-unit fused diffusion kernel (csrc/sg_fused.cu): its closed form
# for a region row's live chunks, and the bound on live chunks per region that
# sizes its register slots.
# ---------------------------------------------------------------------------
FUSED_SRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1706_04552_gb300", "csrc",
                         "sg_fused.cu")


def _region_row_mask(x0, y, n, hc):
    """region_row_mask<HC> as the kernel computes it."""
    if y < 0 or y >= n:
        return 0
    m3 = (y >> 2) & 7
    s8 = 0xFF
    if m3 & 1:
        s8 &= 0x55
    if m3 & 2:
        s8 &= 0x33
    if m3 & 4:
        s8 &= 0x0F
    lt = (s8 >> (8 - hc)) if (x0 >= 32 and ((x0 - 32) & y) == 0) else 0
    tt = s8 if (x0 & y) == 0 else 0
    rt = (s8 & ((1 << hc) - 1)) if (x0 + 32 < n and ((x0 + 32) & y) == 0) else 0
    return lt | (tt << hc) | (rt << (hc + 8))


@pytest.mark.parametrize("kh", [4, 8, 16])
def test_region_row_mask_is_the_chunk_membership_test(kh):
    # bit cc of the mask: the chunk at column x0 - HX + 4 cc on row y lies in
    # the grid and holds a gasket cell, i.e. (x & y) == 0 -- brute force over
    # every 32-unit column and every region row of levels 5..8
    hx = (kh + 3) // 4 * 4
    hc, pc = hx // 4, 8 + 2 * hx // 4
    for r in range(5, 9):
        n = 1 << r
        for x0 in range(0, n, 32):
            for y in range(-kh, n + kh):
                want = 0
                for cc in range(pc):
                    x = x0 - hx + 4 * cc
                    if 0 <= x < n and 0 <= y < n and (x & y) == 0:
                        want |= 1 << cc
                assert _region_row_mask(x0, y, n, hc) == want, (r, x0, y)


def _neighbourhoods(rb):
    """Which of the 3 x 3 tiles around each non-empty tile of a level-rb block
    gasket are non-empty (tiles off the grid count as empty)."""
    nb = 1 << rb
    out = set()
    for by in range(nb):
        for bx in range(nb):
            if bx & by:
                continue
            out.add(tuple(0 <= bx + i < nb and 0 <= by + j < nb and ((bx + i) & (by + j)) == 0
                          for j in (-1, 0, 1) for i in (-1, 0, 1)))
    return out


def _live_in_region(pattern, kh):
    hx = (kh + 3) // 4 * 4
    pc, rows = 8 + 2 * hx // 4, 32 + 2 * kh
    c = 0
    for row in range(rows):
        for cc in range(pc):
            x, y = 4 * cc - hx, row - kh
            if pattern[((y + 32) // 32) * 3 + (x + 32) // 32] and ((x % 32) & (y % 32)) == 0:
                c += 1
    return c


def test_fused_diffusion_live_block_bound():
    # the rows of a group of 4 (starting at a multiple of 4) share their live
    # chunks, so the region's live 4 x 4 blocks are its live chunks / 4.  The
    # set of neighbourhoods is the same at every block level from 3 to 9, and
    # over it the most live blocks in a unit's region are the kernel's MAXB
    # for each halo depth; the levels' own units agree (brute force)
    sets = [_neighbourhoods(rb) for rb in range(3, 10)]
    assert all(s == sets[0] for s in sets) and len(sets[0]) == 13
    with open(FUSED_SRC) as f:
        m = re.search(r"MAXB = KH == 4 \? (\d+) : KH == 8 \? (\d+) : (\d+);", f.read())
    maxb = dict(zip((4, 8, 16), map(int, m.groups())))
    for kh in (4, 8, 16):
        live = [_live_in_region(p, kh) for p in sets[0]]
        assert all(c % 4 == 0 for c in live)
        assert max(live) == 4 * maxb[kh], kh
    # direct count over every unit of a level-11 gasket, KH = 8: blocks from
    # the first row of each group, chunks from every row
    r, kh = 11, 8
    n = 1 << r
    best = 0
    for by in range(n // 32):
        for bx in range(n // 32):
            if bx & by:
                continue
            rows = [_region_row_mask(32 * bx, 32 * by - kh + row, n, 2) for row in range(32 + 2 * kh)]
            assert all(rows[4 * (i // 4)] == rows[i] for i in range(len(rows)))
            best = max(best, sum(bin(rows[4 * g]).count("1") for g in range(len(rows) // 4)))
    assert best == maxb[8]
