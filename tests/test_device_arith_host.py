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


def _member_rank(S, tx, ty):
    rank = sum(1 << (S - bin(t).count("1")) for t in range(ty))
    k = bit = 0
    for bpos in range(S):
        if not (ty >> bpos) & 1:
            k |= ((tx >> bpos) & 1) << bit
            bit += 1
    return rank + k


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
def test_lookup_table_rank_and_unrolled_slots(S):
    R = 1 << S
    ranks = {}
    for ty in range(R):
        for tx in range(R):
            if tx & ty == 0:
                ranks[_member_rank(S, tx, ty)] = (ty, tx)
    # every member gets a distinct rank in 0 .. 3^S - 1, in row-major order
    assert sorted(ranks) == list(range(3 ** S))
    assert [ranks[i] for i in range(3 ** S)] == sorted(ranks.values())
    cells = {_unrolled(S, e) for e in range(3 ** S)}
    assert len(cells) == 3 ** S
    assert all(x & y == 0 and 0 <= x < R and 0 <= y < R for x, y in cells)
