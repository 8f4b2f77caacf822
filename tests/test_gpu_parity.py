"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.

Bit-exact: the block map, the write pass (u8 and f32 bit patterns) and every
CA state.  Diffusion: maximum relative error over gasket cells <= 1e-5 against
the FP64 oracle, and exactly 0 off the gasket.  Small levels are compared
element by element over the whole grid (every tile, both maps, every rho);
full-size workloads (the configurations the benchmark times) are compared
element by element where the oracle can do the whole grid, and otherwise on
sampled windows whose interiors the oracle computes exactly (light cones).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs, workloads  # noqa: E402

pytestmark = pytest.mark.gpu

RHOS = (1, 2, 4, 8, 16, 32, 64)
ALL_MAPS = tuple(sg.MAPS)
STENCIL_MAPS = ("lambda", "bbox")
DIFF_TOL = 1e-5
DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).ravel()).to(DEV)


def to_host(t, n):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(n, n)


def rhos_for(r):
    return [p for p in RHOS if p <= (1 << r)]


def max_rel_err(got, want):
    on = want != 0
    if not on.any():
        return 0.0
    return float(np.max(np.abs(got[on].astype(np.float64) - want[on]) /
                        np.maximum(np.abs(want[on]), 1e-30)))


# --------------------------------------------------------------- block map

@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("rb", list(range(0, 13)) + [16])
def test_block_map_bit_exact(orc, rb, order):
    bx, by = sg.block_map(rb, order)
    ebx, eby = orc.block_map(rb, sg.ORDERS[order])
    torch.cuda.synchronize()
    assert np.array_equal(bx.cpu().numpy().view(np.uint32), ebx)
    assert np.array_equal(by.cpu().numpy().view(np.uint32), eby)


# -------------------------------------------------------------- write pass

def _vk(orc, name):
    return {"hash": orc.VAL_HASH, "linear31": orc.VAL_LINEAR31, "const": orc.VAL_CONST}[name]


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("mapk", ALL_MAPS)
@pytest.mark.parametrize("r", [0, 1, 3, 6, 9, 11])
def test_write_matches_oracle(orc, r, mapk, dtype):
    n = 1 << r
    rng = np.random.default_rng(100 + r)
    if dtype == "u8":
        before = rng.integers(0, 256, (n, n), dtype=np.uint8)
        const = 0x5A
    else:
        before = (rng.standard_normal((n, n)) - 5.0).astype(np.float32)
        const = int(np.float32(2.5).view(np.uint32))
    for rho in rhos_for(r):
        for vname, val in (("hash", 1), ("linear31", 0), ("const", const)):
            g = to_dev(before)
            sg.map_write(g, r, rho, mapk, vname, val)
            want = before.copy()
            orc.map_write(r, want, _vk(orc, vname), val)
            got = to_host(g, n)
            if dtype == "f32":
                got, want = got.view(np.uint32), want.view(np.uint32)
            assert np.array_equal(got, want), (r, rho, mapk, vname)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [4, 9, 11])
def test_write_every_order_and_store(orc, r, dtype):
    # both walking orders of Pi and both store paths, every map and rho
    n = 1 << r
    rng = np.random.default_rng(300 + r)
    if dtype == "u8":
        before = rng.integers(0, 256, (n, n), dtype=np.uint8)
    else:
        before = (rng.standard_normal((n, n)) - 5.0).astype(np.float32)
    want = before.copy()
    orc.map_write(r, want, orc.VAL_HASH, 3)
    elem = 1 if dtype == "u8" else 4
    for mapk in ALL_MAPS:
        for rho in rhos_for(r):
            for order in ("rowmajor", "interleaved"):
                for store in ("scatter", "staged", "tma"):
                    if store != "scatter" and rho * elem < 16:
                        continue
                    g = to_dev(before)
                    sg.map_write(g, r, rho, mapk, "hash", 3, order=order, store=store)
                    got = to_host(g, n)
                    if dtype == "f32":
                        ok = np.array_equal(got.view(np.uint32), want.view(np.uint32))
                    else:
                        ok = np.array_equal(got, want)
                    assert ok, (mapk, rho, order, store)
    sg.device_status()


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [4, 9, 11])
def test_write_fill_on_zero_grid(orc, r, dtype):
    # write-only tiles: on a grid that is 0 off the gasket the result is the
    # oracle's pass; on any grid, touched tiles hold v at gasket cells and 0
    # elsewhere, and untouched tiles keep their content
    n = 1 << r
    np_dt = np.uint8 if dtype == "u8" else np.float32
    zero = np.zeros((n, n), dtype=np_dt)
    want = zero.copy()
    orc.map_write(r, want, orc.VAL_HASH, 2)
    rng = np.random.default_rng(500 + r)
    noisy = (rng.integers(1, 256, (n, n)) if dtype == "u8"
             else rng.standard_normal((n, n)) + 10.0).astype(np_dt)
    elem = 1 if dtype == "u8" else 4
    for mapk in ALL_MAPS:
        for rho in rhos_for(r):
            if rho * elem < 16:
                continue
            for order in ("rowmajor", "interleaved"):
                g = to_dev(zero)
                sg.map_write(g, r, rho, mapk, "hash", 2, order=order, store="fill")
                got = to_host(g, n)
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (mapk, rho, order)
            g = to_dev(noisy)
            sg.map_write(g, r, rho, mapk, "hash", 2, store="fill")
            got = to_host(g, n)
            nb = n // rho
            t = got.reshape(nb, rho, nb, rho)
            ref = noisy.reshape(nb, rho, nb, rho)
            wt = want.reshape(nb, rho, nb, rho)
            for by in range(nb):
                for bx in range(nb):
                    if bx & by:
                        assert np.array_equal(t[by, :, bx, :], ref[by, :, bx, :])
                    else:
                        assert np.array_equal(t[by, :, bx, :].view(np.uint8),
                                              wt[by, :, bx, :].view(np.uint8))


@pytest.mark.parametrize("mapk", ALL_MAPS)
def test_write_level12_every_rho(orc, mapk):
    r, n = 12, 4096
    before = np.random.default_rng(7).integers(0, 256, (n, n), dtype=np.uint8)
    want = before.copy()
    orc.map_write(r, want, orc.VAL_HASH, 1)
    for rho in RHOS:
        g = to_dev(before)
        sg.map_write(g, r, rho, mapk, "hash", 1)
        assert np.array_equal(to_host(g, n), want), rho


def test_write_on_side_stream(orc):
    r, n = 9, 512
    s = torch.cuda.Stream()
    g = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        sg.map_write(g, r, 16, "lambda", "hash", 5)
    s.synchronize()
    want = np.zeros((n, n), dtype=np.uint8)
    orc.map_write(r, want, orc.VAL_HASH, 5)
    assert np.array_equal(g.cpu().numpy().reshape(n, n), want)


def test_invalid_arguments_launch_nothing():
    r, n = 8, 256
    g = torch.full((n * n,), 7, dtype=torch.uint8, device=DEV)
    assert sg.sg_map_write(r, 3, 0, 0, g.data_ptr(), 2, 1, 0) == sg.SG_EINVAL
    assert sg.sg_map_write(r, 512, 0, 0, g.data_ptr(), 2, 1, 0) == sg.SG_EINVAL
    with pytest.raises(sg.SGError):
        sg.map_write(g, r, 128)
    torch.cuda.synchronize()
    assert int((g != 7).sum()) == 0


def _headline_grid(dtype, seed):
    """A full-size (n = 2^16) grid filled with seeded random content."""
    r = workloads.WRITE_HEADLINE["r"]
    n = 1 << r
    gen = torch.Generator(device=DEV)
    gen.manual_seed(seed)
    if dtype == "u8":
        return torch.randint(0, 256, (n * n,), dtype=torch.uint8, device=DEV, generator=gen)
    return torch.rand((n * n,), dtype=torch.float32, device=DEV, generator=gen) - 2.0


@pytest.mark.slow
def test_write_level16_headline_u8_whole_grid(orc):
    # the launch configuration and input the benchmark times (a zero grid),
    # checked at every cell, twice in a row on the same grid
    w = workloads.WRITE_HEADLINE
    r, n = w["r"], 1 << w["r"]
    g = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    for _ in range(2):
        sg.map_write(g, r, w["rho"], w["map"], w["value"], w["seed"], order=w["order"],
                     store=w["store"])
    got = to_host(g, n)
    want = np.zeros((n, n), dtype=np.uint8)
    orc.map_write(r, want, orc.VAL_HASH, w["seed"])
    assert np.array_equal(got, want)


@pytest.mark.slow
def test_write_level16_preserving_u8_whole_grid(orc):
    # the preserving stores keep arbitrary off-gasket content at full size
    w = dict(workloads.WRITE_HEADLINE, **workloads.WRITE_PRESERVE)
    r, n = w["r"], 1 << w["r"]
    g = _headline_grid("u8", 11)
    before = g.cpu().numpy().reshape(n, n)
    sg.map_write(g, r, w["rho"], w["map"], w["value"], w["seed"], order=w["order"],
                 store=w["store"])
    got = to_host(g, n)
    orc.map_write(r, before, orc.VAL_HASH, w["seed"])
    assert np.array_equal(got, before)


@pytest.mark.slow
def test_write_level16_preserving_f32_whole_grid_in_bands(orc):
    w = dict(workloads.WRITE_HEADLINE, **workloads.WRITE_PRESERVE)
    r, n = w["r"], 1 << w["r"]
    g = _headline_grid("f32", 12)
    g2 = g.view(n, n)
    band = 4096
    before = [g2[y:y + band].cpu().numpy() for y in range(0, n, band)]
    sg.map_write(g, r, w["f32_rho"], w["map"], w["value"], w["seed"], order=w["order"],
                 store=w["store"])
    torch.cuda.synchronize()
    for i, y in enumerate(range(0, n, band)):
        want = before[i]
        orc.map_write(r, want, orc.VAL_HASH, w["seed"], y0=y, y1=y + band)
        got = g2[y:y + band].cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), y


def _sample_cells(r, count, seed):
    """Random gasket cells, random cells, and cells on tile/grid edges."""
    n = 1 << r
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    # random gasket cells: pick y, then x as a random subset of ~y
    y = rng.integers(0, n, count, dtype=np.int64)
    x = rng.integers(0, n, count, dtype=np.int64) & ~y & (n - 1)
    xs.append(x)
    ys.append(y)
    xs.append(rng.integers(0, n, count, dtype=np.int64))
    ys.append(rng.integers(0, n, count, dtype=np.int64))
    edge = np.array([0, 1, 15, 16, 31, 32, 63, 64, n // 2 - 1, n // 2, n - 2, n - 1],
                    dtype=np.int64)
    ex, ey = np.meshgrid(edge, edge)
    xs.append(ex.ravel())
    ys.append(ey.ravel())
    return np.concatenate(xs), np.concatenate(ys)


@pytest.mark.parametrize("store", ["auto", "fill"])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("mapk", ALL_MAPS)
@pytest.mark.parametrize("rho", workloads.WRITE_SWEEP["rhos"])
def test_write_level16_sweep_sampled(orc, rho, mapk, dtype, store):
    r = 16
    n = 1 << r
    if store == "fill" and rho * (1 if dtype == "u8" else 4) < 16:
        pytest.skip("fill stores need 16-byte tile rows")
    g = torch.zeros(n * n, dtype=torch.uint8 if dtype == "u8" else torch.float32, device=DEV)
    sg.map_write(g, r, rho, mapk, "hash", 1, store=store)
    xs, ys = _sample_cells(r, 100_000, rho)
    idx = torch.from_numpy(ys * n + xs).to(DEV)
    got = g[idx].cpu().numpy()
    np_dt = np.uint8 if dtype == "u8" else np.float32
    want = orc.write_expected_at(r, np_dt, orc.VAL_HASH, 1, xs, ys,
                                 np.zeros(len(xs), dtype=np_dt))
    if dtype == "f32":
        got, want = got.view(np.uint32), want.view(np.uint32)
        # every cell holding a value >= 0 is written exactly once: 3^16 of them
        assert int((g >= 0.5 / 2**24).sum()) <= 3 ** 16
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------- CA

def _run_ca(state, r, rho, mapk, steps, check=None, order=None):
    a = to_dev(state)
    b = torch.zeros_like(a)
    for t in range(steps):
        sg.ca_step(a, b, r, rho, mapk, order=order)
        a, b = b, a
        if check is not None:
            check(t + 1, a)
    return a


@pytest.mark.parametrize("mapk", STENCIL_MAPS)
def test_small_config_write_then_ca_bit_exact(orc, mapk):
    w = workloads.SMALL
    r, rho, n = w["r"], w["rho"], 1 << w["r"]
    g = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    sg.map_write(g, r, rho, mapk, w["write_value"], w["write_seed"])
    want = np.zeros((n, n), dtype=np.uint8)
    orc.map_write(r, want, orc.VAL_LINEAR31, w["write_seed"])
    assert np.array_equal(to_host(g, n), want)
    s = inputs.ca_seed_grid(r, w["ca_p"], w["ca_seed"])
    ref = [s]
    for _ in range(w["ca_steps"]):
        ref.append(orc.ca_step(r, ref[-1]))

    def check(t, a):
        assert np.array_equal(to_host(a, n), ref[t]), t
    _run_ca(s, r, rho, mapk, w["ca_steps"], check)


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", STENCIL_MAPS)
@pytest.mark.parametrize("r,p", [(0, 1.0), (1, 1.0), (2, 0.5), (4, 0.5), (6, 0.4),
                                 (9, 0.5), (12, 0.3)])
def test_ca_matches_oracle_every_rho(orc, r, p, mapk, order):
    n = 1 << r
    s0 = inputs.ca_seed_grid(r, p, 3)
    steps = 6
    ref = [s0]
    for _ in range(steps):
        ref.append(orc.ca_step(r, ref[-1]))
    for rho in rhos_for(r):
        def check(t, a, rho=rho):
            assert np.array_equal(to_host(a, n), ref[t]), (rho, t)
        _run_ca(s0, r, rho, mapk, steps, check, order)


def _offgasket_zero(t, r):
    """True iff every off-gasket cell of the n x n device grid is 0."""
    n = 1 << r
    g = t.view(n, n)
    x = torch.arange(n, device=DEV, dtype=torch.int32)
    chunk = max(1, (1 << 26) // n)
    for y0 in range(0, n, chunk):
        y = torch.arange(y0, min(n, y0 + chunk), device=DEV, dtype=torch.int32)
        off = (y[:, None] & x[None, :]) != 0
        if bool((g[y0:y0 + len(y)][off] != 0).any()):
            return False
    return True


def _window_centres(r, count, seed):
    n = 1 << r
    rng = np.random.default_rng(seed)
    y = rng.integers(0, n, count, dtype=np.int64)
    x = rng.integers(0, n, count, dtype=np.int64) & ~y & (n - 1)
    special = [(0, 0), (n - 1, 0), (0, n - 1), (n // 2, 0), (n // 2 - 1, n // 2),
               (n // 2, n // 2 - 1), (n // 4, n // 2), (n - 33, 32)]
    return list(zip(x.tolist(), y.tolist())) + special


@pytest.mark.slow
@pytest.mark.parametrize("r", workloads.STENCILS["levels"])
def test_ca_full_size_light_cones(orc, r):
    w = workloads.STENCILS
    n, steps = 1 << r, w["ca_steps"]
    idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], w["ca_seed"])
    finals = {}
    for mapk, rho in (("lambda", w["ca_rho"]), ("bbox", w["bbox_ca_rho"])):
        a = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
        a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
        b = torch.zeros_like(a)
        for _ in range(steps):
            sg.ca_step(a, b, r, rho, mapk)
            a, b = b, a
        torch.cuda.synchronize()
        finals[mapk] = a
    assert torch.equal(finals["lambda"], finals["bbox"])
    a = finals["lambda"]
    assert _offgasket_zero(a, r)
    R, W = steps + 1, 48
    g2 = a.view(n, n)
    for (cx, cy) in _window_centres(r, 6, r):
        x0, y0 = cx - W // 2, cy - W // 2
        win = inputs.ca_seed_region(r, w["ca_p"], w["ca_seed"], x0 - R, y0 - R,
                                    W + 2 * R, W + 2 * R)
        win = orc.ca_steps(r, win, steps, x0 - R, y0 - R)[R:R + W, R:R + W]
        xa, xb = max(0, x0), min(n, x0 + W)
        ya, yb = max(0, y0), min(n, y0 + W)
        got = g2[ya:yb, xa:xb].cpu().numpy()
        assert np.array_equal(got, win[ya - y0:yb - y0, xa - x0:xb - x0]), (cx, cy)


# --------------------------------------------------------------- diffusion

def _run_diffusion(u0, r, rho, mapk, steps, alpha=0.2, order=None):
    a = to_dev(u0)
    b = torch.zeros_like(a)
    for _ in range(steps):
        sg.diffuse_step(a, b, r, rho, alpha, mapk, order=order)
        a, b = b, a
    return a


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", STENCIL_MAPS)
@pytest.mark.parametrize("r", [0, 1, 2, 5, 8, 11])
def test_diffusion_matches_fp64_oracle_every_rho(orc, r, mapk, order):
    n = 1 << r
    u0 = inputs.uniform_grid(r, 4)
    steps = 12
    want = orc.diffuse_steps(r, u0, steps, 0.2)
    mask = orc.member_grid(r).astype(bool)
    for rho in rhos_for(r):
        got = to_host(_run_diffusion(u0, r, rho, mapk, steps, order=order), n)
        assert not got[~mask].any(), rho
        assert max_rel_err(got[mask], want[mask]) <= DIFF_TOL, rho


@pytest.mark.slow
@pytest.mark.parametrize("r", workloads.STENCILS["levels"])
def test_diffusion_full_size_light_cones(orc, r):
    w = workloads.STENCILS
    n, steps = 1 << r, w["diff_steps"]
    idx, vals = inputs.uniform_sparse(r, w["diff_seed"])
    finals = {}
    for mapk, rho in (("lambda", w["diff_rho"]), ("bbox", w["bbox_diff_rho"])):
        a = torch.zeros(n * n, dtype=torch.float32, device=DEV)
        a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
        b = torch.zeros_like(a)
        for _ in range(steps):
            sg.diffuse_step(a, b, r, rho, w["alpha"], mapk)
            a, b = b, a
        torch.cuda.synchronize()
        finals[mapk] = a
    a = finals["lambda"]
    assert torch.equal(finals["lambda"], finals["bbox"])
    assert _offgasket_zero(a, r)
    # mass: conserved exactly in exact arithmetic (symmetric exchanges)
    m0 = float(np.sum(vals.astype(np.float64)))
    m1 = float(a.view(n, n).double().sum(dim=1).sum()) if r <= 14 else \
        sum(float(a.view(n, n)[y:y + 4096].double().sum()) for y in range(0, n, 4096))
    assert abs(m1 - m0) <= 1e-5 * m0
    R, W = steps + 1, 48
    g2 = a.view(n, n)
    worst = 0.0
    for (cx, cy) in _window_centres(r, 8, 100 + r):
        x0, y0 = cx - W // 2, cy - W // 2
        win = inputs.uniform_region(r, w["diff_seed"], x0 - R, y0 - R, W + 2 * R, W + 2 * R)
        win = orc.diffuse_steps(r, win, steps, w["alpha"], x0 - R, y0 - R)[R:R + W, R:R + W]
        xa, xb = max(0, x0), min(n, x0 + W)
        ya, yb = max(0, y0), min(n, y0 + W)
        got = g2[ya:yb, xa:xb].cpu().numpy()
        want = win[ya - y0:yb - y0, xa - x0:xb - x0]
        assert not got[want == 0].any()
        worst = max(worst, max_rel_err(got, want))
    assert worst <= DIFF_TOL, worst


# ------------------------------------------------- write pass on host memory
@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("store", [None, "staged", "scatter"])
def test_mapped_write_on_pinned_host_memory(orc, dtype, store):
    # the kernel reads and writes a pinned host grid in place; off-gasket
    # content is kept, gasket cells get the values of the oracle
    for r, mapk, rho in ((8, "lambda_unroll", 16), (11, "lambda", 32), (11, "bbox", 64),
                         (10, "lambda_lut", 4)):
        n = 1 << r
        npdt = np.uint8 if dtype == "u8" else np.float32
        noise = inputs.uniform_grid(r, 77).astype(np.float32) * 200.0
        noise[orc.member_grid(r) == 0] = 7.0            # off the gasket: arbitrary content
        init = noise.astype(npdt)
        host = torch.from_numpy(init.ravel().copy()).pin_memory()
        elem = 1 if dtype == "u8" else 4
        if store == "staged" and rho * elem < 16:
            continue
        sg.map_write_mapped(host, r, rho, mapk, "hash", 5, store=store)
        torch.cuda.synchronize()
        want = init.copy()
        orc.map_write(r, want, orc.VAL_HASH, 5)
        got = host.numpy().reshape(n, n)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (r, mapk, rho, store)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_mapped_fill_writes_whole_groups_and_reads_nothing(orc, dtype):
    # fill on a host grid: gasket cells get v, the other cells of every
    # written group (a 32-byte sector, or a 16-byte chunk for 16-byte tile
    # rows) become 0, everything else keeps its content; on a grid that is 0
    # off the gasket that is exactly the oracle's pass
    npdt = np.uint8 if dtype == "u8" else np.float32
    elem = np.dtype(npdt).itemsize
    for r, mapk, rho in ((9, "lambda_unroll", 16), (11, "lambda_unroll", 64),
                         (11, "bbox", 32), (10, "lambda", 16)):
        if rho * elem < 16:
            continue
        n = 1 << r
        noise = (inputs.uniform_grid(r, 31).astype(np.float32) * 200.0 + 3.0).astype(npdt)
        ys, xs = np.mgrid[0:n, 0:n]
        noise[(xs & ys) != 0] = npdt(9)
        host = torch.from_numpy(noise.ravel().copy()).pin_memory()
        sg.map_write_mapped(host, r, rho, mapk, "hash", 6, store="fill")
        torch.cuda.synchronize()
        want = noise.copy()
        orc.map_write(r, want, orc.VAL_HASH, 6)
        ge = (32 if rho * elem >= 32 else 16) // elem
        written = (((xs & ~(ge - 1)) & ys) == 0) & ((xs & ys) != 0)
        want[written] = 0
        got = host.numpy().reshape(n, n)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (r, mapk, rho)
        zero = torch.zeros(n * n, dtype=host.dtype).pin_memory()
        sg.map_write_mapped(zero, r, rho, mapk, "hash", 6, store="fill")
        torch.cuda.synchronize()
        ref = np.zeros((n, n), dtype=npdt)
        orc.map_write(r, ref, orc.VAL_HASH, 6)
        assert np.array_equal(zero.numpy().reshape(n, n).view(np.uint8), ref.view(np.uint8))


def test_mapped_write_refuses_device_memory():
    g = torch.zeros(1 << 16, dtype=torch.uint8, device=DEV)
    assert sg.sg_map_write_mapped(8, 16, 0, 0, g.data_ptr(), 2, 1) == sg.SG_EINVAL


@pytest.mark.slow
def test_mapped_write_level16_sampled(orc):
    # the end-to-end configuration of the benchmark: the level-16 grid in
    # pinned host memory, written in place, sampled against the oracle; and
    # the whole grid against the device pass, byte for byte
    from paper_1706_04552_gb300 import workloads
    m = workloads.WRITE_MAPPED
    r, n = 16, 1 << 16
    host = torch.zeros(n * n, dtype=torch.uint8).pin_memory()
    sg.map_write_mapped(host, r, m["rho"], m["map"], "hash", 1, order=m["order"],
                        store=m["store"])
    torch.cuda.synchronize()
    xs, ys = _sample_cells(r, 100_000, 9)
    got = host.numpy()[ys * n + xs]
    want = orc.write_expected_at(r, np.uint8, orc.VAL_HASH, 1, xs, ys,
                                 np.zeros(len(xs), dtype=np.uint8))
    assert np.array_equal(got, want)
    g = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    sg.map_write(g, r, 64, "lambda_unroll", "hash", 1, order="interleaved", store="fill")
    for y0 in range(0, n, 8192):
        band = slice(y0 * n, (y0 + 8192) * n)
        assert torch.equal(g[band].cpu(), host[band]), y0
