"""GPU parity of the sector store modes of the write pass (SG_STORE_SECTOR,
SG_STORE_MERGE, SG_STORE_MASKED: one lane per unit, 32-byte sector accesses)
against the CPU oracle, bit for bit.

The preserving modes are checked on grids of random content, which must stay
as they were off the gasket.  The write-only mode is checked on the zero grid
(the oracle's pass) and, on random content, against its own definition: every
32-byte sector holding a gasket cell is rewritten whole (0 off the gasket),
every other sector keeps its content."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import workloads  # noqa: E402

from test_gpu_parity import ALL_MAPS, _sample_cells, _vk, to_dev, to_host  # noqa: E402

pytestmark = pytest.mark.gpu
SECTOR_RHOS = {"u8": (32, 64), "f32": (8, 16, 32, 64)}


def _random_grid(n, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, (n, n), dtype=np.uint8)
    return (rng.standard_normal((n, n)) - 5.0).astype(np.float32)


def _const(dtype):
    return 0xA5 if dtype == "u8" else int(np.float32(-1.25).view(np.uint32))


def _same(got, want):
    return np.array_equal(got.view(np.uint8), want.view(np.uint8))


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [5, 6, 9, 11])
def test_preserving_sector_modes_match_oracle(orc, r, dtype):
    n = 1 << r
    before = _random_grid(n, dtype, 700 + r)
    for vname in ("hash", "linear31", "const"):
        val = {"hash": 4, "linear31": 0, "const": _const(dtype)}[vname]
        want = before.copy()
        orc.map_write(r, want, _vk(orc, vname), val)
        for mapk in ALL_MAPS:
            for rho in SECTOR_RHOS[dtype]:
                if rho > n:
                    continue
                for order in ("rowmajor", "interleaved"):
                    for store in ("merge", "masked"):
                        g = to_dev(before)
                        sg.map_write(g, r, rho, mapk, vname, val, order=order, store=store)
                        assert _same(to_host(g, n), want), (vname, mapk, rho, order, store)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("r", [5, 6, 9, 11])
def test_write_only_sector_mode(orc, r, dtype):
    n = 1 << r
    np_dt = np.uint8 if dtype == "u8" else np.float32
    zero = np.zeros((n, n), dtype=np_dt)
    noisy = _random_grid(n, dtype, 900 + r)
    e = 32 if dtype == "u8" else 8                      # elements per 32-byte sector
    ys, xs = np.nonzero(np.ones((n, n), dtype=bool))
    touched = ((xs & ~(e - 1)) & ys) == 0
    for vname in ("hash", "linear31", "const"):
        val = {"hash": 6, "linear31": 0, "const": _const(dtype)}[vname]
        want = zero.copy()
        orc.map_write(r, want, _vk(orc, vname), val)
        # on any grid: touched sectors as on the zero grid, the rest unchanged
        want_noisy = noisy.copy().ravel()
        want_noisy[touched] = want.ravel()[touched]
        for mapk in ALL_MAPS:
            for rho in SECTOR_RHOS[dtype]:
                if rho > n:
                    continue
                for order in ("rowmajor", "interleaved"):
                    g = to_dev(zero)
                    sg.map_write(g, r, rho, mapk, vname, val, order=order, store="sector")
                    assert _same(to_host(g, n), want), (vname, mapk, rho, order)
                g = to_dev(noisy)
                sg.map_write(g, r, rho, mapk, vname, val, store="sector")
                assert _same(to_host(g, n).ravel(), want_noisy), (vname, mapk, rho, "noisy")


@pytest.mark.slow
@pytest.mark.parametrize("store", ["sector", "merge", "masked"])
def test_sector_modes_level16_u8_whole_grid(orc, store):
    # the headline grid (65536^2 uint8), hash seed 1, lambda at rho 64,
    # written twice in a row; the preserving modes on random content
    w = workloads.WRITE_HEADLINE
    r, n = w["r"], 1 << w["r"]
    if store == "sector":
        g = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
        before = np.zeros((n, n), dtype=np.uint8)
    else:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(21)
        g = torch.randint(0, 256, (n * n,), dtype=torch.uint8, device="cuda", generator=gen)
        before = g.cpu().numpy().reshape(n, n)
    for _ in range(2):
        sg.map_write(g, r, 64, w["map"], "hash", w["seed"], order=w["order"], store=store)
    got = to_host(g, n)
    orc.map_write(r, before, orc.VAL_HASH, w["seed"])
    assert np.array_equal(got, before)


@pytest.mark.slow
@pytest.mark.parametrize("rho", [8, 32, 64])
@pytest.mark.parametrize("mapk", ["lambda", "bbox"])
def test_sector_mode_level16_f32_sampled(orc, rho, mapk):
    r = 16
    n = 1 << r
    g = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    sg.map_write(g, r, rho, mapk, "hash", 1, store="sector")
    xs, ys = _sample_cells(r, 100_000, 40 + rho)
    got = g[torch.from_numpy(ys * n + xs).cuda()].cpu().numpy()
    want = orc.write_expected_at(r, np.float32, orc.VAL_HASH, 1, xs, ys,
                                 np.zeros(len(xs), dtype=np.float32))
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_sector_modes_on_pinned_host_memory(orc, dtype):
    # the same kernels writing a grid in page-locked host memory in place
    r = 11
    n = 1 << r
    for store in ("merge", "masked", "sector"):
        before = (np.zeros((n, n), dtype=np.uint8 if dtype == "u8" else np.float32)
                  if store == "sector" else _random_grid(n, dtype, 1300))
        host = torch.from_numpy(before.ravel().copy()).pin_memory()
        for rho in SECTOR_RHOS[dtype]:
            host.copy_(torch.from_numpy(before.ravel()))
            sg.map_write_mapped(host, r, rho, "lambda_unroll", "hash", 8, store=store)
            torch.cuda.synchronize()
            want = before.copy()
            orc.map_write(r, want, orc.VAL_HASH, 8)
            assert _same(host.numpy().reshape(n, n), want), (store, rho)
