"""GPU parity of the fused stencil steps (sg_ca_steps / sg_diffuse_steps):
k steps in one launch against k steps of the CPU oracle (bit-exact for the
CA, within the FP64 tolerance for diffusion), against k single-step launches,
across levels, tile sides, halo depths (k up to SG_FUSE_MAX), both maps and
both walking orders; and at the stencil workloads' full levels through the
oracle's light cones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs, workloads  # noqa: E402

from test_gpu_parity import (DIFF_TOL, _offgasket_zero, _window_centres,  # noqa: E402
                             max_rel_err, to_dev, to_host)

pytestmark = pytest.mark.gpu
DEV = "cuda"
KS = (2, 3, 4, 5, 8, 9, 15, 16)
FUSED_RHOS = (16, 32, 64)


def _rhos(r):
    return [p for p in FUSED_RHOS if p <= (1 << r)]


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", ["lambda", "bbox"])
@pytest.mark.parametrize("r,p", [(4, 1.0), (5, 0.5), (6, 0.4), (8, 0.5), (11, 0.3)])
def test_ca_fused_matches_oracle(orc, r, p, mapk, order):
    n = 1 << r
    s0 = inputs.ca_seed_grid(r, p, 7)
    ref = [s0]
    for _ in range(max(KS)):
        ref.append(orc.ca_step(r, ref[-1]))
    a = to_dev(s0)
    for rho in _rhos(r):
        for k in KS:
            b = torch.full_like(a, 0)
            sg.ca_steps(a, b, r, rho, k, mapk, order=order)
            assert np.array_equal(to_host(b, n), ref[k]), (rho, k)
    assert np.array_equal(to_host(a, n), s0)             # the input is left as it was


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", ["lambda", "bbox"])
@pytest.mark.parametrize("r", [4, 6, 9, 11])
def test_diffusion_fused_matches_fp64_oracle(orc, r, mapk, order):
    n = 1 << r
    u0 = inputs.uniform_grid(r, 5)
    mask = orc.member_grid(r).astype(bool)
    want = {0: u0.astype(np.float64)}
    for k in range(1, max(KS) + 1):
        want[k] = orc.diffuse_steps(r, want[k - 1], 1, 0.2)
    a = to_dev(u0)
    for rho in _rhos(r):
        for k in KS:
            b = torch.zeros_like(a)
            sg.diffuse_steps(a, b, r, rho, k, 0.2, mapk, order=order)
            got = to_host(b, n)
            assert not got[~mask].any(), (rho, k)
            assert max_rel_err(got[mask], want[k][mask]) <= DIFF_TOL, (rho, k)
    assert np.array_equal(to_host(a, n), u0)
    sg.device_status()          # no unit exceeded its live-chunk bound (raises otherwise)


@pytest.mark.parametrize("rho", FUSED_RHOS)
def test_fused_equals_single_steps(rho):
    # the same arithmetic per cell: k fused steps give the single-step result
    # bit for bit, for the CA and for diffusion
    r = 10
    n = 1 << r
    s0 = to_dev(inputs.ca_seed_grid(r, 0.35, 9))
    u0 = to_dev(inputs.uniform_grid(r, 9))
    for k in (2, 7, 16):
        a, b = s0.clone(), torch.zeros_like(s0)
        for _ in range(k):
            sg.ca_step(a, b, r, rho, "lambda")
            a, b = b, a
        f = torch.zeros_like(s0)
        sg.ca_steps(s0, f, r, rho, k, "lambda")
        assert torch.equal(a, f), ("ca", k)
        a, b = u0.clone(), torch.zeros_like(u0)
        for _ in range(k):
            sg.diffuse_step(a, b, r, rho, 0.2, "lambda")
            a, b = b, a
        f = torch.zeros_like(u0)
        sg.diffuse_steps(u0, f, r, rho, k, 0.2, "lambda")
        torch.cuda.synchronize()
        assert torch.equal(a, f), ("diffusion", k, float((a - f).abs().max()))
    assert n == 1 << r


def test_fused_long_runs_match_oracle(orc):
    # many launches of fused steps chained: 64 CA steps as 16 + 16 + 16 + 16
    # and 100 diffusion steps as 6 x 16 + 4, as the benchmark runs them
    r = 9
    n = 1 << r
    s0 = inputs.ca_seed_grid(r, 0.3, 12)
    a, b = to_dev(s0), torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    for _ in range(4):
        sg.ca_steps(a, b, r, 64, 16)
        a, b = b, a
    assert np.array_equal(to_host(a, n), orc.ca_steps(r, s0, 64))
    u0 = inputs.uniform_grid(r, 12)
    a, b = to_dev(u0), torch.zeros(n * n, dtype=torch.float32, device=DEV)
    for k in (16,) * 6 + (4,):
        sg.diffuse_steps(a, b, r, 32, k, 0.2)
        a, b = b, a
    mask = orc.member_grid(r).astype(bool)
    got = to_host(a, n)
    want = orc.diffuse_steps(r, u0, 100, 0.2)
    assert not got[~mask].any()
    assert max_rel_err(got[mask], want[mask]) <= DIFF_TOL


def _chunks(steps, k):
    out = [k] * (steps // k)
    if steps % k:
        out.append(steps % k)
    return out


@pytest.mark.slow
@pytest.mark.parametrize("r", workloads.STENCILS["levels"])
def test_fused_full_size_light_cones(orc, r):
    w = workloads.STENCILS
    n = 1 << r
    # CA: the timed launch configuration, checked against single steps over
    # the whole grid and against the oracle on windows
    idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], w["ca_seed"])
    a = torch.zeros(n * n, dtype=torch.uint8, device=DEV)
    a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    s0 = a.clone()
    b = torch.zeros_like(a)
    for k in _chunks(w["ca_steps"], w["ca_fuse"]):
        sg.ca_steps(a, b, r, w["ca_fuse_rho"], k)
        a, b = b, a
    c, d = s0, torch.zeros_like(s0)
    for _ in range(w["ca_steps"]):
        sg.ca_step(c, d, r, w["ca_rho"], "lambda")
        c, d = d, c
    torch.cuda.synchronize()
    assert torch.equal(a, c)
    assert _offgasket_zero(a, r)
    steps, R, W = w["ca_steps"], w["ca_steps"] + 1, 32
    g2 = a.view(n, n)
    for (cx, cy) in _window_centres(r, 3, 200 + r):
        x0, y0 = cx - W // 2, cy - W // 2
        win = inputs.ca_seed_region(r, w["ca_p"], w["ca_seed"], x0 - R, y0 - R,
                                    W + 2 * R, W + 2 * R)
        win = orc.ca_steps(r, win, steps, x0 - R, y0 - R)[R:R + W, R:R + W]
        xa, xb, ya, yb = max(0, x0), min(n, x0 + W), max(0, y0), min(n, y0 + W)
        got = g2[ya:yb, xa:xb].cpu().numpy()
        assert np.array_equal(got, win[ya - y0:yb - y0, xa - x0:xb - x0]), (cx, cy)
    del a, b, c, d, s0
    # diffusion
    idx, vals = inputs.uniform_sparse(r, w["diff_seed"])
    a = torch.zeros(n * n, dtype=torch.float32, device=DEV)
    a[torch.from_numpy(idx).to(DEV)] = torch.from_numpy(vals).to(DEV)
    b = torch.zeros_like(a)
    for k in _chunks(w["diff_steps"], w["diff_fuse"]):
        sg.diffuse_steps(a, b, r, w["diff_fuse_rho"], k, w["alpha"])
        a, b = b, a
    torch.cuda.synchronize()
    assert _offgasket_zero(a, r)
    steps, R, W = w["diff_steps"], w["diff_steps"] + 1, 48
    g2 = a.view(n, n)
    worst = 0.0
    for (cx, cy) in _window_centres(r, 6, 300 + r):
        x0, y0 = cx - W // 2, cy - W // 2
        win = inputs.uniform_region(r, w["diff_seed"], x0 - R, y0 - R, W + 2 * R, W + 2 * R)
        win = orc.diffuse_steps(r, win, steps, w["alpha"], x0 - R, y0 - R)[R:R + W, R:R + W]
        xa, xb, ya, yb = max(0, x0), min(n, x0 + W), max(0, y0), min(n, y0 + W)
        got = g2[ya:yb, xa:xb].cpu().numpy()
        want = win[ya - y0:yb - y0, xa - x0:xb - x0]
        assert not got[want == 0].any()
        worst = max(worst, max_rel_err(got, want))
    assert worst <= DIFF_TOL, worst
