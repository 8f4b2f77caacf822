"""GPU parity of the single-step stencils with each tile and its halo staged
by one 2-D bulk tensor copy (staging="tma", SG_STORE_TMA in sg_launch_opts)
against the 16-byte chunk staging and the CPU oracle.  The staged region and
the arithmetic are the same, so the results are equal bit for bit (CA and
diffusion alike); every wait of the copies completed (device status)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs  # noqa: E402

from test_gpu_parity import DIFF_TOL, max_rel_err, to_dev, to_host  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", ["lambda", "bbox"])
@pytest.mark.parametrize("r", [5, 6, 8, 11])
def test_ca_tma_staging_equals_chunks_and_oracle(orc, r, mapk, order):
    n = 1 << r
    s0 = inputs.ca_seed_grid(r, 0.45, 60 + r)
    want = orc.ca_step(r, s0)
    a = to_dev(s0)
    for rho in (32, 64):
        if rho > n:
            continue
        b1, b2 = torch.zeros_like(a), torch.zeros_like(a)
        sg.ca_step(a, b1, r, rho, mapk, order=order)
        sg.ca_step(a, b2, r, rho, mapk, order=order, staging="tma")
        assert torch.equal(b1, b2), (rho,)
        assert np.array_equal(to_host(b2, n), want), (rho,)
    sg.device_status()


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("mapk", ["lambda", "bbox"])
@pytest.mark.parametrize("r", [4, 5, 8, 11])
def test_diffusion_tma_staging_equals_chunks_and_oracle(orc, r, mapk, order):
    n = 1 << r
    u0 = inputs.uniform_grid(r, 70 + r)
    want = orc.diffuse_steps(r, u0.astype(np.float64), 1, 0.2)
    mask = orc.member_grid(r).astype(bool)
    a = to_dev(u0)
    for rho in (16, 32):
        if rho > n:
            continue
        b1, b2 = torch.zeros_like(a), torch.zeros_like(a)
        sg.diffuse_step(a, b1, r, rho, 0.2, mapk, order=order)
        sg.diffuse_step(a, b2, r, rho, 0.2, mapk, order=order, staging="tma")
        assert torch.equal(b1, b2), (rho,)
        got = to_host(b2, n)
        assert not got[~mask].any()
        assert max_rel_err(got[mask], want[mask]) <= DIFF_TOL
    sg.device_status()


@pytest.mark.slow
def test_tma_staging_level15_sequences_equal_chunks():
    # the benchmark's level-15 configurations: 32 CA steps at rho 64 and 20
    # diffusion steps at rho 32, TMA staging against chunk staging
    r = 15
    n = 1 << r
    for kind, rho, steps in (("ca", 64, 32), ("diffusion", 32, 20)):
        if kind == "ca":
            idx, vals = inputs.ca_seed_sparse(r, 0.3, 0)
            dt = torch.uint8
        else:
            idx, vals = inputs.uniform_sparse(r, 0)
            dt = torch.float32
        runs = []
        for staging in (None, "tma"):
            a = torch.zeros(n * n, dtype=dt, device="cuda")
            a[torch.from_numpy(idx).cuda()] = torch.from_numpy(vals).cuda()
            b = torch.zeros_like(a)
            for _ in range(steps):
                if kind == "ca":
                    sg.ca_step(a, b, r, rho, "lambda", staging=staging)
                else:
                    sg.diffuse_step(a, b, r, rho, 0.2, "lambda", staging=staging)
                a, b = b, a
            runs.append(a)
        assert torch.equal(runs[0], runs[1]), kind
    sg.device_status()
