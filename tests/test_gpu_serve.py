"""GPU tests of the continuous-batching server: every request's result is
the same alone and in the mix (bit-exact CA), with and without evictions to
host memory, in batched and per-gasket modes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300.serve import ServeConfig, Server, make_trace, summarize  # noqa: E402

pytestmark = pytest.mark.gpu


def _serve_and_check(orc, cfg, expect_evictions=False):
    server = Server(cfg)
    initial = [g.host.clone() for g in server.gaskets]
    trace = make_trace(cfg)
    snap = {}

    def on_complete(req, g):
        snap[req] = g.cur.clone()

    res = server.run(trace, on_complete)
    torch.cuda.synchronize()
    t, gid, k = trace
    assert len(snap) == len(t)
    # replay every gasket alone with single-gasket launches, request by request
    for i, g in enumerate(server.gaskets):
        reqs = [j for j in range(len(t)) if gid[j] == i]
        if not reqs:
            continue
        a = initial[i].cuda()
        b = torch.zeros_like(a)
        rho = min(cfg.rho, 1 << g.level)
        for j in reqs:
            for _ in range(int(k[j])):
                sg.ca_step(a, b, g.level, rho, "lambda")
                a, b = b, a
            torch.cuda.synchronize()
            assert torch.equal(a, snap[j]), (i, j)
        if g.level <= 8:
            n = 1 << g.level
            want = orc.ca_steps(g.level, initial[i].numpy().reshape(n, n), int(sum(k[j] for j in reqs)))
            assert np.array_equal(server.state_of(i), want)
    s = summarize(res, cfg)
    assert s["requests"] == len(t)
    if expect_evictions:
        # gaskets go out to host memory and come back (preloading is not counted)
        assert s["evictions"] > 0 and s["loads"] > 0
    return s


def test_serve_batched_same_alone_and_in_the_mix(orc):
    cfg = ServeConfig(gaskets=48, level_max=11, rate=2000.0, duration=0.25, seed=7)
    s = _serve_and_check(orc, cfg)
    assert s["launches"] == s["iterations"]


def test_serve_with_evictions_to_host(orc):
    # a budget of a few MB forces idle gaskets out to pinned host memory
    cfg = ServeConfig(gaskets=32, level_max=10, rate=3000.0, duration=0.2, seed=9,
                      budget_bytes=3 << 20)
    _serve_and_check(orc, cfg, expect_evictions=True)


def test_serve_per_gasket_mode(orc):
    cfg = ServeConfig(gaskets=24, level_max=10, rate=2000.0, duration=0.15, seed=11,
                      mode="per_gasket")
    s = _serve_and_check(orc, cfg)
    assert s["launches"] >= s["iterations"]


def test_serve_fused_same_alone_and_in_the_mix(orc):
    # iterations advance gaskets by up to 16 fused steps, grouped by the steps
    # left in each head request; every result still equals stepping alone
    cfg = ServeConfig(gaskets=48, level_max=11, rate=3000.0, duration=0.25, seed=8, fuse=16)
    s = _serve_and_check(orc, cfg)
    assert s["launches"] >= s["iterations"]


def test_serve_fused_with_evictions_to_host(orc):
    cfg = ServeConfig(gaskets=32, level_max=10, rate=3000.0, duration=0.2, seed=10,
                      budget_bytes=3 << 20, fuse=8)
    _serve_and_check(orc, cfg, expect_evictions=True)
