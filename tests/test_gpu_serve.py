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


@pytest.mark.parametrize("engine", ["native", "python"])
def test_serve_batched_same_alone_and_in_the_mix(orc, engine):
    cfg = ServeConfig(gaskets=48, level_max=11, rate=2000.0, duration=0.25, seed=7,
                      engine=engine)
    s = _serve_and_check(orc, cfg)
    assert s["launches"] == s["iterations"]


@pytest.mark.parametrize("engine,pipeline", [("native", 2), ("native", 1), ("python", 1)])
def test_serve_with_evictions_to_host(orc, engine, pipeline):
    # a budget of a few MB forces idle gaskets out to pinned host memory
    cfg = ServeConfig(gaskets=32, level_max=10, rate=3000.0, duration=0.2, seed=9,
                      budget_bytes=3 << 20, engine=engine, pipeline=pipeline)
    _serve_and_check(orc, cfg, expect_evictions=True)


def test_serve_per_gasket_mode(orc):
    cfg = ServeConfig(gaskets=24, level_max=10, rate=2000.0, duration=0.15, seed=11,
                      mode="per_gasket")
    s = _serve_and_check(orc, cfg)
    assert s["launches"] >= s["iterations"]


@pytest.mark.parametrize("engine,pipeline", [("native", 2), ("native", 4), ("python", 1)])
def test_serve_fused_same_alone_and_in_the_mix(orc, engine, pipeline):
    # iterations advance gaskets by up to 16 fused steps, grouped by the steps
    # left in each head request; every result still equals stepping alone
    cfg = ServeConfig(gaskets=48, level_max=11, rate=3000.0, duration=0.25, seed=8, fuse=16,
                      engine=engine, pipeline=pipeline)
    s = _serve_and_check(orc, cfg)
    assert s["launches"] >= s["iterations"]


def test_serve_fused_with_evictions_to_host(orc):
    cfg = ServeConfig(gaskets=32, level_max=10, rate=3000.0, duration=0.2, seed=10,
                      budget_bytes=3 << 20, fuse=8)
    _serve_and_check(orc, cfg, expect_evictions=True)


@pytest.mark.parametrize("engine", ["native", "python"])
def test_serve_contains_host_side_failures(orc, engine):
    # failures injected on the host: one batched launch is refused (an SGError
    # from the C ABI, as a bad plan would give; in the native core its
    # host-side injection) and one gasket's copy onto the device fails.  The
    # affected requests are reported failed; every other request still equals
    # stepping its gasket alone through the steps that actually ran, and the
    # trace is served to the end.
    cfg = ServeConfig(gaskets=24, level_max=9, rate=3000.0, duration=0.15, seed=13,
                      budget_bytes=1 << 20, fuse=4, engine=engine)
    server = Server(cfg)
    initial = [g.host.clone() for g in server.gaskets]
    trace = make_trace(cfg)
    t, gid, k = trace
    with_reqs = sorted(set(int(x) for x in gid))
    launch_victim = with_reqs[0]
    load_victim = next(i for i in reversed(with_reqs)
                       if not server.gaskets[i].resident and i != launch_victim)
    fired = {"launch": 0, "load": 0}
    launch, make_resident = server._launch, server._make_resident

    def failing_launch(group, kk):
        if fired["launch"] == 0 and any(g.gid == launch_victim and g.steps_done > 0
                                        for g in group):
            fired["launch"] += 1
            raise sg.SGError("sg_batch_ca_steps", sg.SG_ECUDA, "injected")
        return launch(group, kk)

    def failing_resident(g, protect):
        if fired["load"] == 0 and g.gid == load_victim and not g.resident:
            fired["load"] += 1
            raise RuntimeError("injected copy failure")
        return make_resident(g, protect)

    if engine == "native":
        server.sched.inject_launch_failure(launch_victim)
        fired["launch"] += 1
    else:
        server._launch = failing_launch
    server._make_resident = failing_resident
    snap = {}

    def on_complete(req, g):
        snap[req] = g.cur.clone()

    res = server.run(trace, on_complete)
    torch.cuda.synchronize()
    assert fired == {"launch": 1, "load": 1}
    failed = res["failed"]
    ran = {req: steps for req, _, steps, _ in server.failures}
    assert failed.sum() == len(server.failures) >= 2
    assert set(np.nonzero(failed)[0]) == set(ran)
    assert all("injected" in err for _, _, _, err in server.failures)
    assert len(snap) + failed.sum() == len(t)
    assert not np.isnan(res["latency_s"]).any()
    for i, g in enumerate(server.gaskets):
        reqs = [j for j in range(len(t)) if gid[j] == i]
        a = initial[i].cuda()
        b = torch.zeros_like(a)
        rho = min(cfg.rho, 1 << g.level)
        for j in reqs:
            for _ in range(ran.get(j, int(k[j]))):
                sg.ca_step(a, b, g.level, rho, "lambda")
                a, b = b, a
            if not failed[j]:
                torch.cuda.synchronize()
                assert torch.equal(a, snap[j]), (i, j)


def _full_size_sample(levels):
    """Gaskets whose every request is checked at the full serving size: every
    gasket of level >= 11 (the seeded draw of 500 gaskets holds one each at
    levels 12, 13 and 15, five at 11 and none at 14), and the first three of
    each level 6..10."""
    pick = [i for i, r in enumerate(levels) if r >= 11]
    for r in range(6, 11):
        pick += [i for i, lr in enumerate(levels) if lr == r][:3]
    return sorted(pick)


@pytest.mark.parametrize("mode,fuse", [("batched", 1), ("batched", 16), ("per_gasket", 1)])
def test_serve_full_size_config_bit_exact(orc, mode, fuse):
    # The serving configuration itself: 500 resident gaskets of levels 6..15
    # drawn toward small levels (seed 3), Poisson arrivals at 2000 req/s for
    # 2 s (seed 4), 1-32 CA steps per request, 40 GB device budget.  For a
    # sample spread over every level present, every completed request's state
    # is kept and compared bit for bit with the gasket stepped alone through
    # the same requests; sampled gaskets of level <= 10 are also compared
    # with the CPU oracle after their last request.
    cfg = ServeConfig(mode=mode, fuse=fuse)
    assert (cfg.gaskets, cfg.level_min, cfg.level_max, cfg.rate, cfg.duration,
            cfg.budget_bytes) == (500, 6, 15, 2000.0, 2.0, 40 << 30)
    server = Server(cfg)
    levels = [g.level for g in server.gaskets]
    sample = set(_full_size_sample(levels))
    assert len(sample) >= 20 and {15, 13, 12, 11} <= {levels[i] for i in sample}
    initial = {i: server.gaskets[i].host.clone() for i in sample}
    trace = make_trace(cfg)
    t, gid, k = trace
    snap = {}

    def on_complete(req, g):
        if g.gid in sample:
            snap[req] = g.cur.clone()

    res = server.run(trace, on_complete)
    torch.cuda.synchronize()
    assert not res["failed"].any()
    s = summarize(res, cfg)
    assert s["requests"] == len(t) > 3000
    checked = 0
    for i in sorted(sample):
        g = server.gaskets[i]
        reqs = [j for j in range(len(t)) if gid[j] == i]
        a = initial[i].cuda()
        b = torch.zeros_like(a)
        rho = min(cfg.rho, 1 << g.level)
        for j in reqs:
            for _ in range(int(k[j])):
                sg.ca_step(a, b, g.level, rho, "lambda")
                a, b = b, a
            torch.cuda.synchronize()
            assert torch.equal(a, snap.pop(j)), (i, g.level, j)
            checked += 1
        if g.level <= 10 and reqs:
            n = 1 << g.level
            want = orc.ca_steps(g.level, initial[i].numpy().reshape(n, n),
                                int(sum(k[j] for j in reqs)))
            assert np.array_equal(server.state_of(i), want), (i, g.level)
    assert checked >= 100 and not snap
