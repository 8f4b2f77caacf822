"""GPU parity of the batched CA: one launch per step over the prefix-summed
work list of many gaskets of uneven levels, bit-exact against the CPU oracle
and against stepping every gasket alone; CUDA-graph replay and the
autotuner give the same states."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _states(levels, p, seed):
    a, b, host = [], [], []
    for i, r in enumerate(levels):
        s0 = inputs.ca_seed_grid(r, p, inputs.instance_seed(seed, i))
        host.append(s0)
        a.append(torch.from_numpy(s0.ravel()).to(DEV))
        b.append(torch.zeros_like(a[-1]))
    return a, b, host


def _current(a, b, steps):
    return a if steps % 2 == 0 else b


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("rho", [16, 32, 64])
def test_batch_matches_oracle(orc, rho, order):
    levels = [6, 9, 7, 6, 10, 8, 11, 6]
    levels = [r for r in levels if (1 << r) >= rho]
    a, b, host = _states(levels, 0.4, 11)
    batch = sg.CABatch(levels, a, b, rho=rho)
    steps = 5
    for k in range(steps):
        batch.step(k & 1, order=order)
    torch.cuda.synchronize()
    cur = _current(a, b, steps)
    for i, r in enumerate(levels):
        n = 1 << r
        want = orc.ca_steps(r, host[i], steps)
        assert np.array_equal(cur[i].cpu().numpy().reshape(n, n), want), (i, r)


def test_batch_graph_equals_steps(orc):
    levels = [8, 5, 10, 7, 9]
    a1, b1, host = _states(levels, 0.5, 3)
    a2, b2, _ = _states(levels, 0.5, 3)
    stepped = sg.CABatch(levels, a1, b1, rho=32)
    graphed = sg.CABatch(levels, a2, b2, rho=32)
    for k in range(6):
        stepped.step(k & 1)
    g = graphed.graph(6, 0)
    g.launch()
    torch.cuda.synchronize()
    for i in range(len(levels)):
        assert torch.equal(a1[i], a2[i]) and torch.equal(b1[i], b2[i])
    g.launch()                      # replaying continues from the new state
    for k in range(6):
        stepped.step(k & 1)
    torch.cuda.synchronize()
    for i, r in enumerate(levels):
        assert torch.equal(a1[i], a2[i])
        n = 1 << r
        assert np.array_equal(a2[i].cpu().numpy().reshape(n, n), orc.ca_steps(r, host[i], 12))
    g.close()


def test_batch_autotune_leaves_state_and_steps_right(orc):
    levels = [9, 6, 8, 7]
    a, b, host = _states(levels, 0.3, 5)
    before = [t.clone() for t in a]
    batch = sg.CABatch(levels, a, b, autotune=3)
    torch.cuda.synchronize()
    assert batch.rho in (16, 32, 64) and batch.opts is not None
    for t0, t1 in zip(before, a):
        assert torch.equal(t0, t1)
    for k in range(4):
        batch.step(k & 1)
    torch.cuda.synchronize()
    for i, r in enumerate(levels):
        n = 1 << r
        assert np.array_equal(a[i].cpu().numpy().reshape(n, n), orc.ca_steps(r, host[i], 4))


@pytest.mark.slow
def test_batch_config_64_gaskets_bit_exact(orc):
    # the batched workload the benchmark times: 64 gaskets, levels 8..14
    w = workloads.BATCH
    levels = inputs.batch_levels(w["count"], w["level_lo"], w["level_hi"], w["level_seed"])
    a, b, host = _states(levels, w["ca_p"], w["ca_seed"])
    sa = [t.clone() for t in a]
    sb = [torch.zeros_like(t) for t in b]
    batch = sg.CABatch(levels, a, b, autotune=w["autotune_steps"])
    g = batch.graph(w["steps"], 0)
    g.launch()
    for k in range(w["steps"]):
        for i, r in enumerate(levels):
            src, dst = (sa[i], sb[i]) if k % 2 == 0 else (sb[i], sa[i])
            sg.ca_step(src, dst, r, batch.rho, "lambda")
    torch.cuda.synchronize()
    for i in range(len(levels)):
        assert torch.equal(a[i], sa[i]), i
    small = [i for i, r in enumerate(levels) if r <= 9][:6]
    for i in small:
        r = levels[i]
        n = 1 << r
        want = orc.ca_steps(r, host[i], w["steps"])
        assert np.array_equal(a[i].cpu().numpy().reshape(n, n), want), (i, r)
    g.close()


# ------------------------------------------------- fused batch steps
def _launch_state(a, b, launches):
    return a if launches % 2 == 0 else b


@pytest.mark.parametrize("order", ["rowmajor", "interleaved"])
@pytest.mark.parametrize("rho", [16, 32, 64])
def test_batch_fused_matches_oracle(orc, rho, order):
    levels = [6, 9, 7, 6, 10, 8, 11, 6]
    levels = [r for r in levels if (1 << r) >= rho]
    a, b, host = _states(levels, 0.4, 13)
    batch = sg.CABatch(levels, a, b, rho=rho)
    ks = (2, 5, 16, 1, 3)                      # five launches, alternating parity
    for j, k in enumerate(ks):
        batch.steps(k, j & 1, order=order)
    torch.cuda.synchronize()
    cur = _launch_state(a, b, len(ks))
    for i, r in enumerate(levels):
        n = 1 << r
        want = orc.ca_steps(r, host[i], sum(ks))
        assert np.array_equal(cur[i].cpu().numpy().reshape(n, n), want), (i, r)


def test_batch_fused_graph_equals_single_steps(orc):
    levels = [8, 5, 10, 7, 9]
    a1, b1, host = _states(levels, 0.5, 4)
    a2, b2, _ = _states(levels, 0.5, 4)
    single = sg.CABatch(levels, a1, b1, rho=32)
    fused = sg.CABatch(levels, a2, b2, rho=32)
    g1 = single.graph(40, 0)                   # 40 launches: state back in a1
    g2 = fused.graph(40, 0, fuse=16)           # 16 + 16 + 8: three launches, state in b2
    g1.launch()
    g2.launch()
    torch.cuda.synchronize()
    for i, r in enumerate(levels):
        assert torch.equal(a1[i], b2[i]), i
        n = 1 << r
        assert np.array_equal(b2[i].cpu().numpy().reshape(n, n), orc.ca_steps(r, host[i], 40))
    g1.close()
    g2.close()


def test_batch_fused_autotune_leaves_state_and_steps_right(orc):
    levels = [9, 6, 8, 7]
    a, b, host = _states(levels, 0.3, 6)
    before = [t.clone() for t in a]
    batch = sg.CABatch(levels, a, b, autotune=2, fuse=8)
    torch.cuda.synchronize()
    assert batch.rho in (16, 32, 64) and batch.opts is not None
    for t0, t1 in zip(before, a):
        assert torch.equal(t0, t1)
    batch.steps(8, 0)
    batch.steps(8, 1)
    torch.cuda.synchronize()
    for i, r in enumerate(levels):
        n = 1 << r
        assert np.array_equal(a[i].cpu().numpy().reshape(n, n), orc.ca_steps(r, host[i], 16))


@pytest.mark.slow
def test_batch_config_64_gaskets_fused_equals_single(orc):
    # the benchmark's batched workload, fused 16 steps per launch, against the
    # single-step batch graph over all 64 gaskets
    w = workloads.BATCH
    levels = inputs.batch_levels(w["count"], w["level_lo"], w["level_hi"], w["level_seed"])
    a1, b1, host = _states(levels, w["ca_p"], w["ca_seed"])
    a2, b2 = [t.clone() for t in a1], [torch.zeros_like(t) for t in b1]
    single = sg.CABatch(levels, a1, b1, rho=64)
    fused = sg.CABatch(levels, a2, b2, autotune=w["autotune_steps"], fuse=w["fuse"])
    g1 = single.graph(w["steps"], 0)
    g2 = fused.graph(w["steps"], 0, fuse=w["fuse"])
    g1.launch()
    g2.launch()
    torch.cuda.synchronize()
    launches = -(-w["steps"] // w["fuse"])
    cur = _launch_state(a2, b2, launches)
    for i in range(len(levels)):
        assert torch.equal(a1[i], cur[i]), i
    for i in [i for i, r in enumerate(levels) if r <= 9][:4]:
        r = levels[i]
        n = 1 << r
        assert np.array_equal(cur[i].cpu().numpy().reshape(n, n),
                              orc.ca_steps(r, host[i], w["steps"])), (i, r)
    g1.close()
    g2.close()
