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
