"""GPU tests of the serving scheduler's native core (include/sg_sched.h) on
its own, without the Python server around it: the advance rule, the order of
completions, the buffer swaps, residency, dropping and the host-side fault
hook, each result checked bit for bit against stepping the gasket alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
RHO = 32


def _state(r, seed):
    idx, vals = inputs.ca_seed_sparse(r, 0.3, seed)
    a = torch.zeros(1 << (2 * r), dtype=torch.uint8)
    a[torch.from_numpy(idx)] = torch.from_numpy(vals)
    return a.cuda()


def _alone(a, r, steps):
    a = a.clone()
    b = torch.zeros_like(a)
    for _ in range(steps):
        sg.ca_step(a, b, r, RHO, "lambda")
        a, b = b, a
    return a


def _advance(left, fuse):
    return min(left, fuse)


def _class(k):
    # launches are shared by advances that stage the same halo
    return 0 if k == 1 else 1 if k <= 4 else 2 if k <= 8 else 3


def _resident(sched, levels, seeds):
    bufs = []
    for g, (r, sd) in enumerate(zip(levels, seeds)):
        a = _state(r, sd)
        b = torch.zeros_like(a)
        sched.set_buffers(g, a.data_ptr(), b.data_ptr())
        bufs.append((a, b))
    return bufs


def _current(sched, g, bufs):
    info = sched.gasket(g)
    a, b = bufs[g]
    assert info.cur in (a.data_ptr(), b.data_ptr())
    return a if info.cur == a.data_ptr() else b


@pytest.mark.parametrize("fuse", [1, 4, 16])
def test_sched_advance_rule_and_results(fuse):
    levels = [5, 6, 7, 9, 5, 8, 7]
    seeds = [11, 12, 13, 14, 15, 16, 17]
    sched = sg.Sched(levels, RHO, fuse)
    bufs = _resident(sched, levels, seeds)
    init = [a.clone() for a, _ in bufs]
    # two requests on gaskets 0 and 1 (run in order), one on most others, none
    # on 6; advances of different lengths share a launch (7 and 6, 3 and 2)
    reqs = [(0, 100, 7), (0, 101, 5), (1, 102, 1), (1, 106, 2), (2, 103, 16), (3, 104, 3),
            (5, 105, 33), (4, 107, 6)]
    sched.submit([g for g, _, _ in reqs], [q for _, q, _ in reqs], [k for _, _, k in reqs])
    stream = torch.cuda.current_stream()
    left = {q: k for _, q, k in reqs}
    queue = {}
    for g, q, _ in reqs:
        queue.setdefault(g, []).append(q)
    done_at, it, steps_done = {}, 0, {g: 0 for g in range(len(levels))}
    while any(queue.values()):
        res = sched.step(stream)
        it += 1
        assert res.iteration == it
        # expected advances: heads of every queue
        want_done = set()
        cells = 0
        groups = set()
        for g, qs in queue.items():
            if not qs:
                continue
            k = _advance(left[qs[0]], fuse)
            groups.add(_class(k))
            left[qs[0]] -= k
            steps_done[g] += k
            cells += 3 ** levels[g] * k
            if left[qs[0]] == 0:
                want_done.add(qs.pop(0))
        done, done_g = sched.completed()
        assert set(done.tolist()) == want_done, it
        assert res.cell_steps == cells and res.n_failed == 0
        assert res.launches == len(groups)                   # one launch per halo class
        for q, g in zip(done.tolist(), done_g.tolist()):
            done_at[q] = (g, steps_done[g], _current(sched, g, bufs).clone())
    assert sched.step(stream).iteration == 0        # nothing left to do
    torch.cuda.synchronize()
    assert set(done_at) == {q for _, q, _ in reqs}
    for q, (g, total, snap) in done_at.items():
        assert torch.equal(snap, _alone(init[g], levels[g], total)), (q, g, total)
    assert torch.equal(_current(sched, 6, bufs), init[6])       # untouched gasket
    for g in range(len(levels)):
        assert sched.gasket(g).steps_done == steps_done[g]
    sched.close()


def test_sched_residency_drop_and_injected_failure():
    levels = [6, 7, 6]
    sched = sg.Sched(levels, RHO, 8)
    bufs = _resident(sched, levels, [1, 2, 3])
    init = [a.clone() for a, _ in bufs]
    sched.set_buffers(1, 0, 0)                      # gasket 1 leaves the device
    sched.submit([0, 1, 1, 2], [10, 11, 12, 13], [3, 2, 4, 8])
    assert sorted(sched.waiting().tolist()) == [1]
    info = sched.gasket(1)
    assert (info.queued, info.head_left, info.resident) == (2, 2, 0)
    req, ran = sched.drop(1)
    assert req.tolist() == [11, 12] and ran.tolist() == [0, 0]
    assert sched.waiting().size == 0
    # the next launch holding gasket 2 is refused on the host: its head fails
    sched.inject_launch_failure(2)
    stream = torch.cuda.current_stream()
    res = sched.step(stream)                        # gasket 0 finishes in one advance of 3
    failed, failed_g, failed_ran = sched.failed()
    assert failed.tolist() == [13] and failed_g.tolist() == [2] and failed_ran.tolist() == [0]
    assert b"injected" in sg.lib().sg_last_error_string()
    done, _ = sched.completed()
    assert done.tolist() == [10]
    assert sched.step(stream).iteration == 0
    torch.cuda.synchronize()
    assert torch.equal(_current(sched, 0, bufs), _alone(init[0], 6, 3))
    assert torch.equal(_current(sched, 2, bufs), init[2])       # nothing ran for it
    assert sched.gasket(2).steps_done == 0
    sched.close()


def test_sched_two_iterations_in_flight_match_one_at_a_time():
    # issuing iteration i + 1 before i has finished changes nothing: the
    # work lists alternate between two page-locked slots
    rng = np.random.default_rng(5)
    levels = [int(x) for x in rng.integers(5, 10, 24)]
    seeds = list(range(100, 124))
    gaskets = rng.integers(0, 24, 200)
    steps = rng.integers(1, 33, 200)
    outs = []
    for sync_each in (True, False):
        sched = sg.Sched(levels, RHO, 16)
        bufs = _resident(sched, levels, seeds)
        init = [a.clone() for a, _ in bufs]
        sched.submit(gaskets, np.arange(200), steps)
        stream = torch.cuda.current_stream()
        while sched.step(stream).iteration:
            if sync_each:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        outs.append([_current(sched, i, bufs).clone() for i in range(24)])
        sched.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    for i in (0, 7, 23):                             # and the plain step sequence
        total = int(steps[gaskets == i].sum())
        assert torch.equal(outs[1][i], _alone(init[i], levels[i], total)), i
