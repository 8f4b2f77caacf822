"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out (an mbarrier nothing arrives on) returns, records SG_ETIMEOUT
in the device status word for the host to read, and leaves the CUDA context
usable -- the bulk-copy write pass that uses the same wait still runs and
matches the oracle afterwards."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402

from test_gpu_parity import to_dev, to_host  # noqa: E402

pytestmark = pytest.mark.gpu
LIMIT_NS = 50_000_000          # 50 ms: short, far above any real copy's latency


def _status():
    h = torch.cuda.current_stream().cuda_stream
    return sg.sg_device_status(h)


def _tma_write_matches_oracle(orc, r=9, rho=32):
    n = 1 << r
    before = np.random.default_rng(5).integers(0, 256, (n, n), dtype=np.uint8)
    want = before.copy()
    orc.map_write(r, want, orc.VAL_HASH, 11)
    g = to_dev(before)
    sg.map_write(g, r, rho, "lambda", "hash", 11, store="tma")
    return np.array_equal(to_host(g, n), want)


def test_completed_wait_records_nothing():
    assert _status() == sg.SG_OK                      # nothing left from earlier tests
    sg.wait_selftest(blocks=304, arrive=True, limit_ns=LIMIT_NS)
    assert _status() == sg.SG_OK


def test_wait_that_runs_out_reports_timeout_and_context_survives(orc):
    assert _status() == sg.SG_OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sg.wait_selftest(blocks=304, arrive=False, limit_ns=LIMIT_NS)
    st = _status()                                    # synchronises the stream
    dt = time.perf_counter() - t0
    assert st == sg.SG_ETIMEOUT
    # every block gave up after about the limit, not before it and not much later
    assert LIMIT_NS * 1e-9 <= dt < 5.0, dt
    assert _status() == sg.SG_OK                      # reading cleared the word
    with pytest.raises(sg.SGError) as ei:             # the tensor-level check raises
        sg.wait_selftest(blocks=1, arrive=False, limit_ns=1_000_000)
        sg.device_status()
    assert ei.value.status == sg.SG_ETIMEOUT
    # the context is intact: kernels still launch and compute the right thing,
    # and the TMA write pass's own bounded waits complete
    assert _tma_write_matches_oracle(orc)
    x = torch.arange(1 << 20, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == float((1 << 20) * ((1 << 20) - 1) // 2)
    assert _status() == sg.SG_OK


def test_timeouts_from_several_launches_collapse_to_one_report():
    # the word keeps the first error; later ones leave it as it is
    for _ in range(3):
        sg.wait_selftest(blocks=8, arrive=False, limit_ns=2_000_000)
    assert _status() == sg.SG_ETIMEOUT
    assert _status() == sg.SG_OK
