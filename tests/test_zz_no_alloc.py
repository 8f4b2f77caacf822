"""The allocation-free batch step (sg_batch_ca_step_noalloc).

It exists for callers that must not allocate device memory when they step
a batch -- a real-time loop with a memory budget fixed at start-up, a plugin
whose host application owns every allocation, a server whose own pool holds
all of HBM.  Its work list lives in a fixed array inside the library instead
of a caller workspace.  Checked here through the C ABI against the regular
batch step (sg_batch_ca_step) on two consecutive calls; the CA is integer,
so the comparison is bit-exact.  This file is collected last.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

import paper_1706_04552_gb300 as sg  # noqa: E402
from paper_1706_04552_gb300 import build as sg_build  # noqa: E402
from paper_1706_04552_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu
MAX_GASKETS = 1024        # SG_NOALLOC_MAX_GASKETS in include/sg.h


@pytest.fixture(scope="module")
def L():
    sg_build.build()
    L = sg.lib()
    L.sg_batch_ca_step_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p]
    L.sg_batch_ca_step_noalloc.restype = ctypes.c_int
    return L


def _batch(levels, seed):
    a, b = [], []
    for i, r in enumerate(levels):
        s0 = inputs.ca_seed_grid(r, 0.4, inputs.instance_seed(seed, i))
        a.append(torch.from_numpy(s0.ravel()).cuda())
        b.append(torch.zeros_like(a[-1]))
    return a, b


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def test_noalloc_step_matches_regular_step_twice(L):
    levels = [9, 6, 11, 8, 7, 10]
    rho = 32
    a1, b1 = _batch(levels, 21)                   # regular: caller workspace
    a2, b2 = _batch(levels, 21)                   # allocation-free variant
    regular = sg.CABatch(levels, a1, b1, rho=rho)
    lv = (ctypes.c_int * len(levels))(*levels)
    pa, pb = _ptrs(a2), _ptrs(b2)
    stream = torch.cuda.current_stream().cuda_stream
    for parity in (0, 1):                          # two calls in a row
        regular.step(parity)
        st = L.sg_batch_ca_step_noalloc(len(levels), lv, pa, pb, rho, parity, None, stream)
        assert st == sg.SG_OK, sg.sg_status_str(st)
        torch.cuda.synchronize()
        for i in range(len(levels)):
            assert torch.equal(a1[i], a2[i]) and torch.equal(b1[i], b2[i]), (parity, i)


def test_noalloc_rejects_more_gaskets_than_its_array(L):
    n = MAX_GASKETS + 1
    t = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    u = torch.zeros_like(t)
    lv = (ctypes.c_int * n)(*([6] * n))
    pa = (ctypes.c_void_p * n)(*([t.data_ptr()] * n))
    pb = (ctypes.c_void_p * n)(*([u.data_ptr()] * n))
    st = L.sg_batch_ca_step_noalloc(n, lv, pa, pb, 16, 0, None, None)
    assert st == sg.SG_EINVAL
    assert b"SG_NOALLOC_MAX_GASKETS" in L.sg_last_error_string()


def test_noalloc_full_array_then_a_smaller_call(L):
    # 1024 gaskets of level 4 (one 16 x 16 tile each) fill the array exactly;
    # the next call, with fewer gaskets of other levels, must not read what
    # the first call left behind it.  Both are compared with the regular step.
    rho = 16
    stream = torch.cuda.current_stream().cuda_stream
    for levels, seed in (([4] * MAX_GASKETS, 31), ([7, 5, 9, 4, 6], 32)):
        a1, b1 = _batch(levels, seed)
        a2, b2 = _batch(levels, seed)
        regular = sg.CABatch(levels, a1, b1, rho=rho)
        lv = (ctypes.c_int * len(levels))(*levels)
        pa, pb = _ptrs(a2), _ptrs(b2)
        for parity in (0, 1):
            regular.step(parity)
            st = L.sg_batch_ca_step_noalloc(len(levels), lv, pa, pb, rho, parity, None, stream)
            assert st == sg.SG_OK, sg.sg_status_str(st)
        torch.cuda.synchronize()
        for i in range(len(levels)):
            assert torch.equal(a1[i], a2[i]) and torch.equal(b1[i], b2[i]), (len(levels), i)


def test_noalloc_refuses_while_the_stream_is_captured(L):
    levels = [6, 7]
    a, b = _batch(levels, 33)
    lv = (ctypes.c_int * 2)(*levels)
    pa, pb = _ptrs(a), _ptrs(b)
    before = [t.clone() for t in b]
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = L.sg_batch_ca_step_noalloc(2, lv, pa, pb, 16, 0, None,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == sg.SG_EUNSUPPORTED
    assert b"captured" in L.sg_last_error_string()
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(b, before))
