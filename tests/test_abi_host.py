"""The C ABI on the host: libsg.so loads, exports every symbol the headers
under include/ declare, reports its status strings and launch accounting, and rejects bad
arguments before launching anything (no call here reaches a kernel)."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

import paper_1706_04552_gb300 as sg
from paper_1706_04552_gb300 import build as sg_build


@pytest.fixture(scope="module")
def L():
    sg_build.build()
    return sg.lib()


def _declared_symbols():
    names = set()
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        names |= set(re.findall(r"SG_API\s+[\w\s\*]+?\b(sg_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for want in ("sg_map_write", "sg_ca_step", "sg_diffuse_step", "sg_block_map",
                 "sg_launch_stats", "sg_status_str", "sg_last_error_string",
                 "sg_abi_version", "sg_device_status", "sg_map_write_ex"):
        assert want in names


def test_library_exports_every_declared_symbol(L):
    for name in _declared_symbols():
        assert hasattr(L, name), name


def test_abi_version_and_status_strings(L):
    assert sg.sg_abi_version() == 2
    assert sg.sg_status_str(0) == "SG_OK"
    for code in range(1, 6):
        assert sg.sg_status_str(code).startswith("SG_E")
    assert "unknown" in sg.sg_status_str(99)
    # the last error message is process-wide: empty in a fresh process, or
    # whatever an earlier test's refused call left there
    msg = sg.lib().sg_last_error_string()
    assert isinstance(msg, bytes)
    fresh = subprocess.run(
        [sys.executable, "-c", "import paper_1706_04552_gb300 as sg; "
         "print(sg.lib().sg_last_error_string())"],
        cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert fresh.returncode == 0 and fresh.stdout.strip() == "b''", fresh.stderr


@pytest.mark.parametrize("r,rho", [(0, 1), (4, 2), (8, 8), (10, 16), (12, 32), (16, 64)])
def test_launch_stats_match_the_oracle(L, orc, r, rho):
    s = rho.bit_length() - 1
    for name, mid in sg.MAPS.items():
        st, launched, useful = sg.sg_launch_stats(r, rho, mid)
        assert st == 0
        assert useful == 3 ** r
        if r <= 12:
            assert (launched, useful) == orc.launch_counts(r, s, mid), name
    _, lam, _ = sg.sg_launch_stats(r, rho, sg.MAPS["lambda"])
    _, bb, _ = sg.sg_launch_stats(r, rho, sg.MAPS["bbox"])
    assert lam == 3 ** (r - s) * 4 ** s and bb == 4 ** r


FAKE = 0x10000  # never dereferenced: every call below fails validation first


@pytest.mark.parametrize("r,rho", [(-1, 1), (17, 1), (4, 3), (4, 0), (4, 32), (8, 128), (3, 16)])
def test_bad_level_or_tile_is_einval(L, r, rho):
    assert sg.sg_map_write(r, rho, 0, 0, FAKE, 2, 1) == sg.SG_EINVAL
    assert sg.sg_ca_step(r, rho, 0, FAKE, FAKE + 4096, 0) == sg.SG_EINVAL
    assert sg.sg_diffuse_step(r, rho, 0, FAKE, FAKE + 4096, 0.2, 0) == sg.SG_EINVAL
    assert sg.sg_launch_stats(r, rho, 0)[0] == sg.SG_EINVAL


def test_bad_pointers_and_enums_are_einval(L):
    assert sg.sg_map_write(8, 16, 0, 0, 0, 2, 1) == sg.SG_EINVAL          # null grid
    assert sg.sg_map_write(8, 16, 9, 0, FAKE, 2, 1) == sg.SG_EINVAL       # bad map
    assert sg.sg_map_write(8, 16, 0, 7, FAKE, 2, 1) == sg.SG_EINVAL       # bad dtype
    assert sg.sg_map_write(8, 16, 0, 0, FAKE, 5, 1) == sg.SG_EINVAL       # bad value kind
    assert sg.sg_map_write(8, 16, 0, 1, FAKE + 2, 2, 1) == sg.SG_EINVAL   # f32 misaligned
    assert sg.sg_ca_step(8, 16, 0, FAKE, FAKE, 0) == sg.SG_EINVAL         # in == out
    assert sg.sg_ca_step(8, 16, 0, 0, FAKE, 0) == sg.SG_EINVAL            # null in
    assert sg.sg_ca_step(8, 16, 0, FAKE + 8, FAKE + 8192, 0) == sg.SG_EINVAL   # misaligned
    assert sg.sg_diffuse_step(8, 16, 0, FAKE, FAKE + 4, 0.2, 0) == sg.SG_EINVAL
    assert sg.sg_diffuse_step(8, 16, 0, FAKE, FAKE + 8192, float("nan"), 0) == sg.SG_EINVAL
    assert sg.sg_block_map(17, 1, FAKE, FAKE + 64, 0) == sg.SG_EINVAL
    assert sg.sg_block_map(4, 1, FAKE, FAKE, 0) == sg.SG_EINVAL
    assert sg.sg_block_map(4, 1, 0, FAKE, 0) == sg.SG_EINVAL
    assert sg.sg_block_map(4, 2, FAKE, FAKE + 64, 0) == sg.SG_EINVAL      # bad order


def test_bad_launch_options_are_rejected_before_launch(L):
    bad = [sg.launch_opts(order=5), sg.launch_opts(store=8), sg.launch_opts(ctas_per_sm=-1),
           sg.launch_opts(ctas_per_sm=65)]
    o = sg.launch_opts(order=1)
    o.reserved[2] = 1
    bad.append(o)
    for opts in bad:
        assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE, 2, 1, opts) == sg.SG_EINVAL
        assert sg.sg_ca_step_ex(8, 16, 0, FAKE, FAKE + 8192, opts) == sg.SG_EINVAL
        assert sg.sg_diffuse_step_ex(8, 16, 0, FAKE, FAKE + 8192, 0.2, opts) == sg.SG_EINVAL
    # staged stores need 16-byte tile rows and a 16-byte aligned grid
    staged = sg.launch_opts(store="staged")
    assert sg.sg_map_write_ex(8, 8, 0, 0, FAKE, 2, 1, staged) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_ex(8, 2, 0, 1, FAKE, 2, 1, staged) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE + 1, 2, 1, staged) == sg.SG_EINVAL
    tma = sg.launch_opts(store="tma")
    assert sg.sg_map_write_ex(8, 8, 0, 0, FAKE, 2, 1, tma) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_ex(8, 2, 0, 1, FAKE, 2, 1, tma) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE + 8, 2, 1, tma) == sg.SG_EINVAL
    assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE, 2, 1, sg.launch_opts(store=8)) == sg.SG_EINVAL
    fill = sg.launch_opts(store="fill")
    assert sg.sg_map_write_ex(8, 8, 0, 0, FAKE, 2, 1, fill) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE + 4, 2, 1, fill) == sg.SG_EINVAL
    # the sector modes need 32-byte tile rows and a 32-byte aligned grid
    for name in ("sector", "merge", "masked"):
        o = sg.launch_opts(store=name)
        assert sg.sg_map_write_ex(8, 16, 0, 0, FAKE, 2, 1, o) == sg.SG_EUNSUPPORTED
        assert sg.sg_map_write_ex(8, 4, 0, 1, FAKE, 2, 1, o) == sg.SG_EUNSUPPORTED
        assert sg.sg_map_write_ex(8, 32, 0, 0, FAKE + 16, 2, 1, o) == sg.SG_EINVAL
        assert sg.sg_map_write_ex(8, 8, 0, 1, FAKE + 16, 2, 1, o) == sg.SG_EINVAL


def test_fused_steps_validate_before_launch(L):
    # every case below is refused on the host, so no kernel is launched
    ca, df = sg.sg_ca_steps, sg.sg_diffuse_steps
    for k in (0, -1, sg.FUSE_MAX + 1):
        assert ca(8, 16, 0, FAKE, FAKE + 8192, k) == sg.SG_EINVAL
        assert df(8, 16, 0, FAKE, FAKE + 8192, 0.2, k) == sg.SG_EINVAL
    for rho in (1, 2, 4, 8):                                  # tiles too narrow to fuse
        assert ca(8, rho, 0, FAKE, FAKE + 8192, 4) == sg.SG_EUNSUPPORTED
        assert df(8, rho, 0, FAKE, FAKE + 8192, 0.2, 4) == sg.SG_EUNSUPPORTED
    assert ca(8, 16, 2, FAKE, FAKE + 8192, 4) == sg.SG_EUNSUPPORTED      # intra-block map
    assert ca(8, 16, 9, FAKE, FAKE + 8192, 4) == sg.SG_EINVAL            # bad map
    assert ca(8, 16, 0, FAKE, FAKE, 4) == sg.SG_EINVAL                   # in == out
    assert ca(8, 16, 0, 0, FAKE, 4) == sg.SG_EINVAL                      # null in
    assert ca(8, 16, 0, FAKE + 8, FAKE + 8192, 4) == sg.SG_EINVAL        # misaligned
    assert ca(17, 16, 0, FAKE, FAKE + 8192, 4) == sg.SG_EINVAL           # bad level
    assert ca(3, 16, 0, FAKE, FAKE + 8192, 4) == sg.SG_EINVAL            # rho > n
    assert df(8, 16, 0, FAKE, FAKE + 8192, float("inf"), 4) == sg.SG_EINVAL
    assert df(8, 16, 0, FAKE, FAKE + 4, 0.2, 4) == sg.SG_EINVAL          # misaligned out
    bad = sg.launch_opts(ctas_per_sm=-3)
    assert ca(8, 16, 0, FAKE, FAKE + 8192, 4, bad) == sg.SG_EINVAL
    assert df(8, 16, 0, FAKE, FAKE + 8192, 0.2, 4, bad) == sg.SG_EINVAL


def test_tma_staging_needs_a_warp_tile_shape(L):
    tma = sg.launch_opts(store="tma")
    for rho in (8, 16):                      # CA: tensor-copy staging at rho 32 and 64 only
        assert sg.sg_ca_step_ex(8, rho, 0, FAKE, FAKE + 65536, tma) == sg.SG_EUNSUPPORTED
    for rho in (4, 8, 64):                   # diffusion: rho 16 and 32 only
        assert sg.sg_diffuse_step_ex(8, rho, 0, FAKE, FAKE + 262144, 0.2, tma) == \
            sg.SG_EUNSUPPORTED
    with pytest.raises(ValueError):
        sg._staging_store("bulk")


def test_stencils_reject_intra_block_maps(L):
    for m in ("lambda_lut", "lambda_unroll"):
        mid = sg.MAPS[m]
        assert sg.sg_ca_step(8, 16, mid, FAKE, FAKE + 8192, 0) == sg.SG_EUNSUPPORTED
        assert sg.sg_diffuse_step(8, 16, mid, FAKE, FAKE + 8192, 0.2, 0) == sg.SG_EUNSUPPORTED


def test_tensor_layer_refuses_cpu_tensors(L):
    torch = pytest.importorskip("torch")
    g = torch.zeros(16 * 16, dtype=torch.uint8)
    with pytest.raises(TypeError):
        sg.map_write(g, 4, 4)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setenv("SG_LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(sg, "_lib", None)
    with pytest.raises(ImportError):
        sg.lib()


def test_batch_workspace_bytes(L):
    assert sg.lib().sg_batch_workspace_bytes(0) == 0
    assert sg.lib().sg_batch_workspace_bytes(65536) == 0
    for count in (1, 2, 3, 64, 1000):
        b = sg.lib().sg_batch_workspace_bytes(count)
        assert b % 16 == 0 and b >= 4 * (count + 1) + 4 * count + 16 * count


def test_batch_plan_validation_is_host_side(L):
    import ctypes
    n = 3
    lv = (ctypes.c_int * n)(8, 9, 10)
    pa = (ctypes.c_void_p * n)(FAKE, FAKE + 0x100000, FAKE + 0x200000)
    pb = (ctypes.c_void_p * n)(FAKE + 0x300000, FAKE + 0x400000, FAKE + 0x500000)
    ws = sg.lib().sg_batch_workspace_bytes(n)
    plan = sg.BatchPlan()
    call = lambda **k: sg.lib().sg_batch_ca_plan(
        k.get("count", n), k.get("lv", lv), pa, k.get("pb", pb), k.get("rho", 16),
        k.get("ws", FAKE + 0x900000), k.get("wsb", ws), ctypes.byref(plan), None)
    assert call(rho=8) == sg.SG_EUNSUPPORTED
    assert call(count=0) == sg.SG_EINVAL
    assert call(wsb=ws - 16) == sg.SG_EINVAL
    assert call(ws=FAKE + 0x900004) == sg.SG_EINVAL
    assert call(lv=(ctypes.c_int * n)(8, 3, 10)) == sg.SG_EINVAL          # level < log2(rho)
    assert call(lv=(ctypes.c_int * n)(8, 17, 10)) == sg.SG_EINVAL
    assert call(pb=(ctypes.c_void_p * n)(FAKE, FAKE + 0x400000, FAKE + 0x500000)) == sg.SG_EINVAL
    bad = sg.BatchPlan()
    assert sg.lib().sg_batch_ca_step(ctypes.byref(bad), 0, None, None) == sg.SG_EINVAL
    h = ctypes.c_void_p()
    assert sg.lib().sg_batch_ca_graph_create(ctypes.byref(bad), 4, 0, None, ctypes.byref(h)) == sg.SG_EINVAL
    assert sg.lib().sg_graph_launch(None, None) == sg.SG_EINVAL
    assert sg.lib().sg_batch_ca_steps(ctypes.byref(bad), 0, 4, None, None) == sg.SG_EINVAL
    assert sg.lib().sg_batch_ca_graph_create_fused(ctypes.byref(bad), 16, 4, 0, None,
                                                   ctypes.byref(h)) == sg.SG_EINVAL
    # a well-formed plan (never launched: only its fields are checked here)
    good = sg.BatchPlan()
    good.workspace, good.workspace_bytes, good.count = FAKE, ws, n
    good.rho, good.total_tiles, good.max_level = 16, 9 + 27 + 81, 10
    for k in (0, -2, sg.FUSE_MAX + 1):
        assert sg.lib().sg_batch_ca_steps(ctypes.byref(good), 0, k, None, None) == sg.SG_EINVAL
        assert sg.lib().sg_batch_ca_graph_create_fused(ctypes.byref(good), 16, k, 0, None,
                                                       ctypes.byref(h)) == sg.SG_EINVAL
    assert sg.lib().sg_batch_ca_steps(ctypes.byref(good), 2, 4, None, None) == sg.SG_EINVAL
    assert sg.lib().sg_batch_ca_graph_create_fused(ctypes.byref(good), 0, 4, 0, None,
                                                   ctypes.byref(h)) == sg.SG_EINVAL
    bad_opts = sg.launch_opts(order=3)
    assert sg.lib().sg_batch_ca_steps(ctypes.byref(good), 0, 4, ctypes.byref(bad_opts),
                                      None) == sg.SG_EINVAL
    for k in (0, sg.FUSE_MAX + 1):
        assert sg.lib().sg_batch_ca_autotune_fused(n, lv, pa, pb, FAKE + 0x900000, ws, 2, k,
                                                   ctypes.byref(plan), ctypes.byref(sg.LaunchOpts()),
                                                   None) == sg.SG_EINVAL


def test_mapped_write_refuses_memory_it_cannot_check(L):
    # ordinary (unregistered) host memory, a null pointer and the bulk-copy
    # store paths are refused before any launch
    import numpy as np
    buf = np.zeros(1 << 16, dtype=np.uint8)
    ptr = buf.ctypes.data
    assert sg.sg_map_write_mapped(8, 16, 0, 0, ptr, 2, 1) == sg.SG_EINVAL
    assert sg.sg_map_write_mapped(8, 16, 0, 0, 0, 2, 1) == sg.SG_EINVAL
    assert sg.sg_map_write_mapped(8, 16, 0, 0, ptr, 2, 1,
                                  sg.launch_opts(store="tma")) == sg.SG_EUNSUPPORTED
    for name in ("sector", "merge", "masked"):             # 16-byte tile rows
        assert sg.sg_map_write_mapped(8, 16, 0, 0, ptr, 2, 1,
                                      sg.launch_opts(store=name)) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_mapped(8, 16, 0, 0, ptr, 2, 1,
                                  sg.launch_opts(store="fill")) == sg.SG_EINVAL
    assert sg.sg_map_write_mapped(8, 8, 0, 0, ptr, 2, 1,           # 8-byte tile rows
                                  sg.launch_opts(store="fill")) == sg.SG_EUNSUPPORTED
    assert sg.sg_map_write_mapped(17, 16, 0, 0, ptr, 2, 1) == sg.SG_EINVAL


def test_wait_selftest_validates_before_launch(L):
    # block counts and wait limits out of range are refused on the host
    for blocks, limit in ((0, 10 ** 6), (1025, 10 ** 6), (1, 999), (1, 2 * 10 ** 9 + 1)):
        assert sg.sg_wait_selftest(blocks, 0, limit) == sg.SG_EINVAL, (blocks, limit)


def test_compact_entries_validate_before_launch(L):
    u8, f32 = sg.DTYPES["u8"], sg.DTYPES["f32"]
    # level, tile side, dtype, pointers, alignment, aliasing
    assert sg.sg_compact_pack(17, 16, u8, FAKE, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_pack(8, 128, u8, FAKE, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_pack(3, 16, u8, FAKE, FAKE + 4096) == sg.SG_EINVAL   # rho > n
    assert sg.sg_compact_pack(8, 16, 2, FAKE, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_pack(8, 16, u8, 0, FAKE) == sg.SG_EINVAL
    assert sg.sg_compact_pack(8, 16, u8, FAKE, FAKE) == sg.SG_EINVAL
    assert sg.sg_compact_pack(8, 16, f32, FAKE + 2, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_unpack(8, 16, f32, FAKE, FAKE + 4098) == sg.SG_EINVAL
    assert sg.sg_compact_unpack(8, 12, u8, FAKE, FAKE + 4096) == sg.SG_EINVAL
    # value kinds, stencil aliasing, alpha, store options
    assert sg.sg_compact_map_write(8, 16, u8, FAKE, 3, 1) == sg.SG_EINVAL
    assert sg.sg_compact_map_write(8, 16, u8, 0, 2, 1) == sg.SG_EINVAL
    assert sg.sg_compact_ca_step(8, 16, FAKE, FAKE) == sg.SG_EINVAL
    assert sg.sg_compact_ca_step(8, 16, 0, FAKE) == sg.SG_EINVAL
    assert sg.sg_compact_diffuse_step(8, 16, FAKE, FAKE + 4096, float("nan")) == sg.SG_EINVAL
    assert sg.sg_compact_diffuse_step(8, 16, FAKE + 1, FAKE + 4096, 0.2) == sg.SG_EINVAL
    opts = sg.launch_opts(store="staged")
    assert sg.sg_compact_ca_step(8, 16, FAKE, FAKE + 4096, opts) == sg.SG_EUNSUPPORTED
    assert sg.sg_compact_map_write(8, 16, u8, FAKE, 2, 1, opts) == sg.SG_EUNSUPPORTED
    assert sg.sg_compact_ca_step(8, 16, FAKE, FAKE + 4096, sg.launch_opts(order=2)) == sg.SG_EINVAL
    assert sg.compact_size(16) == 43046721


def test_compact_fused_steps_validate_before_launch(L):
    assert sg.sg_compact_ca_steps(8, 64, 0, FAKE, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_ca_steps(8, 64, sg.FUSE_MAX + 1, FAKE, FAKE + 4096) == sg.SG_EINVAL
    assert sg.sg_compact_ca_steps(8, 64, 4, FAKE, FAKE) == sg.SG_EINVAL
    assert sg.sg_compact_ca_steps(8, 32, 4, FAKE, FAKE + 4096) == sg.SG_EUNSUPPORTED
    assert sg.sg_compact_ca_steps(5, 64, 4, FAKE, FAKE + 4096) == sg.SG_EINVAL      # rho > n


def test_compact_mapped_write_refuses_memory_it_cannot_check(L):
    import numpy as np
    buf = np.zeros(3 ** 8, dtype=np.uint8)
    u8 = sg.DTYPES["u8"]
    assert sg.sg_compact_map_write_mapped(8, 16, u8, 0, 2, 1) == sg.SG_EINVAL
    assert sg.sg_compact_map_write_mapped(8, 16, u8, buf.ctypes.data, 2, 1) == sg.SG_EINVAL
    assert sg.sg_compact_map_write_mapped(8, 16, u8, buf.ctypes.data, 3, 1) == sg.SG_EINVAL
    assert sg.sg_compact_map_write_mapped(17, 16, u8, buf.ctypes.data, 2, 1) == sg.SG_EINVAL
    assert sg.sg_compact_map_write_mapped(8, 16, u8, buf.ctypes.data, 2, 1,
                                          sg.launch_opts(store="fill")) == sg.SG_EUNSUPPORTED


def test_sched_headers_declare_the_serving_core():
    names = _declared_symbols()
    for want in ("sg_batch_ca_plan_host", "sg_sched_create", "sg_sched_destroy",
                 "sg_sched_set_buffers", "sg_sched_submit", "sg_sched_waiting",
                 "sg_sched_gasket", "sg_sched_drop", "sg_sched_step",
                 "sg_sched_inject_launch_failure"):
        assert want in names


def test_sched_argument_checks_on_the_host(L):
    # everything refused before any CUDA call: no device is needed
    lv = (ctypes.c_int * 3)(6, 7, 8)
    h = ctypes.c_void_p()
    assert L.sg_sched_create(0, lv, 32, 1, None, ctypes.byref(h)) == sg.SG_EINVAL
    assert L.sg_sched_create(3, lv, 48, 1, None, ctypes.byref(h)) == sg.SG_EUNSUPPORTED
    assert L.sg_sched_create(3, lv, 32, 0, None, ctypes.byref(h)) == sg.SG_EINVAL
    assert L.sg_sched_create(3, lv, 32, 17, None, ctypes.byref(h)) == sg.SG_EINVAL
    low = (ctypes.c_int * 3)(6, 4, 8)                  # level 4 holds no 32 x 32 tile
    assert L.sg_sched_create(3, low, 32, 1, None, ctypes.byref(h)) == sg.SG_EINVAL
    assert L.sg_sched_create(3, lv, 32, 1, None, None) == sg.SG_EINVAL
    assert L.sg_sched_destroy(None) == sg.SG_EINVAL
    assert L.sg_sched_step(None, None, None) == sg.SG_EINVAL
    assert L.sg_sched_submit(None, 0, None, None, None) == sg.SG_EINVAL


def test_batch_plan_host_writes_the_work_list(L):
    # the work list image: prefix sums of 3^(r - s), levels, both pointers
    levels = [5, 6, 8]
    rho, s = 32, 5
    n = len(levels)
    nbytes = int(L.sg_batch_workspace_bytes(n))
    img = (ctypes.c_ubyte * nbytes)()
    lv = (ctypes.c_int * n)(*levels)
    pa = (ctypes.c_void_p * n)(0x1000, 0x2000, 0x3000)
    pb = (ctypes.c_void_p * n)(0x1100, 0x2100, 0x3100)
    plan = sg.BatchPlan()
    st = L.sg_batch_ca_plan_host(n, lv, None, pa, pb, rho, img, nbytes, 0x10000, nbytes,
                                 ctypes.byref(plan))
    assert st == sg.SG_OK
    assert plan.count == n and plan.rho == rho and plan.max_level == 8
    assert plan.reserved[0] == 0                       # no per-gasket step counts
    tiles = [3 ** (r - s) for r in levels]
    assert plan.total_tiles == sum(tiles)
    raw = bytes(img)
    prefix = np.frombuffer(raw[:4 * (n + 1)], dtype=np.uint32)
    assert list(prefix) == [0, tiles[0], tiles[0] + tiles[1], sum(tiles)]
    # the image is too small, a pointer is unaligned, a level is below the tile
    assert L.sg_batch_ca_plan_host(n, lv, None, pa, pb, rho, img, nbytes - 16, 0x10000, nbytes,
                                   ctypes.byref(plan)) == sg.SG_EINVAL
    bad = (ctypes.c_void_p * n)(0x1000, 0x2008, 0x3000)
    assert L.sg_batch_ca_plan_host(n, lv, None, bad, pb, rho, img, nbytes, 0x10000, nbytes,
                                   ctypes.byref(plan)) == sg.SG_EINVAL
    low = (ctypes.c_int * n)(4, 6, 8)
    assert L.sg_batch_ca_plan_host(n, low, None, pa, pb, rho, img, nbytes, 0x10000, nbytes,
                                   ctypes.byref(plan)) == sg.SG_EINVAL
    # per-gasket step counts: level in bits 0..7, steps in bits 8..15, the
    # largest in the plan; out-of-range counts are refused
    steps = (ctypes.c_int * n)(3, 8, 1)
    assert L.sg_batch_ca_plan_host(n, lv, steps, pa, pb, rho, img, nbytes, 0x10000, nbytes,
                                   ctypes.byref(plan)) == sg.SG_OK
    assert plan.reserved[0] == 8
    lvl_off = 4 * (n + 1)
    lvl_off = (lvl_off + 15) // 16 * 16
    words = np.frombuffer(bytes(img)[lvl_off:lvl_off + 4 * n], dtype=np.int32)
    assert list(words) == [r | (k << 8) for r, k in zip(levels, (3, 8, 1))]
    for badk in (0, 17):
        steps[1] = badk
        assert L.sg_batch_ca_plan_host(n, lv, steps, pa, pb, rho, img, nbytes, 0x10000, nbytes,
                                       ctypes.byref(plan)) == sg.SG_EINVAL
    # a launch needs k >= every gasket's count (checked before any CUDA call)
    steps[1] = 8
    L.sg_batch_ca_plan_host(n, lv, steps, pa, pb, rho, img, nbytes, 0x10000, nbytes,
                            ctypes.byref(plan))
    assert L.sg_batch_ca_steps(ctypes.byref(plan), 0, 4, None, None) == sg.SG_EINVAL
    assert L.sg_batch_ca_step(ctypes.byref(plan), 0, None, None) == sg.SG_EINVAL
    g = ctypes.c_void_p()
    assert L.sg_batch_ca_graph_create_fused(ctypes.byref(plan), 16, 8, 0, None,
                                            ctypes.byref(g)) == sg.SG_EINVAL
