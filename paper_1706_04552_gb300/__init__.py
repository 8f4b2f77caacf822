"""paper_1706_04552_gb300 -- GB300 (sm_103a) block-space mapping for embedded
Sierpinski gaskets (Navarro, Bustos, Vega, Hitschfeld, arXiv:1706.04552).

Python binding over libsg.so (C ABI in include/sg.h).  The binding only
marshals arguments: every step of the hot path runs in the library's CUDA
kernels, and there is no CPU fallback -- if libsg.so is missing or cannot be
loaded, every call raises.

Two layers:
  * ``sg_map_write``, ``sg_ca_step``, ``sg_diffuse_step``, ``sg_block_map``,
    ``sg_launch_stats``: the C functions with the C names, taking raw
    pointers (ints) and a raw cudaStream_t (int, 0 = legacy default stream);
  * ``map_write``, ``ca_step``, ``diffuse_step``, ``block_map``: the same
    calls on torch tensors, checking device, dtype, shape and contiguity and
    launching on the current torch stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "SGError", "lib", "lib_path",
    "sg_map_write", "sg_ca_step", "sg_diffuse_step", "sg_block_map",
    "sg_map_write_ex", "sg_ca_step_ex", "sg_diffuse_step_ex", "LaunchOpts", "launch_opts",
    "sg_ca_steps", "sg_diffuse_steps", "FUSE_MAX",
    "sg_launch_stats", "sg_status_str", "sg_abi_version", "sg_device_status",
    "device_status", "sg_wait_selftest", "wait_selftest",
    "sg_compact_pack", "sg_compact_unpack", "sg_compact_map_write", "sg_compact_ca_step",
    "sg_compact_diffuse_step", "sg_compact_ca_steps", "compact_size", "compact_pack",
    "compact_unpack", "compact_map_write", "compact_ca_step", "compact_ca_steps",
    "compact_diffuse_step", "sg_compact_map_write_mapped", "compact_map_write_mapped",
    "CABatch", "Graph", "BatchPlan", "Sched", "SchedGasketInfo", "SchedResult",
    "map_write", "map_write_host", "map_write_mapped", "sg_map_write_mapped", "ca_step",
    "diffuse_step", "ca_steps", "diffuse_steps",
    "block_map", "launch_stats",
    "MAPS", "DTYPES", "VALUES", "ORDERS", "STORES",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_build", "libsg.so")

SG_OK, SG_EINVAL, SG_ECUDA, SG_ENOMEM, SG_ETIMEOUT, SG_EUNSUPPORTED = range(6)
MAPS = {"lambda": 0, "bbox": 1, "lambda_lut": 2, "lambda_unroll": 3}
DTYPES = {"u8": 0, "f32": 1}
VALUES = {"const": 0, "linear31": 1, "hash": 2}
ORDERS = {"rowmajor": 0, "interleaved": 1}
STORES = {"auto": 0, "scatter": 1, "staged": 2, "tma": 3, "fill": 4, "sector": 5, "merge": 6,
          "masked": 7}


class LaunchOpts(ctypes.Structure):
    """sg_launch_opts of include/sg.h."""
    _fields_ = [("order", ctypes.c_int), ("store", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class BatchPlan(ctypes.Structure):
    """sg_batch_plan of include/sg.h."""
    _fields_ = [("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("count", ctypes.c_int), ("rho", ctypes.c_int),
                ("total_tiles", ctypes.c_uint32), ("max_level", ctypes.c_uint32),
                ("reserved", ctypes.c_int * 4)]


def launch_opts(order=None, store=None, ctas_per_sm=None):
    """An sg_launch_opts (or None when every field is the default)."""
    if order is None and store is None and ctas_per_sm is None:
        return None
    o = LaunchOpts()
    o.order = -1 if order is None else (ORDERS[order] if isinstance(order, str) else int(order))
    o.store = 0 if store is None else (STORES[store] if isinstance(store, str) else int(store))
    o.ctas_per_sm = 0 if ctas_per_sm is None else int(ctas_per_sm)
    return o

_lock = threading.Lock()
_lib = None


class SGError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str = ""):
        self.status = status
        msg = f"{fn} failed: {sg_status_str(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


def lib_path() -> str:
    return os.environ.get("SG_LIB", _LIB_PATH)


class SchedGasketInfo(ctypes.Structure):
    """sg_sched_gasket_info of include/sg_sched.h."""
    _fields_ = [("level", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("head_left", ctypes.c_int32), ("resident", ctypes.c_int32),
                ("cur", ctypes.c_uint64), ("nxt", ctypes.c_uint64),
                ("last_use", ctypes.c_uint64), ("steps_done", ctypes.c_uint64)]


class SchedResult(ctypes.Structure):
    """sg_sched_result of include/sg_sched.h."""
    _fields_ = [("completed", ctypes.c_void_p), ("completed_gasket", ctypes.c_void_p),
                ("failed", ctypes.c_void_p), ("failed_gasket", ctypes.c_void_p),
                ("failed_steps_run", ctypes.c_void_p), ("max_entries", ctypes.c_int32),
                ("n_completed", ctypes.c_int32), ("n_failed", ctypes.c_int32),
                ("active", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("cell_steps", ctypes.c_uint64), ("iteration", ctypes.c_uint64)]


def lib() -> ctypes.CDLL:
    """Load libsg.so (built in-tree by ``paper_1706_04552_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(
                f"libsg.so not found at {path}: build it with "
                "`python -m paper_1706_04552_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(path)
        i32, u64, vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        p_u64 = ctypes.POINTER(ctypes.c_uint64)
        L.sg_map_write.argtypes = [i32, i32, i32, i32, vp, i32, u64, vp]
        L.sg_map_write.restype = i32
        L.sg_ca_step.argtypes = [i32, i32, i32, vp, vp, vp]
        L.sg_ca_step.restype = i32
        L.sg_diffuse_step.argtypes = [i32, i32, i32, vp, vp, ctypes.c_float, vp]
        L.sg_diffuse_step.restype = i32
        L.sg_block_map.argtypes = [i32, i32, vp, vp, vp]
        L.sg_block_map.restype = i32
        p_opts = ctypes.POINTER(LaunchOpts)
        L.sg_map_write_ex.argtypes = [i32, i32, i32, i32, vp, i32, u64, p_opts, vp]
        L.sg_map_write_ex.restype = i32
        L.sg_ca_step_ex.argtypes = [i32, i32, i32, vp, vp, p_opts, vp]
        L.sg_ca_step_ex.restype = i32
        L.sg_diffuse_step_ex.argtypes = [i32, i32, i32, vp, vp, ctypes.c_float, p_opts, vp]
        L.sg_diffuse_step_ex.restype = i32
        L.sg_map_write_mapped.argtypes = [i32, i32, i32, i32, vp, i32, u64, p_opts, vp]
        L.sg_map_write_mapped.restype = i32
        L.sg_ca_steps.argtypes = [i32, i32, i32, vp, vp, i32, p_opts, vp]
        L.sg_ca_steps.restype = i32
        L.sg_diffuse_steps.argtypes = [i32, i32, i32, vp, vp, ctypes.c_float, i32, p_opts, vp]
        L.sg_diffuse_steps.restype = i32
        L.sg_launch_stats.argtypes = [i32, i32, i32, p_u64, p_u64]
        L.sg_launch_stats.restype = i32
        L.sg_status_str.argtypes = [i32]
        L.sg_status_str.restype = ctypes.c_char_p
        L.sg_last_error_string.argtypes = []
        L.sg_last_error_string.restype = ctypes.c_char_p
        p_plan = ctypes.POINTER(BatchPlan)
        L.sg_batch_workspace_bytes.argtypes = [i32]
        L.sg_batch_workspace_bytes.restype = u64
        L.sg_batch_ca_plan.argtypes = [i32, vp, vp, vp, i32, vp, u64, p_plan, vp]
        L.sg_batch_ca_plan.restype = i32
        L.sg_batch_ca_step.argtypes = [p_plan, i32, p_opts, vp]
        L.sg_batch_ca_step.restype = i32
        L.sg_batch_ca_graph_create.argtypes = [p_plan, i32, i32, p_opts, ctypes.POINTER(vp)]
        L.sg_batch_ca_graph_create.restype = i32
        L.sg_graph_launch.argtypes = [vp, vp]
        L.sg_graph_launch.restype = i32
        L.sg_graph_destroy.argtypes = [vp]
        L.sg_graph_destroy.restype = i32
        L.sg_batch_ca_autotune.argtypes = [i32, vp, vp, vp, vp, u64, i32, p_plan, p_opts, vp]
        L.sg_batch_ca_autotune.restype = i32
        L.sg_batch_ca_steps.argtypes = [p_plan, i32, i32, p_opts, vp]
        L.sg_batch_ca_steps.restype = i32
        L.sg_batch_ca_graph_create_fused.argtypes = [p_plan, i32, i32, i32, p_opts,
                                                     ctypes.POINTER(vp)]
        L.sg_batch_ca_graph_create_fused.restype = i32
        L.sg_batch_ca_autotune_fused.argtypes = [i32, vp, vp, vp, vp, u64, i32, i32, p_plan,
                                                 p_opts, vp]
        L.sg_batch_ca_autotune_fused.restype = i32
        L.sg_device_status.argtypes = [vp]
        L.sg_device_status.restype = i32
        L.sg_wait_selftest.argtypes = [i32, i32, u64, vp]
        L.sg_wait_selftest.restype = i32
        L.sg_compact_pack.argtypes = [i32, i32, i32, vp, vp, p_opts, vp]
        L.sg_compact_pack.restype = i32
        L.sg_compact_unpack.argtypes = [i32, i32, i32, vp, vp, p_opts, vp]
        L.sg_compact_unpack.restype = i32
        L.sg_compact_map_write.argtypes = [i32, i32, i32, vp, i32, u64, p_opts, vp]
        L.sg_compact_map_write.restype = i32
        L.sg_compact_ca_step.argtypes = [i32, i32, vp, vp, p_opts, vp]
        L.sg_compact_ca_step.restype = i32
        L.sg_compact_map_write_mapped.argtypes = [i32, i32, i32, vp, i32, u64, p_opts, vp]
        L.sg_compact_map_write_mapped.restype = i32
        L.sg_compact_ca_steps.argtypes = [i32, i32, i32, vp, vp, p_opts, vp]
        L.sg_compact_ca_steps.restype = i32
        L.sg_compact_diffuse_step.argtypes = [i32, i32, vp, vp, ctypes.c_float, p_opts, vp]
        L.sg_compact_diffuse_step.restype = i32
        L.sg_abi_version.argtypes = []
        L.sg_abi_version.restype = i32
        # the serving scheduler's core (include/sg_sched.h)
        L.sg_batch_ca_plan_host.argtypes = [i32, vp, vp, vp, vp, i32, vp, u64, vp, u64, p_plan]
        L.sg_batch_ca_plan_host.restype = i32
        L.sg_sched_create.argtypes = [i32, vp, i32, i32, p_opts, ctypes.POINTER(vp)]
        L.sg_sched_create.restype = i32
        L.sg_sched_destroy.argtypes = [vp]
        L.sg_sched_destroy.restype = i32
        L.sg_sched_set_buffers.argtypes = [vp, i32, vp, vp]
        L.sg_sched_set_buffers.restype = i32
        L.sg_sched_submit.argtypes = [vp, i32, vp, vp, vp]
        L.sg_sched_submit.restype = i32
        L.sg_sched_waiting.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        L.sg_sched_waiting.restype = i32
        L.sg_sched_gasket.argtypes = [vp, i32, ctypes.POINTER(SchedGasketInfo)]
        L.sg_sched_gasket.restype = i32
        L.sg_sched_drop.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(i32)]
        L.sg_sched_drop.restype = i32
        L.sg_sched_step.argtypes = [vp, vp, ctypes.POINTER(SchedResult)]
        L.sg_sched_step.restype = i32
        L.sg_sched_inject_launch_failure.argtypes = [vp, i32]
        L.sg_sched_inject_launch_failure.restype = i32
        _lib = L
        return L


# ---------------------------------------------------------------- raw C layer

def sg_status_str(status: int) -> str:
    return lib().sg_status_str(int(status)).decode()


def sg_abi_version() -> int:
    return int(lib().sg_abi_version())


def sg_device_status(stream=0) -> int:
    return int(lib().sg_device_status(stream))


def device_status(stream=None):
    """Raise SGError if a kernel recorded a bounded wait that gave up since
    the last check (synchronises the stream)."""
    import torch
    h = torch.cuda.current_stream().cuda_stream if stream is None else (
        stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check("sg_device_status", sg_device_status(h))


def sg_wait_selftest(blocks, arrive, limit_ns, stream=0) -> int:
    return int(lib().sg_wait_selftest(blocks, 1 if arrive else 0, limit_ns, stream))


def wait_selftest(blocks=152, arrive=False, limit_ns=50_000_000, stream=None):
    """Launch the bounded-wait self-test: every block waits on an mbarrier
    that nothing arrives on (unless `arrive`), gives up after `limit_ns` and
    records SG_ETIMEOUT for device_status() to report."""
    import torch
    h = torch.cuda.current_stream().cuda_stream if stream is None else (
        stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check("sg_wait_selftest", sg_wait_selftest(blocks, arrive, limit_ns, h))


def _check(fn: str, status: int) -> None:
    if status != SG_OK:
        detail = lib().sg_last_error_string().decode() if status == SG_ECUDA else ""
        raise SGError(fn, status, detail)


def sg_map_write(r, rho, map_kind, dtype, grid_ptr, value_kind, value_or_seed,
                 stream=0) -> int:
    return int(lib().sg_map_write(r, rho, map_kind, dtype, grid_ptr, value_kind,
                                  value_or_seed & (2**64 - 1), stream))


def sg_ca_step(r, rho, map_kind, in_ptr, out_ptr, stream=0) -> int:
    return int(lib().sg_ca_step(r, rho, map_kind, in_ptr, out_ptr, stream))


def sg_diffuse_step(r, rho, map_kind, in_ptr, out_ptr, alpha, stream=0) -> int:
    return int(lib().sg_diffuse_step(r, rho, map_kind, in_ptr, out_ptr, alpha, stream))


def sg_map_write_ex(r, rho, map_kind, dtype, grid_ptr, value_kind, value_or_seed,
                    opts=None, stream=0) -> int:
    return int(lib().sg_map_write_ex(r, rho, map_kind, dtype, grid_ptr, value_kind,
                                     value_or_seed & (2**64 - 1), _opts_ref(opts), stream))


def sg_ca_step_ex(r, rho, map_kind, in_ptr, out_ptr, opts=None, stream=0) -> int:
    return int(lib().sg_ca_step_ex(r, rho, map_kind, in_ptr, out_ptr, _opts_ref(opts), stream))


def sg_diffuse_step_ex(r, rho, map_kind, in_ptr, out_ptr, alpha, opts=None, stream=0) -> int:
    return int(lib().sg_diffuse_step_ex(r, rho, map_kind, in_ptr, out_ptr, alpha,
                                        _opts_ref(opts), stream))


def sg_map_write_mapped(r, rho, map_kind, dtype, host_ptr, value_kind, value_or_seed,
                        opts=None, stream=0) -> int:
    return int(lib().sg_map_write_mapped(r, rho, map_kind, dtype, host_ptr, value_kind,
                                         value_or_seed & (2**64 - 1), _opts_ref(opts), stream))


def sg_ca_steps(r, rho, map_kind, in_ptr, out_ptr, k, opts=None, stream=0) -> int:
    return int(lib().sg_ca_steps(r, rho, map_kind, in_ptr, out_ptr, k, _opts_ref(opts), stream))


def sg_diffuse_steps(r, rho, map_kind, in_ptr, out_ptr, alpha, k, opts=None, stream=0) -> int:
    return int(lib().sg_diffuse_steps(r, rho, map_kind, in_ptr, out_ptr, alpha, k,
                                      _opts_ref(opts), stream))


def sg_block_map(rb, order, bx_ptr, by_ptr, stream=0) -> int:
    return int(lib().sg_block_map(rb, order, bx_ptr, by_ptr, stream))


def _opts_ref(opts):
    return None if opts is None else ctypes.byref(opts)


def sg_launch_stats(r, rho, map_kind):
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    st = int(lib().sg_launch_stats(r, rho, map_kind, ctypes.byref(a), ctypes.byref(b)))
    return st, a.value, b.value


# ------------------------------------------------------------- tensor layer

def _map_id(m) -> int:
    return MAPS[m] if isinstance(m, str) else int(m)


def _stream_handle(t, stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream(t.device).cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class _NoDeviceSwitch:
    def __enter__(self):
        return None

    def __exit__(self, *exc):
        return False


def _on_device(t):
    """Make t's device current for the call (skipped when it already is)."""
    import torch
    if t.device.index is None or t.device.index == torch.cuda.current_device():
        return _NoDeviceSwitch()
    return torch.cuda.device(t.device)


def _grid_check(t, r, dtypes, name):
    import torch
    n = 1 << r
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor (there is no CPU path)")
    if t.dtype not in dtypes:
        raise TypeError(f"{name}: dtype {t.dtype} not in {dtypes}")
    if not t.is_contiguous() or t.numel() != n * n:
        raise ValueError(f"{name}: expected a contiguous tensor of {n}*{n} elements")


def map_write(grid, r: int, rho: int, map="lambda", value="hash", value_or_seed=1,
              stream=None, order=None, store=None, ctas_per_sm=None):
    """Map-and-write pass on a CUDA tensor (uint8 or float32, n*n elements)."""
    import torch
    _grid_check(grid, r, (torch.uint8, torch.float32), "grid")
    dt = DTYPES["u8"] if grid.dtype == torch.uint8 else DTYPES["f32"]
    vk = VALUES[value] if isinstance(value, str) else int(value)
    opts = launch_opts(order, store, ctas_per_sm)
    with _on_device(grid):
        _check("sg_map_write", sg_map_write_ex(r, rho, _map_id(map), dt, grid.data_ptr(), vk,
                                               value_or_seed, opts,
                                               _stream_handle(grid, stream)))
    return grid


def map_write_host(host_grid, dev_grid, r: int, rho: int, map="lambda", value="hash",
                   value_or_seed=1, stream=None, order=None, store=None):
    """Write pass on a grid that lives in host memory: copies ``host_grid``
    (a pinned CPU tensor) into the caller's device buffer ``dev_grid``,
    launches the pass, and copies the result back, all on one stream.
    Returns without synchronising; the copy back is complete once the stream
    is."""
    import torch
    if host_grid.is_cuda or not host_grid.is_contiguous():
        raise TypeError("host_grid: expected a contiguous CPU tensor")
    if host_grid.dtype != dev_grid.dtype or host_grid.numel() != dev_grid.numel():
        raise ValueError("host_grid and dev_grid must match in dtype and size")
    st = stream if stream is not None else torch.cuda.current_stream(dev_grid.device)
    with torch.cuda.stream(st):
        dev_grid.copy_(host_grid, non_blocking=True)
        map_write(dev_grid, r, rho, map, value, value_or_seed, st, order=order, store=store)
        host_grid.copy_(dev_grid, non_blocking=True)
    return host_grid


def map_write_mapped(host_grid, r: int, rho: int, map="lambda", value="hash", value_or_seed=1,
                     stream=None, order=None, store=None, device=None):
    """Write pass on a grid kept in pinned host memory, read and written in
    place by the kernel over the host link (sg_map_write_mapped).  Returns
    without synchronising: the result is in ``host_grid`` once the stream is
    complete."""
    import torch
    if host_grid.is_cuda or not host_grid.is_contiguous() or not host_grid.is_pinned():
        raise TypeError("host_grid: expected a contiguous pinned CPU tensor")
    if host_grid.dtype not in (torch.uint8, torch.float32):
        raise TypeError("host_grid: expected uint8 or float32")
    if host_grid.numel() != 1 << (2 * r):
        raise ValueError(f"host_grid: expected {1 << (2 * r)} elements for level {r}")
    dt = DTYPES["u8"] if host_grid.dtype == torch.uint8 else DTYPES["f32"]
    vk = VALUES[value] if isinstance(value, str) else int(value)
    opts = launch_opts(order, store, None)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    if stream is None:
        st = torch.cuda.current_stream(dev).cuda_stream
    else:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    with torch.cuda.device(dev):
        _check("sg_map_write_mapped", sg_map_write_mapped(r, rho, _map_id(map), dt,
                                                          host_grid.data_ptr(), vk,
                                                          value_or_seed, opts, st))
    return host_grid


def ca_step(inp, out, r: int, rho: int, map="lambda", stream=None, order=None,
            ctas_per_sm=None, staging=None):
    """One CA step; staging="tma" stages each tile and its halo with one
    bulk tensor copy (rho 32 and 64) instead of 16-byte chunk copies."""
    import torch
    _grid_check(inp, r, (torch.uint8,), "in")
    _grid_check(out, r, (torch.uint8,), "out")
    opts = launch_opts(order, _staging_store(staging), ctas_per_sm)
    with _on_device(inp):
        _check("sg_ca_step", sg_ca_step_ex(r, rho, _map_id(map), inp.data_ptr(),
                                           out.data_ptr(), opts, _stream_handle(inp, stream)))
    return out


def diffuse_step(inp, out, r: int, rho: int, alpha: float = 0.2, map="lambda",
                 stream=None, order=None, ctas_per_sm=None, staging=None):
    """One diffusion step; staging="tma" stages each tile and its halo with
    one bulk tensor copy (rho 16 and 32) instead of 16-byte chunk copies."""
    import torch
    _grid_check(inp, r, (torch.float32,), "in")
    _grid_check(out, r, (torch.float32,), "out")
    opts = launch_opts(order, _staging_store(staging), ctas_per_sm)
    with _on_device(inp):
        _check("sg_diffuse_step", sg_diffuse_step_ex(r, rho, _map_id(map), inp.data_ptr(),
                                                     out.data_ptr(), float(alpha), opts,
                                                     _stream_handle(inp, stream)))
    return out


def _staging_store(staging):
    if staging in (None, "chunks"):
        return None
    if staging == "tma":
        return "tma"
    raise ValueError(f"staging must be None, 'chunks' or 'tma', not {staging!r}")


FUSE_MAX = 16     # SG_FUSE_MAX: most steps one sg_ca_steps / sg_diffuse_steps launch fuses


def ca_steps(inp, out, r: int, rho: int, k: int, map="lambda", stream=None, order=None,
             ctas_per_sm=None):
    """k CA steps in one launch: out = step^k(inp); inp is left unchanged."""
    import torch
    _grid_check(inp, r, (torch.uint8,), "in")
    _grid_check(out, r, (torch.uint8,), "out")
    opts = launch_opts(order, None, ctas_per_sm)
    with _on_device(inp):
        _check("sg_ca_steps", sg_ca_steps(r, rho, _map_id(map), inp.data_ptr(), out.data_ptr(),
                                          int(k), opts, _stream_handle(inp, stream)))
    return out


def diffuse_steps(inp, out, r: int, rho: int, k: int, alpha: float = 0.2, map="lambda",
                  stream=None, order=None, ctas_per_sm=None):
    """k diffusion steps in one launch: out = step^k(inp); inp is left unchanged."""
    import torch
    _grid_check(inp, r, (torch.float32,), "in")
    _grid_check(out, r, (torch.float32,), "out")
    opts = launch_opts(order, None, ctas_per_sm)
    with _on_device(inp):
        _check("sg_diffuse_steps", sg_diffuse_steps(r, rho, _map_id(map), inp.data_ptr(),
                                                    out.data_ptr(), float(alpha), int(k), opts,
                                                    _stream_handle(inp, stream)))
    return out


def block_map(rb: int, order="interleaved", device="cuda", stream=None):
    """Run the device lambda decode for every launch index; returns (bx, by)
    as uint32-valued int32 CUDA tensors (bit patterns, all values < 2^16)."""
    import torch
    total = 3 ** rb
    bx = torch.empty(total, dtype=torch.int32, device=device)
    by = torch.empty(total, dtype=torch.int32, device=device)
    oid = ORDERS[order] if isinstance(order, str) else int(order)
    with _on_device(bx):
        _check("sg_block_map", sg_block_map(rb, oid, bx.data_ptr(), by.data_ptr(),
                                            _stream_handle(bx, stream)))
    return bx, by


# ------------------------------------------------------------------ batches

class CABatch:
    """Many gaskets of uneven levels stepped together (sg_batch_* calls).

    levels: gasket levels; bufs_a / bufs_b: uint8 CUDA tensors of n_i*n_i
    cells (0 off the gasket; the state to step starts in bufs_a).  rho picks
    the tile side; autotune=K times K launches per candidate and plans with
    the fastest (rho, walking order, CTAs per SM) for launches of `fuse`
    steps (1: single steps, sg_batch_ca_step; more: sg_batch_ca_steps).  The
    work list lives in a workspace tensor this object owns."""

    def __init__(self, levels, bufs_a, bufs_b, rho=64, autotune=None, stream=None, fuse=1):
        import torch
        self.levels = [int(r) for r in levels]
        count = len(self.levels)
        if not (len(bufs_a) == len(bufs_b) == count):
            raise ValueError("one pair of buffers per gasket")
        for r, a, b in zip(self.levels, bufs_a, bufs_b):
            _grid_check(a, r, (torch.uint8,), "bufs_a")
            _grid_check(b, r, (torch.uint8,), "bufs_b")
        self.bufs_a, self.bufs_b = list(bufs_a), list(bufs_b)
        dev = self.bufs_a[0].device
        nbytes = int(lib().sg_batch_workspace_bytes(count))
        if nbytes == 0:
            raise ValueError(f"batch of {count} gaskets is out of range")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        lv = (ctypes.c_int * count)(*self.levels)
        pa = (ctypes.c_void_p * count)(*[t.data_ptr() for t in self.bufs_a])
        pb = (ctypes.c_void_p * count)(*[t.data_ptr() for t in self.bufs_b])
        self.plan = BatchPlan()
        self.opts = None
        st = _stream_handle(self.workspace, stream)
        with _on_device(self.workspace):
            if autotune and int(fuse) > 1:
                self.opts = LaunchOpts()
                _check("sg_batch_ca_autotune_fused", int(lib().sg_batch_ca_autotune_fused(
                    count, lv, pa, pb, self.workspace.data_ptr(), nbytes, int(autotune),
                    int(fuse), ctypes.byref(self.plan), ctypes.byref(self.opts), st)))
            elif autotune:
                self.opts = LaunchOpts()
                _check("sg_batch_ca_autotune", int(lib().sg_batch_ca_autotune(
                    count, lv, pa, pb, self.workspace.data_ptr(), nbytes, int(autotune),
                    ctypes.byref(self.plan), ctypes.byref(self.opts), st)))
            else:
                _check("sg_batch_ca_plan", int(lib().sg_batch_ca_plan(
                    count, lv, pa, pb, int(rho), self.workspace.data_ptr(), nbytes,
                    ctypes.byref(self.plan), st)))

    @property
    def rho(self):
        return self.plan.rho

    def step(self, parity=0, stream=None, order=None, ctas_per_sm=None):
        opts = self.opts if (order is None and ctas_per_sm is None) else launch_opts(
            order, None, ctas_per_sm)
        with _on_device(self.workspace):
            _check("sg_batch_ca_step", int(lib().sg_batch_ca_step(
                ctypes.byref(self.plan), int(parity), _opts_ref(opts),
                _stream_handle(self.workspace, stream))))

    def steps(self, k, parity=0, stream=None, order=None, ctas_per_sm=None):
        """k fused steps of every gasket in one launch (parity as for step)."""
        opts = self.opts if (order is None and ctas_per_sm is None) else launch_opts(
            order, None, ctas_per_sm)
        with _on_device(self.workspace):
            _check("sg_batch_ca_steps", int(lib().sg_batch_ca_steps(
                ctypes.byref(self.plan), int(parity), int(k), _opts_ref(opts),
                _stream_handle(self.workspace, stream))))

    def graph(self, steps, start_parity=0, fuse=1):
        """A CUDA graph of `steps` consecutive steps (see Graph), as launches
        of `fuse` fused steps (the last launch takes the remainder)."""
        h = ctypes.c_void_p()
        with _on_device(self.workspace):
            if int(fuse) > 1:
                _check("sg_batch_ca_graph_create_fused", int(lib().sg_batch_ca_graph_create_fused(
                    ctypes.byref(self.plan), int(steps), int(fuse), int(start_parity),
                    _opts_ref(self.opts), ctypes.byref(h))))
            else:
                _check("sg_batch_ca_graph_create", int(lib().sg_batch_ca_graph_create(
                    ctypes.byref(self.plan), int(steps), int(start_parity),
                    _opts_ref(self.opts), ctypes.byref(h))))
        return Graph(h, self)


class Graph:
    """An instantiated CUDA graph made by libsg; launch() replays it."""

    def __init__(self, handle, owner=None):
        self.handle = handle
        self._owner = owner            # keeps the workspace and buffers alive

    def launch(self, stream=None):
        import torch
        st = torch.cuda.current_stream().cuda_stream if stream is None else (
            stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check("sg_graph_launch", int(lib().sg_graph_launch(self.handle, st)))

    def close(self):
        if self.handle:
            lib().sg_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sched:
    """The serving scheduler's native core (include/sg_sched.h): per-gasket
    request queues and one batched iteration per step(), built and launched
    in C++.  Argument marshalling only; arrays are numpy."""

    def __init__(self, levels, rho=32, fuse=1, opts=None):
        import numpy as np
        self._np = np
        lv = np.ascontiguousarray(levels, dtype=np.int32)
        self.count = int(lv.size)
        h = ctypes.c_void_p()
        _check("sg_sched_create", int(lib().sg_sched_create(
            self.count, lv.ctypes.data, int(rho), int(fuse), _opts_ref(opts), ctypes.byref(h))))
        self._h = h
        n = max(self.count, 1)
        self._done = np.zeros(n, dtype=np.int64)
        self._done_g = np.zeros(n, dtype=np.int32)
        self._fail = np.zeros(n, dtype=np.int64)
        self._fail_g = np.zeros(n, dtype=np.int32)
        self._fail_ran = np.zeros(n, dtype=np.int32)
        self._res = SchedResult()
        self._res.completed = self._done.ctypes.data
        self._res.completed_gasket = self._done_g.ctypes.data
        self._res.failed = self._fail.ctypes.data
        self._res.failed_gasket = self._fail_g.ctypes.data
        self._res.failed_steps_run = self._fail_ran.ctypes.data
        self._res.max_entries = n
        self._wait = np.zeros(n, dtype=np.int32)

    def close(self):
        if self._h is not None and self._h.value:
            _check("sg_sched_destroy", int(lib().sg_sched_destroy(self._h)))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_buffers(self, g, cur_ptr, nxt_ptr):
        _check("sg_sched_set_buffers", int(lib().sg_sched_set_buffers(
            self._h, int(g), int(cur_ptr) or None, int(nxt_ptr) or None)))

    def submit(self, gaskets, requests, steps):
        np = self._np
        g = np.ascontiguousarray(gaskets, dtype=np.int32)
        r = np.ascontiguousarray(requests, dtype=np.int64)
        k = np.ascontiguousarray(steps, dtype=np.int32)
        if not (g.size == r.size == k.size):
            raise ValueError("one gasket, request id and step count per request")
        _check("sg_sched_submit", int(lib().sg_sched_submit(
            self._h, int(g.size), g.ctypes.data, r.ctypes.data, k.ctypes.data)))

    def waiting(self):
        n = ctypes.c_int(0)
        _check("sg_sched_waiting", int(lib().sg_sched_waiting(
            self._h, self._wait.ctypes.data, int(self._wait.size), ctypes.byref(n))))
        return self._wait[:n.value].copy()

    def gasket(self, g) -> SchedGasketInfo:
        info = SchedGasketInfo()
        _check("sg_sched_gasket", int(lib().sg_sched_gasket(self._h, int(g), ctypes.byref(info))))
        return info

    def drop(self, g):
        """Remove gasket g's queued requests: (request ids, steps run of each)."""
        np = self._np
        q = self.gasket(g).queued
        req = np.zeros(max(q, 1), dtype=np.int64)
        ran = np.zeros(max(q, 1), dtype=np.int32)
        n = ctypes.c_int(0)
        _check("sg_sched_drop", int(lib().sg_sched_drop(
            self._h, int(g), req.ctypes.data, ran.ctypes.data, int(req.size), ctypes.byref(n))))
        return req[:n.value], ran[:n.value]

    def inject_launch_failure(self, g):
        _check("sg_sched_inject_launch_failure",
               int(lib().sg_sched_inject_launch_failure(self._h, int(g))))

    def step(self, stream):
        """One iteration on `stream` (a torch stream or a raw handle).  Returns
        the SchedResult; completed()/failed() give its arrays."""
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check("sg_sched_step", int(lib().sg_sched_step(self._h, st, ctypes.byref(self._res))))
        return self._res

    def completed(self):
        n = self._res.n_completed
        return self._done[:n], self._done_g[:n]

    def failed(self):
        n = self._res.n_failed
        return self._fail[:n], self._fail_g[:n], self._fail_ran[:n]


def launch_stats(r: int, rho: int, map="lambda"):
    st, launched, useful = sg_launch_stats(r, rho, _map_id(map))
    _check("sg_launch_stats", st)
    return launched, useful


# ---------------------------------------------------------------- compact layout
# Arrays of the 3^r gasket cells only, tile by tile in launch order (layout in
# include/sg.h).  Raw C layer, then tensor functions.

def sg_compact_pack(r, rho, dtype, grid_ptr, compact_ptr, opts=None, stream=0) -> int:
    return int(lib().sg_compact_pack(r, rho, dtype, grid_ptr, compact_ptr,
                                     _opts_ref(opts), stream))


def sg_compact_unpack(r, rho, dtype, compact_ptr, grid_ptr, opts=None, stream=0) -> int:
    return int(lib().sg_compact_unpack(r, rho, dtype, compact_ptr, grid_ptr,
                                       _opts_ref(opts), stream))


def sg_compact_map_write(r, rho, dtype, compact_ptr, value_kind, value_or_seed, opts=None,
                         stream=0) -> int:
    return int(lib().sg_compact_map_write(r, rho, dtype, compact_ptr, value_kind,
                                          value_or_seed & (2**64 - 1), _opts_ref(opts),
                                          stream))


def sg_compact_ca_step(r, rho, in_ptr, out_ptr, opts=None, stream=0) -> int:
    return int(lib().sg_compact_ca_step(r, rho, in_ptr, out_ptr, _opts_ref(opts), stream))


def sg_compact_map_write_mapped(r, rho, dtype, host_ptr, value_kind, value_or_seed, opts=None,
                                stream=0) -> int:
    return int(lib().sg_compact_map_write_mapped(r, rho, dtype, host_ptr, value_kind,
                                                 value_or_seed & (2**64 - 1), _opts_ref(opts),
                                                 stream))


def sg_compact_ca_steps(r, rho, k, in_ptr, out_ptr, opts=None, stream=0) -> int:
    return int(lib().sg_compact_ca_steps(r, rho, k, in_ptr, out_ptr, _opts_ref(opts), stream))


def sg_compact_diffuse_step(r, rho, in_ptr, out_ptr, alpha, opts=None, stream=0) -> int:
    return int(lib().sg_compact_diffuse_step(r, rho, in_ptr, out_ptr, alpha,
                                             _opts_ref(opts), stream))


def compact_size(r: int) -> int:
    """Elements of a level-r compact array: the 3^r gasket cells."""
    return 3 ** r


def _compact_check(t, r, dtypes, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor (there is no CPU path)")
    if t.dtype not in dtypes:
        raise TypeError(f"{name}: dtype {t.dtype} not in {dtypes}")
    if not t.is_contiguous() or t.numel() != 3 ** r:
        raise ValueError(f"{name}: expected a contiguous tensor of 3^{r} elements")


def _dtype_id(t):
    import torch
    return DTYPES["u8"] if t.dtype == torch.uint8 else DTYPES["f32"]


def compact_pack(grid, compact, r: int, rho: int, order=None, stream=None, ctas_per_sm=None):
    """compact <- the gasket cells of the embedded ``grid`` (same dtype)."""
    import torch
    _grid_check(grid, r, (torch.uint8, torch.float32), "grid")
    _compact_check(compact, r, (grid.dtype,), "compact")
    with _on_device(grid):
        _check("sg_compact_pack", sg_compact_pack(
            r, rho, _dtype_id(grid), grid.data_ptr(), compact.data_ptr(),
            launch_opts(order, None, ctas_per_sm), _stream_handle(grid, stream)))
    return compact


def compact_unpack(compact, grid, r: int, rho: int, order=None, stream=None, ctas_per_sm=None):
    """The gasket cells of the embedded ``grid`` <- compact (others unchanged)."""
    import torch
    _grid_check(grid, r, (torch.uint8, torch.float32), "grid")
    _compact_check(compact, r, (grid.dtype,), "compact")
    with _on_device(grid):
        _check("sg_compact_unpack", sg_compact_unpack(
            r, rho, _dtype_id(grid), compact.data_ptr(), grid.data_ptr(),
            launch_opts(order, None, ctas_per_sm), _stream_handle(grid, stream)))
    return grid


def compact_map_write(compact, r: int, rho: int, value="hash", value_or_seed=1, order=None,
                      stream=None, ctas_per_sm=None):
    """Map-and-write pass on a compact array (uint8 or float32, 3^r elements)."""
    import torch
    _compact_check(compact, r, (torch.uint8, torch.float32), "compact")
    vk = VALUES[value] if isinstance(value, str) else int(value)
    with _on_device(compact):
        _check("sg_compact_map_write", sg_compact_map_write(
            r, rho, _dtype_id(compact), compact.data_ptr(), vk, value_or_seed,
            launch_opts(order, None, ctas_per_sm), _stream_handle(compact, stream)))
    return compact


def compact_map_write_mapped(host_compact, r: int, rho: int, value="hash", value_or_seed=1,
                             order=None, stream=None, device=None):
    """Compact write pass straight into a pinned CPU tensor of 3^r elements
    (sg_compact_map_write_mapped).  Returns without synchronising."""
    import torch
    if host_compact.is_cuda or not host_compact.is_contiguous() or not host_compact.is_pinned():
        raise TypeError("host_compact: expected a contiguous pinned CPU tensor")
    if host_compact.dtype not in (torch.uint8, torch.float32):
        raise TypeError("host_compact: expected uint8 or float32")
    if host_compact.numel() != 3 ** r:
        raise ValueError(f"host_compact: expected 3^{r} elements")
    vk = VALUES[value] if isinstance(value, str) else int(value)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    if stream is None:
        st = torch.cuda.current_stream(dev).cuda_stream
    else:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    with torch.cuda.device(dev):
        _check("sg_compact_map_write_mapped", sg_compact_map_write_mapped(
            r, rho, _dtype_id(host_compact), host_compact.data_ptr(), vk, value_or_seed,
            launch_opts(order, None, None), st))
    return host_compact


def compact_ca_step(inp, out, r: int, rho: int, order=None, stream=None, ctas_per_sm=None):
    import torch
    _compact_check(inp, r, (torch.uint8,), "in")
    _compact_check(out, r, (torch.uint8,), "out")
    with _on_device(inp):
        _check("sg_compact_ca_step", sg_compact_ca_step(
            r, rho, inp.data_ptr(), out.data_ptr(), launch_opts(order, None, ctas_per_sm),
            _stream_handle(inp, stream)))
    return out


def compact_ca_steps(inp, out, r: int, rho: int, k: int, order=None, stream=None,
                     ctas_per_sm=None):
    """k CA steps in one launch on compact states (rho = 64 for k > 1)."""
    import torch
    _compact_check(inp, r, (torch.uint8,), "in")
    _compact_check(out, r, (torch.uint8,), "out")
    with _on_device(inp):
        _check("sg_compact_ca_steps", sg_compact_ca_steps(
            r, rho, k, inp.data_ptr(), out.data_ptr(), launch_opts(order, None, ctas_per_sm),
            _stream_handle(inp, stream)))
    return out


def compact_diffuse_step(inp, out, r: int, rho: int, alpha: float = 0.2, order=None,
                         stream=None, ctas_per_sm=None):
    import torch
    _compact_check(inp, r, (torch.float32,), "in")
    _compact_check(out, r, (torch.float32,), "out")
    with _on_device(inp):
        _check("sg_compact_diffuse_step", sg_compact_diffuse_step(
            r, rho, inp.data_ptr(), out.data_ptr(), float(alpha),
            launch_opts(order, None, ctas_per_sm), _stream_handle(inp, stream)))
    return out
