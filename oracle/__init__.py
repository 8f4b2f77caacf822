"""CPU oracle for the embedded Sierpinski-gasket hot path (arXiv:1706.04552).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library
(``paper_1706_04552_gb300``) never imports it, and it imports nothing from the
product: the two share no code.  Inputs both sides consume come from the seeded
generators in ``paper_1706_04552_gb300.inputs``, which hold none of the
method's arithmetic and are never imported here.

The arithmetic lives in ``sg_oracle.c`` (plain single-threaded C, double
precision for the diffusion step); this module only compiles it with gcc and
marshals numpy arrays.  Every function is pinned by the CPU tests in
``tests/test_oracle_pins.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

U8, F32 = 0, 1
VAL_CONST, VAL_LINEAR31, VAL_HASH = 0, 1, 2
MAP_LAMBDA, MAP_BBOX, MAP_LAMBDA_LUT, MAP_LAMBDA_UNROLL = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``sg_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, no
    fast-math, no contraction so double results follow the source order)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SG_ORACLE_LIB points the wrapper at another build of sg_oracle.c;
        # the mutation test uses it to load copies with planted mistakes.
        path = os.environ.get("SG_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        u64, i64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
        vp = ctypes.c_void_p
        p_u64 = ctypes.POINTER(ctypes.c_uint64)
        lib.or_member.argtypes = [u64, u64]
        lib.or_member.restype = i32
        lib.or_member_paper.argtypes = [i32, u64, u64]
        lib.or_member_paper.restype = i32
        lib.or_gasket_recursive.argtypes = [i32, vp]
        lib.or_gasket_recursive.restype = None
        lib.or_count_members.argtypes = [i32]
        lib.or_count_members.restype = u64
        lib.or_pi_extent.argtypes = [i32, p_u64, p_u64]
        lib.or_pi_extent.restype = None
        lib.or_lambda_paper.argtypes = [i32, u64, u64, p_u64, p_u64]
        lib.or_lambda_paper.restype = None
        lib.or_omega_of_index.argtypes = [i32, i32, u64, p_u64, p_u64]
        lib.or_omega_of_index.restype = None
        lib.or_block_of_index.argtypes = [i32, i32, u64, p_u64, p_u64]
        lib.or_block_of_index.restype = None
        lib.or_block_map.argtypes = [i32, i32, vp, vp]
        lib.or_block_map.restype = None
        lib.or_launch_counts.argtypes = [i32, i32, i32, p_u64, p_u64]
        lib.or_launch_counts.restype = None
        lib.or_splitmix64_next.argtypes = [u64]
        lib.or_splitmix64_next.restype = u64
        lib.or_cell_hash.argtypes = [i32, u64, u64, u64]
        lib.or_cell_hash.restype = u64
        lib.or_map_write_rows.argtypes = [i32, i32, vp, u64, u64, i32, u64]
        lib.or_map_write_rows.restype = None
        lib.or_ca_step_region.argtypes = [i32, i64, i64, i64, i64, vp, vp]
        lib.or_ca_step_region.restype = None
        lib.or_diffuse_step_region.argtypes = [i32, i64, i64, i64, i64, vp, vp,
                                               ctypes.c_double]
        lib.or_diffuse_step_region.restype = None
        lib.or_write_expected_at.argtypes = [i32, i32, i32, u64, u64, vp, vp, vp, vp]
        lib.or_write_expected_at.restype = None
        lib.or_compact_cells.argtypes = [i32, i32, i32, vp, vp]
        lib.or_compact_cells.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# --------------------------------------------------------------------------
# Membership (Section I, Section III-A, Section III-D)
# --------------------------------------------------------------------------

def member(x: int, y: int) -> bool:
    return bool(_load().or_member(x, y))


def member_paper(r: int, x: int, y: int) -> bool:
    return bool(_load().or_member_paper(r, x, y))


def member_grid(r: int) -> np.ndarray:
    """n x n uint8 map of (x & y) == 0, evaluated cell by cell in C."""
    n = 1 << r
    g = np.zeros((n, n), dtype=np.uint8)
    # the write pass with a constant 1 on a zero grid is exactly the map
    _load().or_map_write_rows(r, U8, _ptr(g), 0, n, VAL_CONST, 1)
    return g


def gasket_recursive(r: int) -> np.ndarray:
    n = 1 << r
    bm = np.zeros((n, n), dtype=np.uint8)
    _load().or_gasket_recursive(r, _ptr(bm))
    return bm


def count_members(r: int) -> int:
    return int(_load().or_count_members(r))


# --------------------------------------------------------------------------
# lambda(omega), Theorem 1
# --------------------------------------------------------------------------

def pi_extent(rb: int) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().or_pi_extent(rb, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def lambda_paper(rb: int, wx: int, wy: int) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().or_lambda_paper(rb, wx, wy, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


ORDER_ROWMAJOR, ORDER_INTERLEAVED = 0, 1


def omega_of_index(rb: int, q: int, order: int = ORDER_ROWMAJOR) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().or_omega_of_index(rb, order, q, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def block_of_index(rb: int, q: int, order: int = ORDER_ROWMAJOR) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().or_block_of_index(rb, order, q, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def block_map(rb: int, order: int = ORDER_ROWMAJOR) -> tuple[np.ndarray, np.ndarray]:
    total = 3 ** rb
    bx = np.zeros(total, dtype=np.uint32)
    by = np.zeros(total, dtype=np.uint32)
    _load().or_block_map(rb, order, _ptr(bx), _ptr(by))
    return bx, by


def launch_counts(r: int, s: int, map_kind: int) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().or_launch_counts(r, s, map_kind, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


# --------------------------------------------------------------------------
# Values and the map-and-write pass (Section IV)
# --------------------------------------------------------------------------

def splitmix64_next(state: int) -> int:
    return int(_load().or_splitmix64_next(state & (2**64 - 1)))


def cell_hash(r: int, x: int, y: int, seed: int) -> int:
    return int(_load().or_cell_hash(r, x, y, seed & (2**64 - 1)))


def map_write(r: int, grid: np.ndarray, value_kind: int, value: int,
              y0: int = 0, y1: int | None = None) -> np.ndarray:
    """Write pass over rows [y0, y1) of the level-r grid, in place.  ``grid``
    holds exactly those rows (uint8 or float32, pitch n)."""
    n = 1 << r
    y1 = n if y1 is None else y1
    assert grid.shape == (y1 - y0, n)
    dt = U8 if grid.dtype == np.uint8 else F32
    assert grid.dtype in (np.uint8, np.float32)
    _load().or_map_write_rows(r, dt, _ptr(grid), y0, y1, value_kind,
                              value & (2**64 - 1))
    return grid


def write_expected_at(r: int, dtype, value_kind: int, value: int, xs, ys,
                      before) -> np.ndarray:
    """Content of the listed cells after the write pass: v(x, y) at gasket
    cells, ``before`` elsewhere (one value per listed cell)."""
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    ys = np.ascontiguousarray(ys, dtype=np.uint64)
    before = np.ascontiguousarray(before, dtype=dtype)
    out = np.empty(len(xs), dtype=dtype)
    dt = U8 if np.dtype(dtype) == np.uint8 else F32
    _load().or_write_expected_at(r, dt, value_kind, value & (2**64 - 1), len(xs),
                                 _ptr(xs), _ptr(ys), _ptr(before), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Stencils
# --------------------------------------------------------------------------

def ca_step(r: int, state: np.ndarray, x0: int = 0, y0: int = 0) -> np.ndarray:
    """One gasket-restricted B3/S23 step of the region whose top-left cell is
    (x0, y0); ``state`` is that region (uint8, h x w)."""
    assert state.dtype == np.uint8 and state.ndim == 2
    state = np.ascontiguousarray(state)
    h, w = state.shape
    out = np.empty_like(state)
    _load().or_ca_step_region(r, x0, y0, w, h, _ptr(state), _ptr(out))
    return out


def diffuse_step(r: int, u: np.ndarray, alpha: float = 0.2,
                 x0: int = 0, y0: int = 0) -> np.ndarray:
    """One explicit diffusion step in double precision of the region whose
    top-left cell is (x0, y0)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    h, w = u.shape
    out = np.empty_like(u)
    _load().or_diffuse_step_region(r, x0, y0, w, h, _ptr(u), _ptr(out),
                                   float(alpha))
    return out


def ca_steps(r: int, state: np.ndarray, steps: int, x0: int = 0,
             y0: int = 0) -> np.ndarray:
    for _ in range(steps):
        state = ca_step(r, state, x0, y0)
    return state


def diffuse_steps(r: int, u: np.ndarray, steps: int, alpha: float = 0.2,
                  x0: int = 0, y0: int = 0) -> np.ndarray:
    u = np.asarray(u, dtype=np.float64)
    for _ in range(steps):
        u = diffuse_step(r, u, alpha, x0, y0)
    return u


# --------------------------------------------------------------------------
# Compact storage: only the 3^r gasket cells, tile by tile in launch order
# --------------------------------------------------------------------------

def compact_cells(r: int, s: int, order: int = ORDER_INTERLEAVED):
    """(xs, ys): the cell that each element of a level-r compact array with
    tile side 2^s holds (3^r entries each, uint64)."""
    assert 0 <= s <= min(r, 6)
    total = 3 ** r
    xs = np.zeros(total, dtype=np.uint64)
    ys = np.zeros(total, dtype=np.uint64)
    _load().or_compact_cells(r, s, order, _ptr(xs), _ptr(ys))
    return xs, ys


def compact_pack(r: int, s: int, grid: np.ndarray, order: int = ORDER_INTERLEAVED):
    """The compact array of an embedded n x n grid: its gasket cells, read in
    the compact order."""
    xs, ys = compact_cells(r, s, order)
    return np.asarray(grid)[ys.astype(np.int64), xs.astype(np.int64)].copy()


def compact_unpack(r: int, s: int, compact: np.ndarray, grid: np.ndarray,
                   order: int = ORDER_INTERLEAVED):
    """Write a compact array's elements into their cells of ``grid`` (in
    place); every other cell keeps its content."""
    xs, ys = compact_cells(r, s, order)
    grid[ys.astype(np.int64), xs.astype(np.int64)] = compact
    return grid


def compact_ca_step(r: int, s: int, compact: np.ndarray,
                    order: int = ORDER_INTERLEAVED) -> np.ndarray:
    """One CA step on a compact state: the embedded step of the state it
    stands for (off-gasket cells 0), read back in the compact order."""
    n = 1 << r
    g = compact_unpack(r, s, compact, np.zeros((n, n), dtype=np.uint8), order)
    return compact_pack(r, s, ca_step(r, g), order)


def compact_diffuse_step(r: int, s: int, compact: np.ndarray, alpha: float = 0.2,
                         order: int = ORDER_INTERLEAVED) -> np.ndarray:
    """One diffusion step (double precision) on a compact field, through the
    embedded step as for compact_ca_step."""
    n = 1 << r
    g = compact_unpack(r, s, np.asarray(compact, dtype=np.float64),
                       np.zeros((n, n), dtype=np.float64), order)
    return compact_pack(r, s, diffuse_step(r, g, alpha), order)
