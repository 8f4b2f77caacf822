"""Named workload presets (the sizes, seeds and launch configurations the
benchmark times and the full-size parity tests check).

Every input is synthetic and seeded (see ``inputs``).  Level r means an
n x n grid with n = 2^r; the gasket has 3^r cells.
"""
from __future__ import annotations

# Small end-to-end case: level 10 in a uint8 grid, rho = 16; a write pass of
# (x*31 + y) & 0xFF, then 16 double-buffered CA steps from Bernoulli(0.5)
# seeded with 0; lambda and bounding-box maps both run.
SMALL = dict(r=10, rho=16, write_value="linear31", write_seed=0,
             ca_p=0.5, ca_seed=0, ca_steps=16)

# Map-and-write sweep: levels 8..16 in uint8 and float32 grids, rho in
# {8, 16, 32, 64}, value = hash of (x, y) with seed 1.
WRITE_SWEEP = dict(levels=tuple(range(8, 17)), rhos=(8, 16, 32, 64),
                   dtypes=("u8", "f32"), value="hash", seed=1)

# The headline: the write pass at n = 2^16 into a zero-filled 4.3 GB uint8
# grid (the paper's benchmark: write into the gasket of a zero matrix).
# Map, rho, walking order and store path are the measured best on GB300;
# the bounding box and the float32 grid get their own measured best rho and
# store path (the write sweep).
WRITE_HEADLINE = dict(r=16, dtype="u8", value="hash", seed=1,
                      map="lambda_unroll", rho=64, order="interleaved", store="fill",
                      bbox_rho=64, bbox_store="sector", f32_rho=8, f32_store="sector")

# The same pass with stores that keep arbitrary off-gasket content
# (read-merge-write of whole 32-byte sectors, one lane per 32 x 32 unit; the
# library default for such tiles).
WRITE_PRESERVE = dict(map="lambda_unroll", rho=64, order="interleaved", store="merge")

# The same pass on a grid kept in pinned host memory, read and written in
# place over the host link (sg_map_write_mapped), with 32-byte
# read-merge-write stores (the library default there too); staged chunks and
# the write-only fill and sector stores are measured beside it.
WRITE_MAPPED = dict(map="lambda_unroll", rho=64, order="rowmajor", store="merge")

# Stencils at levels 14 and 15: 256 CA steps from Bernoulli(0.3) seeded with
# 0; 100 diffusion steps (alpha = 0.2) from U[0,1) seeded with 0.
STENCILS = dict(levels=(14, 15), ca_p=0.3, ca_seed=0, ca_steps=256,
                diff_seed=0, diff_steps=100, alpha=0.2,
                ca_rho=64, diff_rho=32, bbox_ca_rho=64, bbox_diff_rho=64,
                # the same sequences with k steps fused per launch
                ca_fuse=16, ca_fuse_rho=64, diff_fuse=8, diff_fuse_rho=32)

# The same write pass and stencil sequences on compact arrays (the 3^r
# gasket cells only, tiles in launch order): 43 MB instead of 4.3 GB for the
# level-16 uint8 grid.
COMPACT = dict(rho=64, order="interleaved")

# Batched: 64 gaskets with levels drawn uniformly from 8..14 (seed 2), each
# with its own uint8 CA state (Bernoulli(0.3), seed 2 + i * 2^32), 64 CA
# steps each: one launch per step over the prefix-summed work list (captured
# in a CUDA graph, autotuned) against 64 separate per-gasket launches.
BATCH = dict(count=64, level_lo=8, level_hi=14, level_seed=2, ca_p=0.3, ca_seed=2,
             steps=64, autotune_steps=4,
             fuse=16)                   # steps per launch of the fused batched form

