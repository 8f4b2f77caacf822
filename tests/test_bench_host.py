"""Host-side pieces of bench.py: the algorithmic-bytes formula (checked by
brute force over small grids), the clock-sample summary and the row-band cell
count of the reference arm."""
import os

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("r", [5, 7, 9, 10])
@pytest.mark.parametrize("elem,granule", [(1, 32), (1, 128), (4, 32), (4, 128)])
def test_touched_bytes_brute_force(orc, r, elem, granule):
    n = 1 << r
    per = granule // elem
    if per > n:
        pytest.skip("granule wider than the grid")
    mask = orc.member_grid(r).reshape(n, n // per, per)
    touched = int(mask.any(axis=2).sum())
    assert bench.touched_bytes(r, elem, granule) == touched * granule


def test_touched_bytes_level16_figures():
    # the per-launch algorithmic bytes quoted for the headline workload
    assert bench.touched_bytes(16, 1, 128) == 322_486_272
    assert bench.touched_bytes(16, 1, 32) == 181_398_528
    assert bench.touched_bytes(16, 4, 128) == 725_594_112
    assert bench.touched_bytes(16, 4, 32) == 408_146_688


def test_band_cells_match_member_counts(orc):
    r = 10
    g = orc.member_grid(r)
    for y0, y1 in ((0, 64), (100, 300), (512, 1024)):
        assert bench.band_cells(r, y0, y1) == int(g[y0:y1].sum())
    assert bench.band_cells(r, 0, 1 << r) == 3 ** r


def test_clock_summary():
    rows = [["0", "2070", "2070", "500.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["0", "1980", "2070", "610.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["0", "2070", "2070", "620.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = bench.summarize_clocks(rows)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.summarize_clocks([])["samples"] == 0


def test_all_cores_oracle_baseline_covers_the_grid():
    # the bands of the all-cores baseline tile the grid exactly once
    import bench
    out = bench.cpu_baseline_all_cores(dict(r=8, seed=1), band=32)
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    assert "8 bands of 32 rows" in out["sample"]


def test_unit_digest_follows_code_not_comments(tmp_path, monkeypatch):
    from paper_1706_04552_gb300 import build as b
    assert b.code_text('a; // c\n/* d */ "e//f" \'/\' b') == 'a; "e//f" \'/\' b'
    files = [os.path.basename(f) for f in b.unit_files("sg_write_u8.cu")]
    for want in ("sg_write_u8.cu", "sg_write.cuh", "sg_device.cuh", "sg_tma.cuh", "sg.h"):
        assert want in files
    # a copy of the sources: a comment edit keeps the digest, a code edit changes it
    import shutil
    csrc = tmp_path / "csrc"
    shutil.copytree(b.CSRC, csrc)
    monkeypatch.setattr(b, "CSRC", str(csrc))
    d0 = b.unit_digest("sg_write_u8.cu")
    p = csrc / "sg_device.cuh"
    p.write_text(p.read_text() + "\n// a note\n")
    assert b.unit_digest("sg_write_u8.cu") == d0
    p.write_text(p.read_text() + "\nconstexpr int kUnused = 1;\n")
    assert b.unit_digest("sg_write_u8.cu") != d0


def test_recorded_traffic_needs_the_current_digest():
    import bench
    # the committed record names a kernel; an unknown key or unit gives None
    assert bench.recorded_traffic("no_such_kernel", "sg_write_u8.cu") is None


def test_balanced_chunks_cover_the_sequence_evenly():
    assert bench.balanced_chunks(100, 8) == [8] * 9 + [7] * 4
    assert bench.balanced_chunks(256, 16) == [16] * 16
    for total in range(1, 300):
        for k in (1, 2, 3, 4, 8, 16):
            c = bench.balanced_chunks(total, k)
            assert sum(c) == total and max(c) <= k and len(c) == -(-total // k)
            assert max(c) - min(c) <= 1
