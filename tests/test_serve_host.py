"""Host-side pieces of the server: the seeded level mix and request trace."""
import numpy as np

from paper_1706_04552_gb300.serve import (ServeConfig, gasket_levels, launch_groups,
                                          make_trace, steps_this_iteration)


def test_levels_are_geometric_toward_small_levels():
    cfg = ServeConfig(gaskets=20000)
    lv = gasket_levels(cfg)
    assert lv.min() >= 6 and lv.max() <= 15
    counts = np.bincount(lv - 6, minlength=10)
    # P(6 + k) proportional to 0.5^k: each level about half as common as the one below
    for k in range(4):
        assert 0.4 < counts[k + 1] / counts[k] < 0.6
    assert np.array_equal(gasket_levels(cfg), lv)           # seeded


def test_trace_is_poisson_and_seeded():
    cfg = ServeConfig(rate=2000.0, duration=5.0)
    t, g, k = make_trace(cfg)
    assert abs(len(t) - 10000) < 4 * 100                     # mean 10000, sd 100
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] <= 5.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000) < 0.05 / 2000         # exponential gaps
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05
    assert g.min() >= 0 and g.max() < cfg.gaskets
    assert k.min() >= 1 and k.max() <= 32
    t2, g2, k2 = make_trace(cfg)
    assert np.array_equal(t, t2) and np.array_equal(g, g2) and np.array_equal(k, k2)


def test_fused_launch_groups_never_cross_a_request():
    assert launch_groups(1) == [1]
    assert launch_groups(16) == [1, 2, 4, 8, 16]
    assert launch_groups(12) == [1, 2, 4, 8]
    for fuse in (1, 2, 5, 8, 16):
        groups = launch_groups(fuse)
        for steps in range(1, 40):
            # a request of `steps` steps is served in iterations that each
            # take a group size <= the steps still left; they add up exactly
            left, seen = steps, []
            while left:
                k = steps_this_iteration(left, groups)
                assert 1 <= k <= min(left, fuse) and k in groups
                seen.append(k)
                left -= k
            assert sum(seen) == steps
            assert len(seen) <= steps // fuse + 5


def test_default_config_fits_whole_tiles_and_the_budget():
    # every gasket of the default mix holds whole rho-tiles (level >= log2 rho,
    # as the batch calls require), and the preloaded states fit the budget
    cfg = ServeConfig()
    assert cfg.rho in (16, 32, 64) and cfg.level_min >= cfg.rho.bit_length() - 1
    assert cfg.engine == "native" and cfg.pipeline >= 1 and 1 <= cfg.fuse <= 16
    lv = gasket_levels(cfg)
    assert int(np.sum(2 * 4 ** lv.astype(np.int64))) <= cfg.budget_bytes
