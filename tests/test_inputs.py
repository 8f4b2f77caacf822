"""The seeded input generators: deterministic, zero off the gasket, the
stated distributions, and region draws consistent with full-grid draws."""
import numpy as np

from paper_1706_04552_gb300 import inputs


def test_gasket_cells_row_major_and_complete():
    for r in (0, 1, 4, 9):
        xs, ys = inputs.gasket_cells(r)
        assert len(xs) == 3 ** r
        assert np.all((xs & ys) == 0)
        key = (ys << r) | xs
        assert np.all(np.diff(key) > 0)


def test_seed_is_zero_off_gasket_and_deterministic():
    r = 8
    a = inputs.ca_seed_grid(r, 0.3, 0)
    b = inputs.ca_seed_grid(r, 0.3, 0)
    assert np.array_equal(a, b)
    ys, xs = np.nonzero(a)
    assert np.all((xs & ys) == 0)
    assert set(np.unique(a)) <= {0, 1}
    c = inputs.ca_seed_grid(r, 0.3, 1)
    assert not np.array_equal(a, c)


def test_bernoulli_density_and_uniform_range():
    r = 12
    idx, st = inputs.ca_seed_sparse(r, 0.3, 0)
    assert len(idx) == 3 ** r
    assert abs(st.mean() - 0.3) < 0.01
    idx2, u = inputs.uniform_sparse(r, 0)
    assert np.array_equal(idx, idx2)
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    assert abs(float(u.mean()) - 0.5) < 0.01
    # 24-bit values: exact multiples of 2^-24
    assert np.all((u.astype(np.float64) * 2**24) % 1 == 0)


def test_region_draws_match_full_grid():
    r = 7
    full_s = inputs.ca_seed_grid(r, 0.5, 3)
    full_u = inputs.uniform_grid(r, 3)
    win_s = inputs.ca_seed_region(r, 0.5, 3, -5, 10, 40, 30)
    win_u = inputs.uniform_region(r, 3, 100, -3, 40, 30)
    assert np.array_equal(win_s[:, 5:], full_s[10:40, 0:35])
    assert not win_s[:, :5].any()
    assert np.array_equal(win_u[3:, :28], full_u[0:27, 100:128])
    assert not win_u[:, 28:].any() and not win_u[:3].any()


def test_hash_matches_published_first_output():
    # the cell with key 0 and seed 0 is SplitMix64 state 0
    h = inputs.cell_hash(10, np.array([0]), np.array([0]), 0)
    assert int(h[0]) == 0xE220A8397B1DCDAF
