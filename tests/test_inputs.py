"""Host-side input recipe and region helpers (no GPU): the synthetic workloads of Sec. VII."""
import numpy as np

from paper_1804_09137_gb300 import inputs


def test_jittered_grid_cells_and_determinism():
    """Point (r, l) lies within 0.4 / side of its cell centre ((r - 0.5) / side, (l - 0.5) / side)."""
    side = 17
    x, y = inputs.jittered_grid(side)
    assert x.shape == (side * side,) and y.shape == (side * side,)
    r, l = np.meshgrid(np.arange(1, side + 1), np.arange(1, side + 1), indexing="ij")
    cx, cy = ((r - 0.5) / side).ravel(), ((l - 0.5) / side).ravel()
    assert np.all(np.abs(x - cx) <= 0.4 / side + 1e-15) and np.all(np.abs(y - cy) <= 0.4 / side + 1e-15)
    assert np.all((x > 0) & (x < 1) & (y > 0) & (y < 1))
    x2, y2 = inputs.jittered_grid(side)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
    x3, _ = inputs.jittered_grid(side, seed=inputs.SEED + 1)
    assert not np.array_equal(x, x3)


def test_non_square_sizes_take_a_subset_of_the_grid():
    x, y = inputs.locations(1000)
    assert len(x) == 1000
    xs, ys = inputs.jittered_grid(32)  # ceil(sqrt(1000)) = 32
    grid = set(zip(xs.tolist(), ys.tolist()))
    assert all(p in grid for p in zip(x.tolist(), y.tolist()))
    assert len(set(zip(x.tolist(), y.tolist()))) == 1000


def test_holdout_partitions_the_points():
    obs, held = inputs.holdout(500, 37)
    assert len(held) == 37 and len(obs) == 463
    assert np.array_equal(np.sort(np.concatenate([obs, held])), np.arange(500))
    o2, h2 = inputs.holdout(500, 37)
    assert np.array_equal(held, h2) and np.array_equal(obs, o2)


def test_region_draws_ranges():
    n, th = inputs.region_draws(512)
    assert n.shape == (512,) and th.shape == (512, 3)
    assert n.min() >= 500 and n.max() <= 8000
    assert np.all((th[:, 0] >= 0.5) & (th[:, 0] <= 2.0))
    assert np.all((th[:, 1] >= 0.03) & (th[:, 1] <= 0.3))
    assert set(np.unique(th[:, 2]).tolist()) <= {0.5, 1.0, 1.5}


def test_standard_normal_streams_are_independent():
    e1 = inputs.standard_normal(1000)
    e2 = inputs.standard_normal(1000, stream=inputs.STREAM_NOISE + 10)
    assert abs(np.mean(e1)) < 0.15 and abs(np.std(e1) - 1.0) < 0.1
    assert abs(np.corrcoef(e1, e2)[0, 1]) < 0.15


def test_region_size_classes_and_options():
    from paper_1804_09137_gb300 import regions

    assert [regions.size_class(n) for n in (500, 1999, 2000, 3999, 4000, 8000)] == [0, 0, 1, 1, 2, 2]
    choice = {0: (0, 0, 0.0, {}), 1: (768, 192, 0.0, {}), 2: (384, 0, 0.0, {})}
    o = regions.make_opts(1500, choice, 1e-8)  # one tile covering the region
    assert o.nb == 1500 and o.eps == 1e-8 and o.metric == 0
    o = regions.make_opts(3000, choice, 1e-8)  # the autotuned rank cap
    assert o.nb == 768 and o.rank_cap == 192
    o = regions.make_opts(5000, choice, 1e-8)  # no cap chosen: half the tile
    assert o.nb == 384 and o.rank_cap == 192
    o = regions.make_opts(700, {0: (1024, 0, 0.0, {})}, 1e-8)  # a tile larger than the region: single tile
    assert o.nb == 700
    sizes, thetas, pts = regions.region_problems(R=6)
    assert len(pts) == 6 and all(len(p[0]) == int(n) for p, n in zip(pts, sizes))
