"""Schedule autotuner host logic (no device): candidate order and selection."""
from paper_2606_05687_b300 import autotune as A


def test_candidates_start_at_the_defaults_and_cover_the_grid():
    c = A.candidates()
    n = 1
    for v in A.DEFAULT_GRID.values():
        n *= len(v)
    assert len(c) == n and len({tuple(sorted(x.items())) for x in c}) == n
    assert c[0] == A.LIBRARY_DEFAULTS
    # one-parameter neighbours come before two-parameter ones
    diffs = [sum(1 for k in A.LIBRARY_DEFAULTS if x[k] != A.LIBRARY_DEFAULTS[k]) for x in c]
    assert diffs == sorted(diffs)
    assert len(A.candidates(limit=5)) == 5


def test_select_best_takes_the_fastest_fully_certified_entry():
    t = [{"config": {"a": 1}, "ms": 3.0, "certified": 10, "instances": 10},
         {"config": {"a": 2}, "ms": 1.0, "certified": 9, "instances": 10},
         {"config": {"a": 3}, "ms": 2.0, "certified": 10, "instances": 10},
         {"config": {"a": 4}, "ms": 2.0, "certified": 10, "instances": 10}]
    assert A.select_best(t)["config"] == {"a": 3}
    # with no fully certified entry, the most certified one wins
    assert A.select_best([t[1], dict(t[0], certified=8)])["config"] == {"a": 2}
    assert A.select_best([]) is None


def test_library_defaults_match_the_c_defaults():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc
    cfg = pinmpc.default_config(13, 8, 3, 16, 20)
    for k, v in A.LIBRARY_DEFAULTS.items():
        assert abs(getattr(cfg, k) - v) < 1e-9, k
    assert A.library_defaults(13, 8, 3) == A.LIBRARY_DEFAULTS
    # each shape's defaults are a point of the default grid, and the search
    # for that shape starts there
    for shape in ((13, 8, 3), (13, 2, 6), (9, 8, 3), (9, 2, 6)):
        d = A.library_defaults(*shape)
        assert all(d[k] in A.DEFAULT_GRID[k] for k in d), (shape, d)
        assert A.candidates(limit=1, defaults=d)[0] == d
    assert A.library_defaults(13, 2, 6) == {"check_start": 32, "check_every": 20, "refine_alpha": 0.001,
                                            "rho": 300.0, "refine_steps": 4}
    assert A.library_defaults(9, 2, 6) == A.LIBRARY_DEFAULTS


def test_launch_shapes_join_the_grid():
    grid = {"rho": (100.0,), "horizon_classes": ((), (10,), (10, 20))}
    c = A.candidates(grid)
    assert [x["horizon_classes"] for x in c] == [(), (10,), (10, 20)]
    assert all(x["rho"] == 100.0 for x in c)


def test_library_defaults_skip_launch_shape_keys():
    import __graft_entry__
    __graft_entry__.build()
    d = A.library_defaults(13, 8, 3, ("rho", "horizon_classes"))
    assert d == {"rho": 100.0}


def test_ragged_class_sets_below_the_stride():
    from paper_2606_05687_b300 import pinmpc
    assert pinmpc.horizon_classes_for(10) == []
    assert pinmpc.horizon_classes_for(20) == [10]
    assert pinmpc.horizon_classes_for(30) == [10, 20]
    assert pinmpc.horizon_classes_for(40) == [10, 20, 32]
    assert pinmpc.horizon_classes_for(64) == [10, 20, 32]
