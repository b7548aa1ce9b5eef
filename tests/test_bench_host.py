"""Host-side pieces of the benchmark: the fixed algorithmic operation count
behind its roofline."""
import bench


def test_opcount_matches_its_derivation():
    # DDF 5x5 exact: 40 pair terms x (25 angle + 7 L2) + 25*24 adds + 24 compares + 50 logs
    assert bench.opcount(5, "ddf", "exact") == 40 * 32 + 600 + 24 + 50 == 1954
    assert bench.opcount(3, "ddf", "exact") == 12 * 32 + 72 + 8 + 18
    assert bench.opcount(5, "bvdf", "exact") == 40 * 25 + 600 + 24
    assert bench.opcount(3, "bvdf", "rgb") == 12 * 9 + 72 + 8
    assert bench.opcount(5, "vmf", order=1) == 40 * 6 + 600 + 24
    assert bench.opcount(7, "ddf", "exact") == 84 * 32 + 49 * 48 + 48 + 98
    assert bench.opcount_acwddf(3) > bench.opcount(3, "ddf")


def test_opcount_is_independent_of_the_kernel_sources():
    """The count is a function of the configuration only: no kernel source is read."""
    import inspect
    src = inspect.getsource(bench.opcount)
    assert "open(" not in src and "csrc" not in src
