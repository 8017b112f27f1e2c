"""Host logic of the autotuner (no GPU): the fastest candidate wins, ties go
to the earlier one."""
from paper_2503_16028_gb300 import batch


def test_pick_fastest():
    a, b, c = dict(), dict(smooth_sweeps=1), dict(tol_inner=1e-3)
    assert batch.pick_fastest([(a, 3.0), (b, 2.0), (c, 2.5)]) is b
    assert batch.pick_fastest([(a, 2.0), (b, 2.0)]) is a
