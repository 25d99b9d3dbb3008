"""Host logic of the d-sweep: averaging the per-seed rows (no GPU)."""
import pytest

from paper_2405_03474_gb300 import experiments


def test_summarise_averages_each_kernel_and_dimension_over_seeds():
    rows = []
    for seed, scale in ((0, 1.0), (1, 3.0)):
        for kernel, d in (("rbf", 2), ("matern52", 2), ("rbf", 5)):
            rows.append({"kernel": kernel, "d": d, "seed": seed, "err_r1": 4.0 * scale, "err_r3": 2.0 * scale,
                         "err_r5": 1.0 * scale, "err_slq": 3.0 * scale})
    out = {(a["kernel"], a["d"]): a for a in experiments.summarise(rows)}
    assert set(out) == {("rbf", 2), ("matern52", 2), ("rbf", 5)}
    for acc in out.values():
        assert acc["count"] == 2
        assert acc["err_r1"] == pytest.approx(8.0) and acc["err_r3"] == pytest.approx(4.0)
        assert acc["err_r5"] == pytest.approx(2.0) and acc["err_slq"] == pytest.approx(6.0)
