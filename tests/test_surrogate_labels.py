"""Host logic of the surrogate's label job: checkpoint, resume, and extension of a
shorter run of the same Sobol sequence (a counting stand-in replaces the estimator)."""
import numpy as np

from paper_2405_03474_gb300 import inputs, surrogate


class _Counting:
    def __init__(self):
        self.calls = 0

    def __call__(self, theta):
        self.calls += 1
        return float(np.log(theta).sum())


def test_labels_resume_and_extend(tmp_path):
    ck = str(tmp_path / "labels.npz")
    short = inputs.sobol_theta(12, seed=0)
    est = _Counting()
    lab12 = surrogate.generate_labels(est, short, checkpoint=ck, every=4)
    assert est.calls == 12
    np.testing.assert_allclose(lab12, np.log(short).sum(axis=1))
    # the same job again: nothing left to do
    est = _Counting()
    np.testing.assert_array_equal(surrogate.generate_labels(est, short, checkpoint=ck, every=4), lab12)
    assert est.calls == 0
    # a longer run of the same sequence reuses the first 12 labels
    longer = inputs.sobol_theta(20, seed=0)
    np.testing.assert_array_equal(longer[:12], short)
    est = _Counting()
    lab20 = surrogate.generate_labels(est, longer, checkpoint=ck, every=4)
    assert est.calls == 8
    np.testing.assert_allclose(lab20, np.log(longer).sum(axis=1))
    # a different sequence starts afresh
    est = _Counting()
    surrogate.generate_labels(est, inputs.sobol_theta(6, seed=3), checkpoint=ck, every=4)
    assert est.calls == 6


class _NotSpdCorner(_Counting):
    """NaN where the stand-in 'operator' is not positive definite (long lengthscale and
    low noise), as the estimator answers LD_ERR_NOT_SPD there."""

    def __call__(self, theta):
        self.calls += 1
        return float("nan") if theta[0] > 0.5 and theta[2] < 1e-3 else float(np.log(theta).sum())


def test_labels_keep_not_spd_settings_as_nan_across_resume(tmp_path):
    ck = str(tmp_path / "labels.npz")
    th = inputs.sobol_theta(64, seed=0)
    corner = (th[:, 0] > 0.5) & (th[:, 2] < 1e-3)
    assert corner.any() and not corner.all()
    lab = surrogate.generate_labels(_NotSpdCorner(), th[:40], checkpoint=ck, every=8)
    est = _NotSpdCorner()
    lab = surrogate.generate_labels(est, th, checkpoint=ck, every=8)
    assert est.calls == 24
    assert np.array_equal(np.isnan(lab), corner)
    np.testing.assert_allclose(lab[~corner], np.log(th[~corner]).sum(axis=1))
