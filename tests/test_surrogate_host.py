"""Host-side logic of the learned surrogates (no GPU): evaluation and the
calibration of the fallback margin."""
import numpy as np

from paper_2602_10114_gb300.surrogate import calibrate_margin, evaluate


def test_margin_calibration_meets_its_target():
    """The calibrated fallback margin is the smallest one at which at most the
    target fraction of colliding samples would be skipped."""
    rng = np.random.default_rng(3)
    exact = rng.uniform(-0.1, 0.4, 20000)
    pred = exact + rng.normal(0, 0.03, exact.size)
    for target in (1e-3, 1e-2):
        m = calibrate_margin(pred, exact, 0.03, target)
        assert evaluate(pred, exact, 0.03, m)["fn_rate"] <= target
        # any smaller margin skips more colliding samples than allowed
        m2 = float(np.nextafter(np.float32(0.03 + m), np.float32(-1)) - 0.03) - 1e-6
        if m2 > 0:
            assert evaluate(pred, exact, 0.03, m2)["fn_rate"] > target


def test_evaluate_counts_false_negatives_over_colliding_samples():
    exact = np.array([-0.02, -0.01, 0.0, 0.02, 0.2, 0.5])
    pred = np.array([0.07, 0.01, 0.2, 0.1, 0.3, -0.1])
    ev = evaluate(pred, exact, 0.03, 0.03)          # skip when pred >= 0.06
    assert ev["colliding"] == 2 and ev["false_negatives"] == 1 and ev["fn_rate"] == 0.5
    # cost-active samples (exact < B): the two colliding, 0.0 and 0.02; skipped: 0.07, 0.2, 0.1
    assert ev["fn_rate_active"] == 3 / 4
    assert ev["skip_fraction"] == 4 / 6
