"""Pins of the warm-start reference (CPU): BF16 rounding against its
definition, and the analytic gradient against central finite differences."""
import numpy as np

from oracle import warmstart_ref as ws


def test_bf16_rounding_ties_to_even():
    one = np.float32(1.0)
    ulp = 2.0 ** -7  # bf16 spacing at 1
    vals = np.array([1.0, 1.0 + ulp / 2, 1.0 + 1.5 * ulp, 1.0 + 0.49 * ulp, -3.0, 0.0], dtype=np.float32)
    r = ws.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                  # tie -> even mantissa
    assert r[2] == 1.0 + 2 * ulp        # tie -> even mantissa (rounds up)
    assert r[3] == 1.0
    assert r[4] == -3.0 and r[5] == 0.0
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    assert np.max(np.abs(ws.bf16_round(x) - x) / np.abs(x)) <= 2.0 ** -8 + 1e-12
    assert one == 1.0


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(ws.NPARAMS) * 0.3
    F = rng.standard_normal((40, ws.IN))
    T = rng.standard_normal((40, 2))
    wt = rng.uniform(0.5, 1.5, 40)
    loss, g = ws.loss_and_grad(p, F, T, wt)
    idx = rng.choice(ws.NPARAMS, 60, replace=False)
    for q in idx:
        e = np.zeros(ws.NPARAMS)
        e[q] = 1e-6
        fd = (ws.loss_and_grad(p + e, F, T, wt)[0] - ws.loss_and_grad(p - e, F, T, wt)[0]) / 2e-6
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q])), (q, fd, g[q])
