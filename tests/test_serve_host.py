"""Host-side logic of the serving loop, no GPU: Poisson arrival times."""
import numpy as np

from paper_2206_06079_gb300 import serve


def test_poisson_times_rate_and_order():
    rng = np.random.default_rng(0)
    t = serve.poisson_times(30.0, 200.0, rng)
    assert np.all(np.diff(t) > 0) and t[-1] < 200.0
    assert abs(len(t) / 200.0 - 30.0) < 1.5
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 30.0) < 0.003 and abs(gaps.std() - 1 / 30.0) < 0.004  # exponential gaps
