"""The steady-state detector (host logic, CPU): window means of the
particle count, peak density and outer-wall current, steady when two
consecutive windows agree within 2%."""
import numpy as np

from paper_2206_14662_gb300.steady import SteadyDetector, window_steps


def _run(f, W=100, every=10, n=4000):
    d = SteadyDetector(W)
    for step in range(every, n + 1, every):
        v = f(step)
        if d.add(step, n=v, n_max=2 * v, i_outer=3 * v):
            return d.steady_step
    return None


def test_constant_is_steady_after_two_windows():
    assert _run(lambda s: 5.0) == 200


def test_drift_below_and_above_the_tolerance():
    # growth by 1% per window: steady at the first check; by 5% per window:
    # never
    assert _run(lambda s: 100.0 * 1.01 ** (s / 100)) == 200
    assert _run(lambda s: 100.0 * 1.05 ** (s / 100)) is None


def test_relaxation_becomes_steady_when_the_drift_has_decayed():
    # exponential approach: window means differ by less than 2% only once
    # the remaining drift is small
    tau = 400.0
    s = _run(lambda t: 1.0 + 9.0 * np.exp(-t / tau), n=10000)
    assert s is not None
    m = lambda a, b: np.mean([1 + 9 * np.exp(-t / tau) for t in range(a + 10, b + 1, 10)])
    assert abs(m(s - 100, s) - m(s - 200, s - 100)) <= 0.02 * m(s - 200, s - 100)
    assert abs(m(s - 200, s - 100) - m(s - 300, s - 200)) > 0.02 * m(s - 300, s - 200)


def test_breathing_is_steady_in_the_mean():
    # oscillation with a period much shorter than the window
    assert _run(lambda s: 10.0 + 3.0 * np.sin(2 * np.pi * s / 20.0)) == 200


def test_window_length():
    assert window_steps({"dt": 1e-12}, 1e8) == 50000
    assert window_steps({"dt": 1e-12}, 1e11) == 2000
