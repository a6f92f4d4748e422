"""The kernels' stopping test sqrt(rr) <= stop skips the square root when rr lies above
stop2_hi = fl(fl(stop * stop) * (1 + 1e-12)) (cg_device.cuh: stop2_high / below_stop).
IEEE-754 double multiplication and square root are correctly rounded on the host as on
the GPU, so the claim that this never changes the decision is checked here in numpy:
for stops over the whole exponent range and rr swept across the threshold ulp by ulp,
rr > stop2_hi must imply sqrt(rr) > stop."""
import numpy as np


def stop2_high(stop):
    s = stop * stop * (1.0 + 1e-12)
    return s if s >= 1e-300 else np.inf


def below_stop(rr, stop, s2):
    return rr <= s2 and np.sqrt(rr) <= stop


def test_prefilter_gives_the_exact_decision():
    rng = np.random.default_rng(5)
    stops = np.concatenate([10.0 ** rng.uniform(-150, 150, 400), [1e-8, 1.0, 3.0, 1e150, 1e-149]])
    for stop in stops:
        s2 = stop2_high(stop)
        if not np.isfinite(s2):
            continue
        # rr at, below and above the threshold, and around stop^2 itself
        for base in (s2, stop * stop):
            rr = base
            for _ in range(64):
                rr = np.nextafter(rr, -np.inf)
            for _ in range(128):
                assert below_stop(rr, stop, s2) == (np.sqrt(rr) <= stop), (stop, rr)
                rr = np.nextafter(rr, np.inf)
        # far above and far below
        for f in (1e-6, 0.5, 0.999999, 1.000001, 2.0, 1e6):
            rr = stop * stop * f
            assert below_stop(rr, stop, s2) == (np.sqrt(rr) <= stop)


def test_extreme_stops_take_the_exact_test():
    for stop in (1e-160, 0.0, np.nan, 1e160, np.inf):
        with np.errstate(over="ignore", invalid="ignore"):
            s2 = stop2_high(stop)
        assert s2 == np.inf or s2 >= 1e-300
