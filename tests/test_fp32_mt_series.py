"""The FP32 reduced walk's chi^2 draw (Marsaglia-Tsang, ACM TOMS 26 (2000)) writes
the log acceptance test d - d v + d log v, v = (1 + t)^3, t = c x, as
d (3 log1p(t) - 3t - 3t^2 - t^3) to avoid the cancellation of d - d v in single
precision, and evaluates that bracket for |t| < 1/4 by its Taylor series
-9/2 t^2 - 3/4 t^4 + 3/5 t^5 - 1/2 t^6 + 3/7 t^7 - 3/8 t^8 + 1/3 t^9 - 3/10 t^10.
Pinned here against high-precision arithmetic (the identity and the series'
relative error < 3e-7) and by the law of the draws it accepts (scipy's chi^2)."""
import math

import mpmath as mp
import numpy as np
from scipy import stats


def bracket_series(t):
    """The series as the kernel evaluates it (Horner in t, times t^2)."""
    return t * t * (-4.5 + t * t * (-0.75 + t * (0.6 + t * (-0.5 + t * (3.0 / 7.0 + t * (-0.375 + t * (1.0 / 3.0
                                                                                                    + t * -0.3)))))))


def bracket_exact(t):
    t = mp.mpf(t)
    return 3 * mp.log1p(t) - 3 * t - 3 * t ** 2 - t ** 3


def test_bracket_identity():
    mp.mp.dps = 40
    for d in (0.5, 3.1, 497.6666666666667):
        for t in (-0.9, -0.3, -1e-3, 2e-4, 0.2, 1.7):
            v = (1 + mp.mpf(t)) ** 3
            lhs = d * bracket_exact(t)
            rhs = d - d * v + d * mp.log(v)
            assert abs(lhs - rhs) <= mp.mpf(10) ** -30 * (1 + abs(rhs))


def test_series_relative_error_below_3e7():
    mp.mp.dps = 40
    worst = 0.0
    for t in np.concatenate([np.linspace(-0.2499, 0.2499, 2001), [1e-6, -1e-6, 1e-3]]):
        if t == 0.0:
            continue
        ex = bracket_exact(float(t))
        worst = max(worst, float(abs((mp.mpf(bracket_series(float(t))) - ex) / ex)))
    assert worst < 3e-7
    # the first dropped term (3/11 t^11) is what bounds it at |t| = 1/4
    assert worst > 1e-8


def test_accepted_draws_follow_chi2():
    """2 d v over the accepted attempts is chi^2 with m degrees of freedom."""
    rng = np.random.default_rng(20)
    for m in (2, 7, 996):
        d = 0.5 * m - 1.0 / 3.0
        c = 1.0 / math.sqrt(9.0 * d)
        out = []
        while len(out) < 20000:
            x = rng.standard_normal()
            t = c * x
            if t <= -1.0:
                continue
            term = bracket_series(t) if abs(t) < 0.25 else 3.0 * math.log1p(t) - t * (3.0 + t * (3.0 + t))
            if math.log(1.0 - rng.random()) < 0.5 * x * x + d * term:
                out.append(2.0 * d * (1.0 + t) ** 3)
        assert stats.kstest(out, stats.chi2(m).cdf).pvalue > 1e-3
