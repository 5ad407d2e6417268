"""The least-squares step of the coarse predictor u_* (Sec. 2.3.3) behind the C ABI.

mpwos_fit_torus_series runs on the host, so these tests need no GPU: the fit is
pinned by exact recovery of a series in its span (Example 1's u) and by numpy's
SVD least squares on noisy data.
"""
import math

import numpy as np
import pytest

from paper_2606_21883_b300 import workloads as W


def test_predictor_fit_recovers_a_series_in_its_span():
    """The least-squares step of the coarse predictor (mpwos_fit_torus_series, host
    only): fed exact values of Example 1's u (a series in the basis) it returns u's
    coefficients; fed noisy values, it agrees with numpy's least squares."""
    import paper_2606_21883_b300 as M
    w = W.torus_cut(P=2, walks=1)
    terms = W.torus_cut_terms()
    pts = W.torus_domain_points(w.problem, 300)
    th = np.arctan2(pts[:, 2], np.hypot(pts[:, 0], pts[:, 1]) - 1.0)
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    assert np.all(pts @ w.problem.bnd_normal > w.problem.bnd_offset)
    u_star = M.fit_torus_series(pts, W.torus_series_value(terms, th, ph), 1.0)
    assert len(u_star.coef) == 49
    rng = np.random.default_rng(0)
    th2, ph2 = rng.uniform(0, 2 * math.pi, 50), rng.uniform(0, 2 * math.pi, 50)
    got = W.torus_series_value([(c, *md) for c, md in zip(u_star.coef, u_star.modes)], th2, ph2)
    assert np.allclose(got, W.torus_series_value(terms, th2, ph2), atol=1e-9)
    # noisy data: the same minimiser as an SVD least-squares solve of the design matrix
    u = W.torus_series_value(terms, th, ph) + rng.normal(0.0, 0.05, len(th))
    fit = M.fit_torus_series(pts, u, 1.0, max_m=2, max_q=3)
    trig = (np.cos, np.sin)
    A = np.stack([trig[md[2]](md[0] * th) * trig[md[3]](md[1] * ph) for md in fit.modes], axis=1)
    ref, *_ = np.linalg.lstsq(A, u, rcond=None)
    assert len(fit.coef) == 5 * 7
    assert np.allclose(fit.coef, ref, atol=1e-10)
    with pytest.raises(M.MpwosError):
        M.fit_torus_series(pts[:40], u[:40], 1.0)     # 40 points, 49 unknowns
