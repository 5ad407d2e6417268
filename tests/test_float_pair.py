"""The FP32 walks carry each walk's weight W and score S in float pairs (hi + lo,
error-free transformations on FP32 operations) instead of FP64.  This restates
those operations with correctly rounded float32 arithmetic and pins their
precision against 50-digit arithmetic: about 2^-46 relative per operation, and
a relative error of order K 2^-46 on S after K steps (K = 525 on the torus:
~1e-11, far below the walks' Monte Carlo noise), for both accumulation forms
(the general one, S += (W omega) F and W *= c, and the constant-radius loop's
V = W omega with S.lo accumulated unnormalised and renormalised every 64 steps)."""
import mpmath as mp
import numpy as np

f32 = np.float32


def fma(a, b, c):
    # a*b is exact in float64 (two 24-bit significands); one rounding of the sum to
    # float64 and one to float32 (the double rounding is far below the bounds tested)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def f2_from_double(x):
    hi = f32(x)
    return hi, f32(x - np.float64(hi))


def f2_mul(x, y):
    p = f32(x[0] * y[0])
    e = fma(x[0], y[0], -p)
    e = fma(x[0], y[1], e)
    e = fma(x[1], y[0], e)
    return fast_two_sum(p, e)


def f2_mul_f(x, f):
    p = f32(x[0] * f)
    e = fma(x[0], f, -p)
    e = fma(x[1], f, e)
    return fast_two_sum(p, e)


def f2_add(x, y):
    s = f32(x[0] + y[0])
    bb = f32(s - x[0])
    err = f32(f32(x[0] - f32(s - bb)) + f32(y[0] - bb))
    return fast_two_sum(s, f32(err + f32(x[1] + y[1])))


def value(x):
    return mp.mpf(float(x[0])) + mp.mpf(float(x[1]))


def test_single_operations_near_2_pow_46():
    mp.mp.dps = 50
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(2000):
        a = f2_from_double(rng.uniform(0.1, 10.0))
        b = f2_from_double(rng.uniform(0.1, 10.0))
        f = f32(rng.uniform(-1.0, 1.0))
        for got, exact in ((f2_mul(a, b), value(a) * value(b)), (f2_add(a, b), value(a) + value(b)),
                           (f2_mul_f(a, f), value(a) * mp.mpf(float(f)))):
            worst = max(worst, float(abs(value(got) - exact) / abs(exact)))
    assert worst < 2.0 ** -44
    assert worst > 2.0 ** -60      # a float pair, not an exact sum: the bound is attained in scale


def _walk(K, c, omega, F):
    """Exact sum over k of omega c^k F_k, and the sum of its absolute terms."""
    s, a, w = mp.mpf(0), mp.mpf(0), mp.mpf(omega)
    for k in range(K):
        t = w * mp.mpf(float(F[k]))
        s += t
        a += abs(t)
        w *= mp.mpf(c)
    return s, a


def test_general_accumulation_after_525_steps():
    mp.mp.dps = 50
    rng = np.random.default_rng(6)
    for c_d in (0.97, 0.9990234375, 0.5):
        K = 525
        F = rng.uniform(-1.0, 1.0, K).astype(np.float32)
        c, om = f2_from_double(c_d), f2_from_double((1.0 - c_d) / 2.0)
        W, S = (f32(1.0), f32(0.0)), (f32(0.0), f32(0.0))
        for k in range(K):
            S = f2_add(S, f2_mul_f(f2_mul(W, om), F[k]))
            W = f2_mul(W, c)
        exact, scale = _walk(K, value(c), value(om), F)
        assert float(abs(value(S) - exact) / scale) < K * 2.0 ** -44


def test_constant_radius_accumulation_after_525_steps():
    mp.mp.dps = 50
    rng = np.random.default_rng(7)
    c_d = 0.97
    K = 525
    F = rng.uniform(-1.0, 1.0, K).astype(np.float32)
    c, om = f2_from_double(c_d), f2_from_double((1.0 - c_d) / 2.0)
    V, S = om, (f32(0.0), f32(0.0))
    for k0 in range(0, K, 64):
        for k in range(k0, min(k0 + 64, K)):
            ph = f32(V[0] * F[k])
            pl = fma(V[1], F[k], fma(V[0], F[k], -ph))
            sh = f32(S[0] + ph)
            bb = f32(sh - S[0])
            err = f32(f32(S[0] - f32(sh - bb)) + f32(ph - bb))
            S = (sh, f32(S[1] + f32(err + pl)))
            vh = f32(V[0] * c[0])
            V = (vh, fma(V[1], c[0], fma(V[0], c[1], fma(V[0], c[0], -vh))))
        S = fast_two_sum(S[0], S[1])
    exact, scale = _walk(K, value(c), value(om), F)
    rel = float(abs(value(S) - exact) / scale)
    assert rel < K * 2.0 ** -44
    assert rel < 1e-10                                   # the ~1e-11 the precision statement quotes
    assert rel < 1e-13                                   # in fact ~5e-15: the terms' errors do not add up linearly
    # FP32 alone would be ~1e-7 here: the pair is what carries the weight
    s32, w32 = f32(0.0), f32(value(om))
    for k in range(K):
        s32 = f32(s32 + f32(w32 * F[k]))
        w32 = f32(w32 * f32(c_d))
    assert float(abs(mp.mpf(float(s32)) - exact) / scale) > 100 * rel
