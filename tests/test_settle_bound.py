"""The fill's exact early exit (no GPU needed).

The CUDA fill stops a hole pixel's candidate walk once an interval bound proves that the
remaining candidates cannot change its rounded color (Alg. 3, Eq. 6 with the exit stated
in the kernel source).  This test restates that bound with exact rational arithmetic
(upward rounding to binary32 done by hand, the reciprocal taken exactly) and checks, on
random and adversarial candidate sequences run in binary32 step by step, that whenever
the bound declares a pixel settled its color equals the color of the full walk.  It
checks the argument, not the CUDA code; the GPU parity tests check the code.
"""
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def _ru(x: Fr) -> f32:
    """Smallest binary32 value >= x."""
    f = f32(float(x))
    if Fr(float(f)) < x:
        f = np.nextafter(f, f32(np.inf), dtype=f32)
    return f


def _add(acc, wrem, t, col):
    """One Eq. 6 step in binary32, each operation rounded to nearest."""
    a = f32(wrem * f32(0.5))
    b = f32(f32(f32(0.3) * wrem) * t)
    wgt = f32(a + b)
    if wgt == 0:
        return acc, wrem, False
    acc = (acc + (col * wgt).astype(f32)).astype(f32)
    return acc, f32(wrem - wgt), True


def _result(acc, wrem):
    den = f32(f32(1) - wrem)
    q = [Fr(float(a)) / Fr(float(den)) for a in acc]
    # rint of the correctly rounded quotient, ties to even, clamped
    return [int(min(255, max(0, np.rint(f32(float(x)))))) for x in q]


def _settled(acc, wrem):
    """The kernel's bound with the exact reciprocal (tighter than the kernel's)."""
    den = f32(f32(1) - wrem)
    inv = _ru(Fr(1) / Fr(float(den)))
    e1 = _ru(Fr(float(f32(255.0000152587890625))) * Fr(float(wrem)))
    e = _ru(Fr(float(_ru(Fr(float(e1)) + Fr(float(min(e1, f32(0.00115))))))) + Fr(float(f32(1.0e-42))))
    out = []
    for a in acc:
        r = np.rint(a)
        if r < 255:
            hi = _ru(Fr(float(_ru(Fr(float(a)) + Fr(float(e))))) * Fr(float(inv)))
            if not hi < f32(r + f32(0.5)):
                return None
        out.append(int(min(r, 255)))
    return out


def _walk(cols, t):
    acc, wrem = np.zeros(4, f32), f32(1)
    early = None
    for c in cols:
        acc, wrem, ok = _add(acc, wrem, t, c)
        if not ok:
            break
        if early is None and wrem <= f32(2.0 ** -9):
            early = _settled(acc, wrem)
    return early, _result(acc, wrem)


def _check(cols, t):
    early, full = _walk(cols, t)
    if early is not None:
        assert early == full, (early, full, t)
    return early is not None


def test_bound_agrees_with_the_full_walk_on_random_sequences():
    rng = np.random.default_rng(2506)
    settled = 0
    for _ in range(400):
        n = int(rng.integers(8, 60))
        cols = rng.integers(0, 256, (n, 4)).astype(f32)
        settled += _check(cols, f32(rng.uniform(0, 1)))
    assert settled > 300  # the exit is taken on most walks


def test_bound_agrees_on_smooth_backgrounds_and_half_integer_limits():
    """Slowly varying colors (a background gradient) drive the sums toward the same
    value from below; on one GPU pixel this ended exactly at 165.5 (rounded to 166),
    which an exit taken one step early would have rounded to 165."""
    rng = np.random.default_rng(7)
    for k in range(300):
        base = rng.integers(1, 250, 4)
        n = 60
        drift = rng.integers(-1, 2, (n, 4)).cumsum(axis=0) // 3
        cols = np.clip(base + drift, 0, 255).astype(f32)
        _check(cols, f32((k % 53 + 1) / 54.0))
    # two colors a level apart in a ratio that puts the weighted mean near x.5
    for lo in (0, 17, 128, 165, 254):
        for t in (f32(9 / 53), f32(0.5), f32(0.25), f32(0.999)):
            cols = np.array([[lo + (i % 2)] * 4 for i in range(80)], dtype=f32)
            _check(cols, t)


def test_bound_agrees_when_the_remaining_candidates_are_extreme():
    """After a random prefix every later candidate is 255 (the most the remaining weight
    can add) or 0 (the least): the bound's slack must cover the first and the sum's
    lower end the second."""
    rng = np.random.default_rng(11)
    for k in range(600):
        pre = rng.integers(0, 256, (int(rng.integers(1, 14)), 4))
        tail = np.full((60, 4), 255 if k % 2 == 0 else 0)
        _check(np.vstack([pre, tail]).astype(f32), f32(rng.uniform(0, 1)))


def test_the_exit_never_fires_before_the_threshold():
    """Above wrem = 2^-9 the bound is not consulted; the walk runs on."""
    cols = np.full((4, 4), 200, dtype=f32)
    early, full = _walk(cols, f32(0.5))
    assert early is None and full == [200, 200, 200, 200]
