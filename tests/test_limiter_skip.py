"""The step limiter skips a distance's division when num >= 2 s den (2 s den normal): the
rounded quotient can then not be below the running minimum s, so the limiter's
comparison is false either way and the step is unchanged.  Checked here in IEEE FP32
(round to nearest, no FMA) on random and adversarial operands, brute force."""
import numpy as np

F = np.float32


def may_limit(num, den, s):
    bound = F(2.0) * s * den
    return ~((num >= bound) & (bound >= F(2.0 ** -100)))


def test_skipped_quotients_never_beat_the_minimum():
    rng = np.random.default_rng(7)
    n = 2_000_000
    # magnitudes over the whole normal range, plus values straddling the bound
    s = (10.0 ** rng.uniform(-30, 30, n)).astype(F)
    den = (10.0 ** rng.uniform(-30, 30, n)).astype(F)
    with np.errstate(over="ignore", under="ignore", invalid="ignore", divide="ignore"):
        bound = F(2.0) * s * den
        scale = F(1.0) + rng.uniform(-1e-6, 1e-6, n).astype(F)
        num = np.where(rng.random(n) < 0.5, bound * scale,
                       (10.0 ** rng.uniform(-30, 30, n)).astype(F))
        num = np.nextafter(num, np.where(rng.random(n) < 0.5, F(0), F(np.inf))).astype(F)
        skip = ~may_limit(num, den, s)
        q = num / den
    ok = np.isfinite(s) & np.isfinite(den) & (den > 0) & np.isfinite(num)
    assert skip[ok].sum() > n // 10  # the skip is exercised
    assert np.all(q[skip & ok] >= s[skip & ok])


def test_edge_cases_compute_the_division():
    inf = F(np.inf)
    # s = +inf (no plane ahead), s = 0 (on a plane), tiny products: never skipped
    assert may_limit(F(1.0), F(0.5), inf)
    assert may_limit(F(1.0), F(0.5), F(0.0))
    assert may_limit(F(1e-30), F(1e-20), F(1e-20))
    # far from the wall: skipped, and the quotient is indeed >= s
    assert not may_limit(F(200.0), F(0.001), F(2.3))
