"""Pins for the oracle's Gaussian sketch entries (Sec. 3.1: Omega_k iid N(0,1)).

The counter-based stream must (a) evaluate ln and cos correctly (checked against numpy's
library routines and exact special values), (b) produce standard-normal entries (moments and
a Kolmogorov-Smirnov test against the normal CDF), (c) give independent entries across the
(k, i, j) counter coordinates, and (d) make any column prefix independent of how columns are
drawn (the property Algorithm 5 relies on when it appends columns).
"""
import math

import numpy as np
import pytest

from oracle import philox as P

EPS = np.finfo(np.float64).eps


def test_own_log_matches_library_within_4ulp():
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.random(400_000), 2.0 ** -rng.uniform(0, 53, 200_000),
                        1.0 - rng.random(100_000) * 1e-6, [2.0 ** -53, 0.5, 0.25, 1.0]])
    u = u[(u > 0) & (u <= 1)]
    got, ref = P.own_log(u), np.log(u)
    ulp = np.spacing(np.abs(ref))
    ulp[ref == 0] = EPS
    assert np.max(np.abs(got - ref) / ulp) <= 4.0


def test_own_log_special_values():
    assert P.own_log(np.array([1.0]))[0] == 0.0
    assert abs(P.own_log(np.array([0.5]))[0] + math.log(2.0)) <= 2 * EPS
    assert abs(P.own_log(np.array([2.0 ** -53]))[0] + 53 * math.log(2.0)) <= 4 * 53 * EPS


def test_own_cos2pi_matches_library():
    rng = np.random.default_rng(1)
    t = np.concatenate([rng.random(500_000), np.arange(0, 1, 1 / 64)])
    got, ref = P.own_cos2pi(t), np.cos(2 * np.pi * t)
    # np.cos(2*pi*t) itself carries the rounding of 2*pi*t (|error| <= 2*pi*2^-53)
    assert np.max(np.abs(got - ref)) <= 4e-16 + 2 * np.pi * EPS


def test_own_cos2pi_exact_points():
    v = P.own_cos2pi(np.array([0.0, 0.25, 0.5, 0.75, 0.125]))
    assert v[0] == 1.0 and v[1] == 0.0 and v[2] == -1.0 and v[3] == 0.0
    assert abs(v[4] - math.sqrt(0.5)) <= 2 * EPS


def test_uniforms_ranges():
    big = np.uint64(0xFFFFFFFF)
    z = np.uint64(0)
    u1, u2 = P.uniforms_from_words(np.array([z, big]), np.array([z, big]), np.array([z, big]), np.array([z, big]))
    assert u1[0] == 2.0 ** -53 and u1[1] == 1.0            # u1 in (0, 1]
    assert u2[0] == 0.0 and u2[1] == 1.0 - 2.0 ** -53      # u2 in [0, 1)


def test_gaussian_moments_and_ks():
    from scipy import stats
    n = 1_000_000
    j = np.arange(n, dtype=np.uint64)
    g = P.gaussian_f64(20251103, 3, j % 97, j // 97)
    se = 1.0 / math.sqrt(n)
    assert abs(g.mean()) < 5 * se
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0) * se
    kurt = np.mean((g - g.mean()) ** 4) / g.var() ** 2
    assert abs(kurt - 3.0) < 5 * math.sqrt(24.0) * se
    assert stats.kstest(g, "norm").pvalue > 1e-4
    # tails: P(|g| > 3) = 0.0027
    assert abs(np.mean(np.abs(g) > 3.0) - 0.0026998) < 6 * math.sqrt(0.0027 / n)


def test_counter_coordinates_are_independent():
    a = P.gaussian_f64(5, 2, np.arange(2000)[:, None], np.arange(200)[None, :])
    b = P.gaussian_f64(5, 3, np.arange(2000)[:, None], np.arange(200)[None, :])   # other core
    c = P.gaussian_f64(6, 2, np.arange(2000)[:, None], np.arange(200)[None, :])   # other seed
    lim = 5.0 / math.sqrt(a.size)
    for x, y in [(a, b), (a, c), (a[:, :-1], a[:, 1:]), (a[:-1], a[1:])]:
        assert abs(np.corrcoef(x.ravel(), y.ravel())[0, 1]) < lim
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_omega_prefix_and_chunk_invariance():
    full = P.omega(99, 4, 17, 0, 40)
    assert np.array_equal(full[:, :13], P.omega(99, 4, 17, 0, 13))
    parts = np.concatenate([P.omega(99, 4, 17, 0, 7), P.omega(99, 4, 17, 7, 31), P.omega(99, 4, 17, 31, 40)], axis=1)
    assert np.array_equal(full, parts)


def test_omega_entries_on_fixed_point_grid():
    om = P.omega(3, 2, 50, 0, 64)
    q = om * 2.0 ** 20
    assert np.array_equal(q, np.rint(q)) and np.abs(q).max() < 2 ** 24
    g = P.gaussian_f64(3, 2, np.arange(50)[:, None], np.arange(64)[None, :])
    assert np.max(np.abs(om - g)) <= 2.0 ** -21


def test_golden_omega_regression():
    """Stored values written by tests/golden/make_golden.py from this oracle (regression pin)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "omega_seed20251103.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    for seed, k, i, j, hexval in rows:
        g = P.gaussian_f64(int(seed), int(k), int(i), int(j))
        assert float(g).hex() == hexval


@pytest.mark.parametrize("planted", ["multiplier", "xor"])
def test_planted_philox_mistake_changes_stream(planted, monkeypatch):
    """A planted error in the round function must change the stored golden values."""
    good = P.gaussian_f64(20251103, 2, np.arange(8), np.arange(8))
    if planted == "multiplier":
        monkeypatch.setattr(P, "_M0", np.uint64(0xD2511F55))
    else:
        monkeypatch.setattr(P, "_W1", np.uint64(0xBB67AE84))
    bad = P.gaussian_f64(20251103, 2, np.arange(8), np.arange(8))
    assert not np.array_equal(good, bad)
