"""Pins of the seeded input generators against the distributions they state
(Sec. 4: uniform cube, unit-sphere surface, Gaussian, Plummer sphere), by
Kolmogorov-Smirnov distances to closed-form CDFs and by moments.  The seeds
are fixed, so every check is deterministic; the bounds are the 1 % critical
values (1.63/sqrt(n) for a KS distance, 4 standard errors for a moment)."""
import math

import numpy as np
import pytest

from paper_2012_06925_gb300 import workloads as W

N = 200_000


def ks_distance(samples, cdf):
    x = np.sort(samples)
    f = cdf(x)
    n = x.size
    i = np.arange(1, n + 1)
    return max(np.max(i / n - f), np.max(f - (i - 1) / n))


KS_1PCT = 1.63 / math.sqrt(N)


@pytest.mark.parametrize("a,rmax", [(0.1, 1.0), (1.0, 100.0)])
def test_plummer_radii_follow_the_truncated_mass_profile(a, rmax):
    """Radial CDF of a Plummer sphere truncated at rmax: m(r)/m(rmax) with
    m(r) = r^3 / (r^2 + a^2)^(3/2); directions uniform."""
    pts = W.plummer(N, np.random.default_rng(11), a=a, rmax=rmax)
    r = np.sqrt((pts * pts).sum(axis=0))
    m = lambda s: s ** 3 / (s * s + a * a) ** 1.5
    assert r.max() <= rmax * (1 + 1e-12)
    assert ks_distance(r, lambda s: m(s) / m(rmax)) < KS_1PCT
    u = pts / r
    assert np.all(np.abs(u.mean(axis=1)) < 4 / math.sqrt(3 * N))
    # half the mass of the untruncated sphere lies within a / sqrt(2^(2/3) - 1)
    if rmax / a >= 100:
        r_half = a / math.sqrt(2 ** (2 / 3) - 1)
        frac = np.mean(r <= r_half)
        assert abs(frac - 0.5 / m(rmax)) < 4 * math.sqrt(0.25 / N)


def test_sphere_surface_is_uniform_on_the_unit_sphere():
    pts = W.sphere_surface(N, np.random.default_rng(12))
    assert np.allclose(np.sqrt((pts * pts).sum(axis=0)), 1.0, atol=1e-15, rtol=0)
    # Archimedes: on the uniform unit sphere every coordinate is U[-1, 1]
    for d in range(3):
        assert ks_distance(pts[d], lambda s: (s + 1) / 2) < KS_1PCT


def test_gaussian_coordinates_have_variance_three():
    pts = W.gaussian(N, np.random.default_rng(13))
    se_var = math.sqrt(2 * 9.0 / N)
    for d in range(3):
        assert abs(pts[d].mean()) < 4 * math.sqrt(3.0 / N)
        assert abs(pts[d].var() - 3.0) < 4 * se_var
        z = pts[d] / math.sqrt(3.0)
        cdf = np.vectorize(lambda s: 0.5 * (1 + math.erf(s / math.sqrt(2))))
        assert ks_distance(z[:20_000], cdf) < 1.63 / math.sqrt(20_000)


def test_uniform_cube_and_charges():
    pts = W.uniform_cube(N, np.random.default_rng(14))
    assert pts.min() >= -1.0 and pts.max() < 1.0
    for d in range(3):
        assert ks_distance(pts[d], lambda s: (s + 1) / 2) < KS_1PCT
    q = W.uniform_charges(N, np.random.default_rng(15))
    assert q.min() >= -1.0 and q.max() < 1.0
    assert ks_distance(q, lambda s: (s + 1) / 2) < KS_1PCT
    g = W.normal_charges(N, np.random.default_rng(16))
    assert abs(g.mean()) < 4 / math.sqrt(N) and abs(g.var() - 1.0) < 4 * math.sqrt(2 / N)


def test_make_problem_is_seeded_and_shaped():
    t1, s1, q1 = W.make_problem("uniform", 1000, seed=3)
    t2, s2, q2 = W.make_problem("uniform", 1000, seed=3)
    assert np.array_equal(t1, t2) and np.array_equal(q1, q2)
    assert np.array_equal(t1, s1)                        # targets are the sources
    assert t1.shape == (3, 1000) and t1.dtype == np.float64 and t1.flags.c_contiguous
    t3, s3, q3 = W.make_problem("uniform", 1000, 700, seed=3, sources_kind="plummer")
    assert t3.shape == (3, 1000) and s3.shape == (3, 700) and q3.shape == (700,)
    assert np.sqrt((s3 * s3).sum(axis=0)).max() <= 1.0 + 1e-12
    assert not np.array_equal(W.make_problem("uniform", 1000, seed=4)[0], t1)


def test_batched_workload_generator():
    probs = W.batched_problems(count=64, seed=4, nmin=1e3, nmax=1e4)
    sizes = np.array([p["points"].shape[1] for p in probs])
    assert sizes.min() >= 1000 and sizes.max() <= 10000
    # N_p log-uniform: log10 N_p is U[3, 4]
    assert ks_distance(np.log10(sizes), lambda s: np.clip(s - 3.0, 0, 1)) < 1.63 / math.sqrt(64)
    assert {p["kernel"] for p in probs} == {W.COULOMB, W.YUKAWA}
    for i, p in enumerate(probs):
        r = np.sqrt((p["points"] ** 2).sum(axis=0))
        if i % 2:
            assert np.allclose(r, 1.0)                  # odd problems on the unit sphere
        else:
            assert np.abs(p["points"]).max() <= 1.0     # even problems in the cube
        if p["kernel"] == W.YUKAWA:
            assert 0.1 <= p["kappa"] <= 2.0
        else:
            assert p["kappa"] == 0.0
