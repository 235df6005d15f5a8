"""The seeded input recipes stand in for the paper's point sets (Sec. 6): the ball of
radius (3N/4pi)^(1/3) and the sphere of radius (N/4pi)^(1/2) (unit volume / surface
density), uniform right-hand sides on [-0.5, 0.5], Gaussian sketches; draws are
reproducible and independent across streams."""
import numpy as np

from paper_2011_07632_gb300 import inputs


def test_ball_has_unit_density_and_uniform_radius():
    n = 200_000
    X = inputs.ball(n, 0)
    R = (3 * n / (4 * np.pi)) ** (1 / 3)
    r = np.linalg.norm(X, axis=1)
    assert r.max() <= R * (1 + 1e-12)
    # uniform in volume: P(r <= R t) = t^3 (binomial standard deviation ~ 7e-4)
    for t in (0.3, 0.5, 0.8):
        assert abs(np.mean(r <= R * t) - t ** 3) < 5e-3
    assert np.abs(X.mean(axis=0)).max() < 0.05 * R
    # the RPY radii of the paper's runs: volume fractions 0.10 and 0.31 at this density
    assert abs(4 / 3 * np.pi * 0.29 ** 3 - 0.102) < 1e-3
    assert abs(4 / 3 * np.pi * 0.42 ** 3 - 0.310) < 1e-3


def test_sphere_has_unit_surface_density():
    n = 100_000
    X = inputs.sphere(n, 0)
    R = np.sqrt(n / (4 * np.pi))
    assert np.allclose(np.linalg.norm(X, axis=1), R, rtol=1e-12)
    # uniform on the sphere: every coordinate of the unit vector is uniform on [-1, 1]
    for a in range(3):
        z = X[:, a] / R
        assert abs(np.mean(z <= 0.5) - 0.75) < 5e-3


def test_rhs_sketch_and_reproducibility():
    b = inputs.rhs_uniform(10_000, 3, 1)
    assert b.flags.f_contiguous and b.min() >= -0.5 and b.max() < 0.5
    assert abs(b.mean()) < 0.01 and abs(b.var() - 1 / 12) < 0.003
    om = inputs.sketch(10_000, 8, 2)
    assert abs(om.mean()) < 0.02 and abs(om.std() - 1) < 0.02
    assert np.array_equal(inputs.ball(100, 7), inputs.ball(100, 7))
    assert not np.array_equal(inputs.ball(100, 7), inputs.ball(100, 8))
    # different streams of one seed are different draws
    assert not np.allclose(inputs.rhs(100, 1, 1)[:, 0], inputs.sketch(100, 1, 1)[:, 0])
