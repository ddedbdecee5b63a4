"""The seeded workloads follow the recipes stated for them: grid, domain,
precision, flow parameters, marker sets (counts before and after the
one-marker-per-cell dedup of the oracle) and motion.  The point sets are
checked against their closed forms, restated here."""
import math

import numpy as np
import pytest

from paper_2301_09349_gb300 import cases as C


def test_fibonacci_points_follow_their_formula():
    n = 37
    X = C.fibonacci_sphere_markers(n, radius=0.5)
    i = np.arange(n)
    z = 1.0 - 2.0 * (i + 0.5) / n
    az = math.pi * (1.0 + math.sqrt(5.0)) * i
    r = np.sqrt(1.0 - z * z)
    np.testing.assert_allclose(X, 0.5 * np.stack([r * np.cos(az), r * np.sin(az), z], 1),
                               rtol=0, atol=1e-15)
    assert np.allclose(np.linalg.norm(X, axis=1), 0.5)


def test_circle_points_are_equally_spaced():
    X = C.circle_markers(101, 0.5, (0.25, -0.5))
    d = np.linalg.norm(np.diff(np.vstack([X, X[:1]]), axis=0), axis=1)
    assert np.allclose(d, 2 * 0.5 * math.sin(math.pi / 101))
    assert np.allclose(np.linalg.norm(X - [0.25, -0.5], axis=1), 0.5)


def test_heated_sphere_recipe(oracle):
    c = C.heated_sphere()
    g = c.grid
    assert g.dim == 3 and g.n == (256, 256, 256) and g.fp_bytes == 4
    assert g.h == pytest.approx(1 / 32) and g.lo == (-3.0, -4.0, -4.0)
    assert (g.Re, g.Mach) == (300.0, 0.3) and np.all(c.Tw == 1.5)
    assert len(c.X) == 3217 == round(math.pi / g.h ** 2)
    rc, keep = oracle.dedup(g, c.X)
    assert rc == 0 and len(keep) == 2842
    assert [(v.grid.Mach, float(v.Tw[0])) for v in C.sphere_variants()] == [
        (0.3, 1.5), (0.3, 0.5), (2.0, 1.5), (2.0, 0.5)]


def test_cylinder_recipes(oracle):
    c = C.heated_cylinder()
    g = c.grid
    assert g.n[:2] == (128, 64) and g.h == 0.125 and g.lo[:2] == (-4.0, -4.0)
    assert g.fp_bytes == 8 and (g.Re, g.Mach) == (40.0, 0.1) and np.all(c.Tw == 1.1)
    assert len(c.X) == 100 and c.motion is None
    rc, keep = oracle.dedup(g, c.X)
    assert rc == 0 and len(keep) == 30
    o = C.oscillating_cylinder()
    g = o.grid
    assert g.n[:2] == (1024, 512) and g.h == 1 / 32 and g.lo[:2] == (-8.0, -8.0)
    assert g.fp_bytes == 4 and (g.Re, g.Mach) == (100.0, 0.2) and np.all(o.Tw == 1.2)
    assert len(o.X) == 101 == round(math.pi / g.h)
    assert (o.motion.amp, o.motion.freq, o.motion.axis) == (0.2, 0.2, 1)
    rc, keep = oracle.dedup(g, o.X)
    assert rc == 0 and len(keep) == 97


def test_adjoint_sphere_recipe(oracle):
    c = C.adjoint_sphere()
    g = c.grid
    assert g.n == (128, 128, 128) and g.h == 1 / 16 and g.fp_bytes == 4
    assert (g.Re, g.Mach) == (100.0, 0.5) and np.all(c.Tw == 1.5)
    assert len(c.X) == 804
    rc, keep = oracle.dedup(g, c.X)
    assert rc == 0 and len(keep) == 698


def test_initial_state_is_free_stream_plus_seeded_density_noise():
    g = C.small_grid(2, (16, 12), h=0.1, fp_bytes=8, Mach=0.3)
    a = C.initial_state(g, 5)
    b = C.initial_state(g, 5)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, C.initial_state(g, 6))
    rho = a[0]
    noise = (rho - 1.0) / 1e-3
    assert abs(noise.mean()) < 0.3 and 0.7 < noise.std() < 1.3
    # velocity and pressure uniform: momentum / rho and p are constant
    u = a[1] / rho
    assert np.allclose(u, u.flat[0]) and np.allclose(a[2] / rho, 0.0)
    p = (g.gamma - 1) * (a[3] - 0.5 * (a[1] ** 2 + a[2] ** 2) / rho)
    assert np.allclose(p, p.flat[0])
