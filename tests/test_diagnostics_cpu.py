"""Host diagnostics and the oracle's surface pressure, pinned to closed forms."""
import numpy as np
import pytest

from paper_2301_09349_gb300 import cases as C
from paper_2301_09349_gb300 import diagnostics


def test_strouhal_of_a_sinusoid():
    t = np.linspace(0.0, 60.0, 6001)
    for f in (0.165, 0.21, 0.33):
        cl = 0.3 * np.sin(2 * np.pi * f * t + 0.4) + 0.05
        assert diagnostics.strouhal(t, cl) == pytest.approx(f, rel=1e-4)
        assert diagnostics.strouhal(t, cl, D=2.0, U=4.0) == pytest.approx(f / 2.0, rel=1e-4)
    assert np.isnan(diagnostics.strouhal(t, np.ones_like(t)))


def test_surface_pressure_is_exact_for_affine_pressure(oracle):
    """Interpolation reproduces affine fields exactly (sum phi = 1,
    sum (r - j) phi = 0), so C_p = 2 (p(X) - p_inf) for p = p_inf + a.x"""
    g = C.small_grid(2, (24, 20), h=0.1, fp_bytes=8, Mach=0.3)
    X = C.circle_markers(20, 0.5, (0.02, 0.01))
    a = np.array([0.3, -0.7])
    p_inf = 1.0 / (g.gamma * g.Mach ** 2)
    x = g.lo[0] + (np.arange(g.n[0]) + 0.5) * g.h
    y = g.lo[1] + (np.arange(g.n[1]) + 0.5) * g.h
    XX, YY = np.meshgrid(x, y)
    p = p_inf + a[0] * XX + a[1] * YY
    U = np.zeros((4, g.n[1], g.n[0]))
    U[0] = 1.2
    U[1] = 0.4
    U[2] = -0.1
    U[3] = p / (g.gamma - 1.0) + 0.5 * (0.4 ** 2 + 0.1 ** 2) / 1.2
    cp = oracle.surface_pressure(g, X, U)
    assert np.allclose(cp, 2.0 * (X @ a), atol=1e-12)


def test_streamwise_case_follows_the_paper_parameters():
    c = C.streamwise_oscillating_cylinder()
    assert c.motion.axis == 0 and c.motion.amp == pytest.approx(0.14)
    assert c.motion.freq == pytest.approx(2 * C.ST0_RE100)
    assert c.grid.Mach == 0.3 and c.grid.Re == 100.0 and np.all(c.Tw == 1.0)
