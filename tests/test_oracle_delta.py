"""Pins of the oracle's regularised delta (Sec. 2.2, the 3-point kernel of
Pinelli et al.) against closed forms and the moment conditions the kernel is
built to satisfy."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_phi_golden_values(oracle):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "delta_values.txt"))
            if l.strip() and not l.startswith("#")][1:]
    r = np.array([float(a) for a, _ in rows])
    want = np.array([float(b) for _, b in rows])
    got = oracle.phi(r)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-16)


def test_phi_symmetric_and_support(oracle):
    r = np.linspace(0, 2.5, 2001)
    np.testing.assert_array_equal(oracle.phi(r), oracle.phi(-r))
    assert np.all(oracle.phi(r[r >= 1.5]) == 0.0)
    assert np.all(oracle.phi(r[r < 1.5]) > 0.0)


@pytest.fixture(scope="module")
def shifts():
    rng = np.random.Generator(np.random.PCG64(7))
    return rng.random(10000) - 0.5


def _stencil(oracle, r):
    j = np.arange(-3, 4)
    x = r[:, None] - j[None, :]
    return x, oracle.phi(x.ravel()).reshape(x.shape)


def test_partition_of_unity(oracle, shifts):
    _, w = _stencil(oracle, shifts)
    np.testing.assert_allclose(w.sum(1), 1.0, atol=4e-16)


def test_first_moment_zero(oracle, shifts):
    x, w = _stencil(oracle, shifts)
    np.testing.assert_allclose((x * w).sum(1), 0.0, atol=6e-16)


def test_sum_of_squares_half(oracle, shifts):
    # the identity that makes an isolated marker's quadrature weight 2^d
    _, w = _stencil(oracle, shifts)
    np.testing.assert_allclose((w * w).sum(1), 0.5, atol=4e-16)


def test_second_moment_not_constant(oracle, shifts):
    # the 3-point kernel does NOT have a constant second moment
    x, w = _stencil(oracle, shifts)
    m2 = (x * x * w).sum(1)
    assert m2.max() - m2.min() > 0.05


@pytest.mark.parametrize("r0", [0.5, 1.5])
def test_c1_continuity(oracle, r0):
    e = 1e-7
    left = (oracle.phi(r0 - e) - oracle.phi(r0 - 2 * e)) / e
    right = (oracle.phi(r0 + 2 * e) - oracle.phi(r0 + e)) / e
    assert abs(oracle.phi(r0 - 1e-12)[0] - oracle.phi(r0 + 1e-12)[0]) < 1e-11
    assert abs(left[0] - right[0]) < 1e-5
    if r0 == 0.5:
        assert abs(left[0] + 1.0) < 1e-5   # phi'(1/2) = -1
    else:
        assert abs(left[0]) < 1e-5         # phi'(3/2) = 0
