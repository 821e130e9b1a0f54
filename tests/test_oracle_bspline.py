"""Pins for oracle/bspline.py against closed forms of cardinal B-splines."""
import numpy as np
import pytest

from oracle import bspline


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8])
def test_partition_of_unity(n):
    f = np.linspace(0.0, 0.999999, 97)
    w, dw = bspline.weights(n, f)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dw.sum(axis=1), 0.0, atol=1e-13)
    assert np.all(w >= 0)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7])
def test_symmetry_and_support(n):
    u = np.linspace(-1, n + 1, 301)
    np.testing.assert_allclose(bspline.M(n, u), bspline.M(n, n - u), atol=1e-14)
    assert np.all(bspline.M(n, u[(u <= 0) | (u >= n)]) == 0)


def test_cubic_and_quintic_closed_forms():
    # cubic: M_4 = (1/6) u^3 on [0,1]; integer values 1/6, 2/3, 1/6
    u = np.linspace(0, 1, 11)
    np.testing.assert_allclose(bspline.M(4, u), u ** 3 / 6, atol=1e-15)
    np.testing.assert_allclose(bspline.M(4, np.array([1.0, 2.0, 3.0])), [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    # order 6 at the integers: (1, 26, 66, 26, 1) / 120
    np.testing.assert_allclose(bspline.M(6, np.arange(1.0, 6.0)), np.array([1, 26, 66, 26, 1]) / 120,
                               atol=1e-15)


def test_derivative_by_finite_difference():
    u = np.linspace(0.05, 5.95, 59)
    h = 1e-6
    fd = (bspline.M(6, u + h) - bspline.M(6, u - h)) / (2 * h)
    np.testing.assert_allclose(bspline.dM(6, u), fd, atol=1e-8)


@pytest.mark.parametrize("K", [8, 32, 50])
def test_moduli_closed_form_order4(K):
    # sum_j M_4(j+1) e^{i j t} = e^{i t} (2/3 + cos(t)/3)  =>  |b|^2 = 9 / (2 + cos t)^2
    t = 2 * np.pi * np.arange(K) / K
    np.testing.assert_allclose(bspline.moduli_sq(K, 4), 9.0 / (2.0 + np.cos(t)) ** 2, rtol=1e-13)


def test_moduli_zero_mode_is_one():
    for n in (4, 6, 8):
        assert abs(bspline.moduli_sq(64, n)[0] - 1.0) < 1e-14
