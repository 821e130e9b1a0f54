"""Pins for oracle/ewald.py: Madelung constant, beta independence, invariances."""
import os

import numpy as np
import pytest

from oracle import ewald, spme

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    with open(os.path.join(GOLDEN, "madelung_nacl.txt")) as fh:
        return float([l for l in fh if not l.startswith("#")][0])


def _rocksalt(a=1.0):
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    x = np.concatenate([fcc, fcc + [.5, 0, 0]]) % 1.0 * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    return x, q


@pytest.mark.parametrize("beta", [4.0, 6.5])
def test_madelung_full_ewald(beta):
    # 4 ion pairs in the conventional cell: E_cell = -4 M / (a/2)
    x, q = _rocksalt(1.0)
    E = ewald.total_energy(x, q, 1.0, beta)
    assert abs(-E / 8.0 - _madelung()) < 1e-11


def test_madelung_with_pme_reciprocal():
    # real space + PME reciprocal (fine mesh, high order) + self term
    x, q = _rocksalt(1.0)
    beta = 5.0
    rec = spme.pme(x, q, 1.0, 32, 8, beta)["E"]
    E = ewald.real_space(x, q, 1.0, beta, 8.0) + rec + ewald.self_energy(q, beta)
    assert abs(-E / 8.0 - _madelung()) < 1e-9


def test_beta_independence():
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 9.0, (14, 3))
    q = np.where(np.arange(14) % 2 == 0, 1.0, -1.0) * rng.uniform(0.5, 1.5, 14)
    q -= q.mean()
    Es = [ewald.total_energy(x, q, 9.0, b) for b in (0.28, 0.4, 0.55)]
    assert np.ptp(Es) < 1e-11 * abs(Es[0])


def test_beta_independence_nonneutral_background():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 8.0, (5, 3))
    q = np.array([1.0, 1.0, -0.5, 0.25, 1.0])
    Es = [ewald.total_energy(x, q, 8.0, b) for b in (0.3, 0.45)]
    assert abs(Es[0] - Es[1]) < 1e-10 * abs(Es[0])


def test_reciprocal_translation_and_newton():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 10.0, (12, 3))
    q = np.tile([1.0, -1.0], 6)
    a = ewald.reciprocal_exact(x, q, 10.0, 0.35)
    b = ewald.reciprocal_exact(x + np.array([0.37, -1.3, 4.1]), q, 10.0, 0.35)
    assert abs(a["E"] - b["E"]) < 1e-12 * abs(a["E"])
    np.testing.assert_allclose(a["phi"], b["phi"], atol=1e-12)
    np.testing.assert_allclose(a["F"].sum(axis=0), 0.0, atol=1e-12)


def test_reciprocal_derivatives_by_finite_difference():
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 8.0, (6, 3))
    q = np.array([1.0, -1.0, 0.5, -0.5, 1.0, -1.0])
    r = ewald.reciprocal_exact(x, q, 8.0, 0.4)
    h = 1e-4
    for i, a in [(0, 0), (3, 2), (5, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = -(ewald.reciprocal_exact(xp, q, 8.0, 0.4)["E"] - ewald.reciprocal_exact(xm, q, 8.0, 0.4)["E"]) / (2 * h)
        assert abs(fd - r["F"][i, a]) < 1e-7 * max(1.0, abs(r["F"][i, a]))
    # energy is quadratic in q: central difference in q is exact up to rounding
    for i in (1, 4):
        qp, qm = q.copy(), q.copy()
        qp[i] += 0.1
        qm[i] -= 0.1
        fd = (ewald.reciprocal_exact(x, qp, 8.0, 0.4)["E"] - ewald.reciprocal_exact(x, qm, 8.0, 0.4)["E"]) / 0.2
        assert abs(fd - r["phi"][i]) < 1e-11 * max(1.0, abs(fd))
