"""Pins for oracle/spme.py (classical smooth PME, FFT route)."""
import numpy as np
import pytest

from oracle import ewald, spme
from paper_2601_18838_gb300 import workloads as wl


def _sys(n=40, box=12.0, seed=7):
    s = wl.random_system(n, box, 32, 6, seed)
    return s.x, s.q, s.box


def test_charge_conservation_and_adjointness():
    x, q, L = _sys()
    q = q * np.linspace(0.5, 1.5, q.size)
    r = spme.pme(x, q, L, 24, 4, 0.35)
    assert abs(r["Q"].sum() - q.sum()) < 1e-12
    assert abs(np.dot(q, r["phi"]) - np.sum(r["Q"] * r["Phi"])) < 1e-11 * abs(np.dot(q, r["phi"]))


def test_converges_to_exact_reciprocal():
    x, q, L = _sys()
    ex = ewald.reciprocal_exact(x, q, L, 0.35)
    errs = []
    for K, n in ((16, 4), (32, 6), (48, 8)):
        p = spme.pme(x, q, L, K, n, 0.35)
        errs.append(np.linalg.norm(p["phi"] - ex["phi"]) / np.linalg.norm(ex["phi"]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-10
    p = spme.pme(x, q, L, 48, 8, 0.35)
    assert abs(p["E"] - ex["E"]) < 1e-10 * abs(ex["E"])
    np.testing.assert_allclose(p["F"], ex["F"], atol=1e-8 * np.abs(ex["F"]).max())


def test_brute_force_circulant_small_mesh():
    # Theta[k, k'] = theta(k - k'), theta(d) = sum_m T(m) cos(2 pi m.d / K), summed term by term
    K = 6
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((K, K, K))
    T = spme.influence(K, 4, 5.0, 0.6)
    m = spme.wrapped_modes(K)
    theta = np.zeros((K, K, K))
    for d0 in range(K):
        for d1 in range(K):
            for d2 in range(K):
                acc = 0.0
                for j0 in range(K):
                    for j1 in range(K):
                        for j2 in range(K):
                            acc += T[j0, j1, j2] * np.cos(2 * np.pi * (m[j0] * d0 + m[j1] * d1 + m[j2] * d2) / K)
                theta[d0, d1, d2] = acc
    idx = np.arange(K)
    D = (idx[:, None] - idx[None, :]) % K
    Theta = theta[D[:, None, None, :, None, None], D[None, :, None, None, :, None], D[None, None, :, None, None, :]]
    Phi = (Theta.reshape(K ** 3, K ** 3) @ Q.ravel()).reshape(K, K, K)
    np.testing.assert_allclose(spme.convolve_fft(Q, T), Phi, atol=1e-12 * np.abs(Phi).max())


def test_shift_by_one_mesh_spacing():
    x, q, L = _sys()
    K = 20
    a = spme.pme(x, q, L, K, 6, 0.35)
    b = spme.pme(x + np.array([L / K, 0.0, 2 * L / K]), q, L, K, 6, 0.35)
    np.testing.assert_allclose(b["phi"], a["phi"], atol=1e-12 * np.abs(a["phi"]).max())
    np.testing.assert_allclose(b["F"], a["F"], atol=1e-11 * np.abs(a["F"]).max())
    np.testing.assert_allclose(np.roll(a["Q"], (1, 0, 2), axis=(0, 1, 2)), b["Q"], atol=1e-13)


def test_forces_and_potentials_are_derivatives():
    x, q, L = _sys(n=10, box=8.0, seed=4)
    K, n, beta = 16, 6, 0.45
    r = spme.pme(x, q, L, K, n, beta)
    h = 1e-4
    for i, a in [(0, 0), (4, 1), (9, 2)]:
        xp, xm = x.copy(), x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = -(spme.pme(xp, q, L, K, n, beta)["E"] - spme.pme(xm, q, L, K, n, beta)["E"]) / (2 * h)
        assert abs(fd - r["F"][i, a]) < 1e-6 * np.abs(r["F"]).max()
    for i in (2, 7):
        qp, qm = q.copy(), q.copy()
        qp[i] += 0.25
        qm[i] -= 0.25
        fd = (spme.pme(x, qp, L, K, n, beta)["E"] - spme.pme(x, qm, L, K, n, beta)["E"]) / 0.5
        assert abs(fd - r["phi"][i]) < 1e-12 * max(1.0, abs(fd))


def test_virial_is_box_scaling_derivative():
    # W = -L dE/dL at fixed fractional coordinates (trace of the reciprocal virial)
    x, q, L = _sys(n=30, box=10.0, seed=9)
    K, n, beta = 24, 6, 0.4
    W = spme.pme(x, q, L, K, n, beta)["W"]
    d = 1e-5
    Ep = spme.pme(x * (1 + d), q, L * (1 + d), K, n, beta)["E"]
    Em = spme.pme(x * (1 - d), q, L * (1 - d), K, n, beta)["E"]
    assert abs(-(Ep - Em) / (2 * d) - W) < 1e-7 * abs(W)


def test_boundary_particles_wrap():
    # particles exactly on the box faces and beyond it map into [0, K)
    L, K = 10.0, 10
    x = np.array([[0.0, 0.0, 0.0], [10.0, 5.0, -10.0], [-0.0, 20.0, 9.999999999999998]])
    g, f = spme.mesh_coords(x, L, K)
    assert np.all((g >= 0) & (g < K)) and np.all((f >= 0) & (f < 1))
    assert np.all(g[0] == 0) and g[1, 0] == 0 and g[1, 2] == 0 and g[2, 1] == 0
