"""Pins of the full reciprocal virial tensor (oracle): the exact tensor equals minus the
strain derivative of the exact reciprocal energy of a deformed (triclinic) cell, the SPME
tensor has the scalar virial as its trace, permutes with the axes and converges to the
exact tensor as the mesh is refined."""
import numpy as np
import pytest

from oracle import ewald, spme
from paper_2601_18838_gb300 import workloads as wl


def _cloud(n, L, seed, neutral=True):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, (n, 3))
    q = rng.choice([-1.0, 1.0], n)
    if neutral:
        q = q - q.mean()
    return x, q


def test_exact_virial_tensor_is_minus_strain_derivative():
    # Pi_ab = -dE/d eps_ab for x -> (1 + eps) x and h -> (1 + eps) h, all nine components
    # (shear strains make the cell triclinic, so the energy is evaluated for a general cell)
    L, beta = 10.0, 0.55
    x, q = _cloud(8, L, 5)
    mmax = ewald._mode_cutoff(L, beta, 1e-18)
    Pi = ewald.reciprocal_virial_exact(x, q, L, beta)
    assert abs(ewald.reciprocal_energy_cell(x, q, L * np.eye(3), beta, mmax)
               - ewald.reciprocal_exact(x, q, L, beta)["E"]) < 1e-12
    d = 1e-5
    fd = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            def energy(t):
                A = np.eye(3)
                A[a, b] += t
                return ewald.reciprocal_energy_cell(x @ A.T, q, A @ (L * np.eye(3)), beta, mmax)
            fd[a, b] = -(energy(d) - energy(-d)) / (2 * d)
    assert np.abs(Pi - fd).max() < 1e-8 * np.abs(Pi).max()
    np.testing.assert_allclose(Pi, Pi.T, atol=1e-14)


def test_spme_virial_tensor_trace_symmetry_permutation():
    L, beta, K, n = 12.0, 0.45, 24, 6
    x, q = _cloud(40, L, 7, neutral=False)
    r = spme.pme(x, q, L, K, n, beta)
    Pi = spme.virial_tensor(r["Q"], K, n, L, beta)
    assert abs(np.trace(Pi) - r["W"]) < 1e-13 * abs(r["W"])
    np.testing.assert_array_equal(Pi, Pi.T)
    # cyclic permutation of the axes permutes the tensor (the mesh treats the axes alike)
    perm = [1, 2, 0]
    r2 = spme.pme(x[:, perm], q, L, K, n, beta)
    Pi2 = spme.virial_tensor(r2["Q"], K, n, L, beta)
    np.testing.assert_allclose(Pi2, Pi[np.ix_(perm, perm)], rtol=0, atol=1e-12 * np.abs(Pi).max())


def test_spme_virial_tensor_converges_to_exact():
    L, beta = 12.0, 0.45
    x, q = _cloud(40, L, 7, neutral=False)
    Pe = ewald.reciprocal_virial_exact(x, q, L, beta)
    errs = []
    for K, n in [(16, 4), (24, 6), (48, 8)]:
        r = spme.pme(x, q, L, K, n, beta)
        errs.append(np.linalg.norm(spme.virial_tensor(r["Q"], K, n, L, beta) - Pe) / np.linalg.norm(Pe))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8, errs


def test_virial_tensor_small_workload_reference():
    # the small box of the GPU tests: its tensor is finite, symmetric and has trace W
    s = wl.small()
    r = spme.pme(s.x, s.q, s.box, s.K, s.order, s.beta)
    Pi = spme.virial_tensor(r["Q"], s.K, s.order, s.box, s.beta)
    assert np.all(np.isfinite(Pi)) and abs(np.trace(Pi) - r["W"]) < 1e-12 * abs(r["W"])
