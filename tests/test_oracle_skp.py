"""Pins for oracle/skp.py (the paper's SKP mesh operator)."""
import numpy as np
import pytest

from oracle import skp, spme
from paper_2601_18838_gb300 import workloads as wl


def _even_vec(rng, K):
    m = spme.wrapped_modes(K)
    base = rng.standard_normal(K // 2 + 1)
    return base[np.abs(m)]


@pytest.mark.parametrize("K", [4, 6])
def test_algorithm2_equals_explicit_kronecker(K):
    rng = np.random.default_rng(K)
    A = [rng.standard_normal((K, K)) for _ in range(3)]
    Q = rng.standard_normal((K, K, K))
    ref = (np.kron(A[0], np.kron(A[1], A[2])) @ Q.ravel()).reshape(K, K, K)
    np.testing.assert_allclose(skp.kron_apply(Q, *A), ref, atol=1e-12)


def test_circulant_eigenvectors():
    K = 12
    rng = np.random.default_rng(0)
    a = _even_vec(rng, K)
    C = skp.circulant(a)
    np.testing.assert_allclose(C, C.T, atol=1e-13)
    k = np.arange(K)
    for j, m in enumerate(spme.wrapped_modes(K)):
        v = np.cos(2 * np.pi * m * k / K)
        np.testing.assert_allclose(C @ v, K * a[j] * v, atol=1e-11)  # eigenvalue K a(m)


def test_axis_convention_single_term():
    # one rank-one term with different factors on each axis == FFT convolution with a0 (x) a1 (x) a2
    K = 10
    rng = np.random.default_rng(1)
    a0, a1, a2 = (_even_vec(rng, K) for _ in range(3))
    s = skp.SKP(K, np.array([0.7]), a0[None], a1[None], a2[None])
    Q = rng.standard_normal((K, K, K))
    T = 0.7 * np.einsum("i,j,k->ijk", a0, a1, a2)
    np.testing.assert_allclose(skp.apply(Q, s), spme.convolve_fft(Q, T), atol=1e-12)


def test_full_rank_equals_pme():
    s = wl.random_system(24, 9.0, 8, 4, 3)
    p = spme.pme(s.x, s.q, s.box, 8, 4, 0.45)
    r = skp.reciprocal(s.x, s.q, s.box, 8, 4, 0.45, 0.0)
    assert r["skp"].R == 64
    np.testing.assert_allclose(r["phi"], p["phi"], atol=1e-13 * np.abs(p["phi"]).max())
    np.testing.assert_allclose(r["F"], p["F"], atol=1e-12 * np.abs(p["F"]).max())
    assert abs(r["E"] - p["E"]) < 1e-13 * abs(p["E"])


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_truncation_bound(tol):
    K = 24
    T = spme.influence(K, 4, 15.0, 0.35)
    s = skp.nkpa(T, tol)
    err = np.linalg.norm(s.tensor() - T)
    assert err <= s.bound * (1 + 1e-9) + 1e-300
    assert s.bound <= tol * s.norm * (1 + 1e-12)
    # the error pieces are orthogonal (u_i orthonormal): exact value from the singular values
    r0 = len(s.r1)
    exact2 = np.sum(s.outer[r0:] ** 2) + sum(s.outer[i] ** 2 * np.sum(s.inner[i][s.r1[i]:] ** 2)
                                             for i in range(r0))
    assert abs(err - np.sqrt(exact2)) < 1e-9 * s.norm
    assert s.R == sum(s.r1)


def test_svd_factors_are_even():
    K = 16
    s = skp.nkpa(spme.influence(K, 4, 12.0, 0.35), 1e-8)
    m = spme.wrapped_modes(K)
    neg = np.array([np.where(m == -mm)[0][0] if -mm in m else j for j, mm in enumerate(m)])
    # odd parts are rounding noise, which grows like eps / sigma for small singular values
    for a in (s.a0, s.a1, s.a2):
        odd = np.abs(a - a[:, neg]).max(axis=1)
        assert np.all(odd * np.abs(s.w) <= 1e-13 * np.abs(s.w).max())


def test_truncated_skp_close_to_pme():
    s = wl.small()
    p = spme.pme(s.x, s.q, s.box, s.K, s.order, s.beta)
    r = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol)
    assert np.linalg.norm(r["phi"] - p["phi"]) / np.linalg.norm(p["phi"]) < 10 * s.skp_tol
    assert np.linalg.norm(r["F"] - p["F"]) / np.linalg.norm(p["F"]) < 100 * s.skp_tol
    assert abs(r["E"] - p["E"]) < 10 * s.skp_tol * abs(p["E"])


def test_skp_derivatives():
    s = wl.random_system(8, 7.0, 12, 6, 21)
    sk = skp.build(12, 6, 7.0, 0.5, 1e-10)
    r = skp.reciprocal(s.x, s.q, s.box, 12, 6, 0.5, 0, skp=sk)
    h = 1e-4
    for i, a in [(1, 0), (6, 2)]:
        xp, xm = s.x.copy(), s.x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        Ep = skp.reciprocal(xp, s.q, s.box, 12, 6, 0.5, 0, skp=sk)["E"]
        Em = skp.reciprocal(xm, s.q, s.box, 12, 6, 0.5, 0, skp=sk)["E"]
        assert abs(-(Ep - Em) / (2 * h) - r["F"][i, a]) < 1e-6 * np.abs(r["F"]).max()
    qp, qm = s.q.copy(), s.q.copy()
    qp[3] += 0.5
    qm[3] -= 0.5
    fd = (skp.reciprocal(s.x, qp, s.box, 12, 6, 0.5, 0, skp=sk)["E"]
          - skp.reciprocal(s.x, qm, s.box, 12, 6, 0.5, 0, skp=sk)["E"])
    assert abs(fd - r["phi"][3]) < 1e-12 * max(1, abs(fd))


def test_sinc_quadrature_meets_tolerance():
    args = np.arange(1.0, 300.0)
    for tol in (1e-4, 1e-8):
        nq, h, err = skp.sinc_search(args, tol)
        w, lam = skp.sinc_rule(nq, h)
        approx = np.exp(-np.outer(args, lam)) @ w
        assert np.max(np.abs(approx * args - 1)) <= tol
        assert err <= tol


def test_sinc_skp_with_correction_nonneutral():
    # q has net charge: without the c_Lambda correction the m = 0 mode leaks in
    s = wl.random_system(31, 10.0, 16, 4, 5)
    assert abs(s.q.sum()) > 0.5
    p = spme.pme(s.x, s.q, s.box, 16, 4, 0.4)
    sk = skp.build(16, 4, 10.0, 0.4, 1e-9, method="sinc")
    r = skp.reciprocal(s.x, s.q, s.box, 16, 4, 0.4, 0, skp=sk)
    rel = np.linalg.norm(r["phi"] - p["phi"]) / np.linalg.norm(p["phi"])
    assert rel < 1e-7
    no_c = skp.SKP(sk.K, sk.w, sk.a0, sk.a1, sk.a2, 0.0)
    r2 = skp.reciprocal(s.x, s.q, s.box, 16, 4, 0.4, 0, skp=no_c)
    np.testing.assert_allclose(r2["phi"] - r["phi"], sk.c * s.q.sum(), rtol=1e-9)
    # SVD and quadrature SKPs agree to their tolerances
    r3 = skp.reciprocal(s.x, s.q, s.box, 16, 4, 0.4, 1e-9)
    assert np.linalg.norm(r3["phi"] - r["phi"]) / np.linalg.norm(p["phi"]) < 1e-7
