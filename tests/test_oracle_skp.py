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


# ---- the two-level generator form handed to kpme_set_skp (§2.3 Eq. kronw, §2.4 Eq. VtV) ----
# The operator is rebuilt here from the generators alone, with circulants formed by index
# arithmetic and mode products written as explicit sums over one axis, following the
# documented contract of kpme_set_skp: term t of outer index i applies C(gen1[t]) on axis 0,
# C(gen2[t]) on axis 1 and C(gen3[i]) on axis 2, C(g)[k, k'] = g((k - k') mod K).

def _circ_from_gen(g):
    K = g.size
    k = np.arange(K)
    return g[(k[:, None] - k[None, :]) % K]


def _apply_generators(Q, r1, gen3, gen2, gen1):
    Phi = np.zeros_like(Q)
    t = 0
    for i, n_in in enumerate(r1):
        C3 = _circ_from_gen(gen3[i])
        Y = np.einsum("ck,abk->abc", C3, Q)            # axis 2
        for _ in range(n_in):
            Z = np.einsum("cj,ajk->ack", _circ_from_gen(gen2[t]), Y)    # axis 1
            Phi += np.einsum("ca,ajk->cjk", _circ_from_gen(gen1[t]), Z)  # axis 0
            t += 1
    assert t == gen2.shape[0] == gen1.shape[0]
    return Phi


@pytest.mark.parametrize("K", [8, 12])
def test_generator_closed_form(K):
    # a mode pair a(m0) = a(-m0) = 1 gives g(d) = 2 cos(2 pi m0 d / K); m0 = 0 gives 1 and the
    # Nyquist mode alone gives (-1)^d; g is the first column of the circulant
    m = spme.wrapped_modes(K)
    d = np.arange(K)
    for m0 in range(K // 2 + 1):
        a = (np.abs(m) == m0).astype(np.float64)
        g = skp.generator(a)
        if m0 == 0:
            ref = np.ones(K)
        elif m0 == K // 2:
            ref = np.cos(np.pi * d)
        else:
            ref = 2.0 * np.cos(2 * np.pi * m0 * d / K)
        np.testing.assert_allclose(g, ref, atol=1e-13)
        np.testing.assert_allclose(g, skp.circulant(a)[:, 0], atol=1e-13)


def test_generators_of_structured_two_level_skp():
    # distinct factors on every axis and distinct weights at both levels, uneven r1: the
    # generator form must reproduce the FFT convolution with sum s_i s_ij a0 (x) a1 (x) a2
    K = 8
    rng = np.random.default_rng(11)
    r1 = [2, 1, 3]
    outer = np.array([3.0, 2.0, 0.5])
    inner = [np.array([1.5, 0.25]), np.array([0.75]), np.array([2.0, 0.5, 0.125])]
    w, a0, a1, a2 = [], [], [], []
    for i, n_in in enumerate(r1):
        u = _even_vec(rng, K)
        for j in range(n_in):
            w.append(outer[i] * inner[i][j])
            a0.append(_even_vec(rng, K))
            a1.append(_even_vec(rng, K))
            a2.append(u)
    s = skp.SKP(K, np.array(w), np.array(a0), np.array(a1), np.array(a2), 0.0, r1, outer, inner)
    gr1, g3, g2, g1 = skp.generators(s)
    assert list(gr1) == r1 and g3.shape == (3, K) and g2.shape == g1.shape == (6, K)
    Q = rng.standard_normal((K, K, K))
    ref = spme.convolve_fft(Q, s.tensor())
    np.testing.assert_allclose(_apply_generators(Q, gr1, g3, g2, g1), ref, atol=1e-12 * np.abs(ref).max())
    # the plausible slips fail: factors of axes 0 and 1 swapped, or the inner weight shared
    bad = _apply_generators(Q, gr1, g3, g1, g2)
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("K,tol", [(8, 1e-5), (12, 1e-8)])
def test_generators_of_nkpa_match_apply(K, tol):
    T = spme.influence(K, 4, 9.0, 0.45)
    s = skp.nkpa(T, tol)
    assert len(s.r1) > 1 and len(set(s.r1)) > 1          # several outer terms, uneven r1
    r1, g3, g2, g1 = skp.generators(s)
    rng = np.random.default_rng(K)
    Q = rng.standard_normal((K, K, K))
    ref = skp.apply(Q, s)
    got = _apply_generators(Q, r1, g3, g2, g1)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    np.testing.assert_allclose(ref, spme.convolve_fft(Q, s.tensor()), atol=1e-12 * np.abs(ref).max())


def test_generators_full_rank_equal_pme_influence():
    # untruncated NKPA: the generator form is the PME mesh operator B(m) C(m) itself
    K = 8
    T = spme.influence(K, 4, 9.0, 0.45)
    s = skp.nkpa(T, 0.0)
    Q = np.random.default_rng(3).standard_normal((K, K, K))
    ref = spme.convolve_fft(Q, T)
    got = _apply_generators(Q, *skp.generators(s))
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
