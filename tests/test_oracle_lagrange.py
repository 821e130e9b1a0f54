"""Pins of the per-cell Lagrange form of KPME (oracle): the basis against the definitions of
interpolation, the geometric decay of Thm. 3, convergence of Algorithm 4 to the direct sum on
the same mode cube, the quadrature SKP against the exact node operator, and forces against
finite differences of the energy."""
import math

import numpy as np
import pytest

from oracle import lagrange as lg


def test_lagrange_basis_definitions():
    t = np.linspace(-1.0, 1.0, 41)
    for Ln in (2, 3, 4, 8, 12):
        S, dS = lg.lagrange_basis(Ln, t)
        tn = lg.lagrange_nodes(Ln)
        np.testing.assert_allclose(S.sum(axis=1), 1.0, atol=1e-13)            # partition of unity
        np.testing.assert_allclose(dS.sum(axis=1), 0.0, atol=1e-10)
        for p in range(Ln):                                                    # exact on degree < Ln
            np.testing.assert_allclose(S @ tn ** p, t ** p, atol=1e-12)
        Sn, _ = lg.lagrange_basis(Ln, tn)
        np.testing.assert_allclose(Sn, np.eye(Ln), atol=1e-14)                 # cardinal at the nodes
        h = 1e-6                                                               # derivative
        Sp, _ = lg.lagrange_basis(Ln, t + h)
        Sm, _ = lg.lagrange_basis(Ln, t - h)
        np.testing.assert_allclose(dS, (Sp - Sm) / (2 * h), atol=1e-6 * max(1.0, np.abs(dS).max()))


def test_interpolation_of_exponential_decays_geometrically():
    # Thm. 3: the interpolation error of exp(2 i pi M x) on a cell of side 1/Kc decays like nu^L
    Kc, M = 8, 4
    hc = 1.0 / Kc
    x = np.linspace(0.0, hc, 301)
    errs = []
    for Ln in range(4, 16, 2):
        S, _ = lg.lagrange_basis(Ln, 2 * x / hc - 1)
        xn = (lg.lagrange_nodes(Ln) + 1) / 2 * hc
        errs.append(np.abs(S @ np.exp(2j * np.pi * M * xn) - np.exp(2j * np.pi * M * x)).max())
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.all(ratios < 0.1), errs
    assert errs[-1] < 5e-11
    # and within the bound of the proof, (pi M r / L)^L (2L)!/(L!)^2 with r = 1/(2 Kc)
    for Ln, e in zip(range(4, 16, 2), errs):
        bound = (math.pi * M / (2 * Kc) / Ln) ** Ln * math.comb(2 * Ln, Ln)
        assert e <= bound


@pytest.fixture(scope="module")
def cloud():
    rng = np.random.default_rng(11)
    L, beta, N, M = 20.0, 0.15, 60, 4
    x = rng.uniform(0.0, L, (N, 3))
    q = rng.choice([-1.0, 1.0], N)
    q -= q.mean()
    return x, q, L, beta, M, lg.direct(x, q, L, beta, M)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_lagrange_kpme_converges_to_direct_sum(cloud):
    x, q, L, beta, M, ref = cloud
    r8 = lg.reciprocal(x, q, L, beta, 4, 8, M)
    r12 = lg.reciprocal(x, q, L, beta, 4, 12, M)
    for r, tol in ((r8, 1e-6), (r12, 1e-9)):
        assert _rel(r["phi"], ref["phi"]) < tol and _rel(r["F"], ref["F"]) < 30 * tol
        assert abs(r["E"] - ref["E"]) < tol * abs(ref["E"])
    assert _rel(r12["phi"], ref["phi"]) < 1e-3 * _rel(r8["phi"], ref["phi"])
    # charge conservation and adjointness of S_X^* and S_Y
    assert abs(r12["Q"].sum() - q.sum()) < 1e-12
    assert abs(float(np.dot(q, r12["phi"])) - float(np.sum(r12["Q"] * r12["Phi"]))) < 1e-10 * abs(r12["E"])


def test_sinc_skp_matches_exact_node_operator(cloud):
    x, q, L, beta, M, _ = cloud
    Qn = lg.spread(x, q, L, 4, 12)
    ex = lg.apply_exact(Qn, 4, 12, L, beta, M)
    w, A, c = lg.sinc_factors(4, 12, L, beta, M, 1e-12)
    sk = lg.apply_skp(Qn, w, A, c, L)
    assert _rel(sk, ex) < 1e-10
    # the m = 0 correction: with non-neutral charges the SKP without it is off by c sum(q)
    q1 = q + 0.3
    Q1 = lg.spread(x, q1, L, 4, 12)
    np.testing.assert_allclose(lg.apply_skp(Q1, w, A, c, L), lg.apply_exact(Q1, 4, 12, L, beta, M),
                               rtol=0, atol=1e-10 * np.abs(lg.apply_exact(Q1, 4, 12, L, beta, M)).max())


def test_lagrange_forces_match_energy_differences(cloud):
    x, q, L, beta, M, _ = cloud
    r = lg.reciprocal(x, q, L, beta, 4, 10, M)
    h = 1e-5
    for i in (0, 7):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(lg.reciprocal(xp, q, L, beta, 4, 10, M)["E"] - lg.reciprocal(xm, q, L, beta, 4, 10, M)["E"]) / (2 * h)
            assert abs(fd - r["F"][i, a]) < 1e-6 * max(1.0, abs(r["F"][i, a]))


def test_quadrature_terms_collapse_to_one_mode_space_diagonal(cloud):
    # Eq. VtV: every term's axis factor is W^* diag(a_lambda) W on the same Fourier rows of the
    # node positions, so the sum over the terms is one diagonal in mode space.  Written here in
    # the real rows the mode-space form uses (1, cos 2 pi m y, sin 2 pi m y; the +-m pairs folded
    # with weight 2, the m = 0 entry zero), against the oracle's term-by-term loop.
    from oracle import skp
    x, q, L, beta, M, _ = cloud
    Kc, Ln, tol = 4, 8, 1e-12
    Qn = lg.spread(x, q, L, Kc, Ln)
    w, A, c = lg.sinc_factors(Kc, Ln, L, beta, M, tol)
    ref = lg.apply_skp(Qn, w, A, c, L)
    m = np.arange(-M, M + 1)
    msq = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    nq, h, _ = skp.sinc_search(np.unique(msq[msq > 0]).astype(np.float64), tol)
    wl, lam = skp.sinc_rule(nq, h)
    assert np.allclose(wl, w)
    y = lg.node_positions(Kc, Ln)
    mu_m = np.array([0] + [k for k in range(1, M + 1) for _ in (0, 1)])         # mode of each row
    U = np.vstack([np.ones_like(y)] + [f(2 * np.pi * k * y) for k in range(1, M + 1) for f in (np.cos, np.sin)])
    kap = np.where(mu_m == 0, 1.0, 2.0)
    s2 = mu_m[:, None, None] ** 2 + mu_m[None, :, None] ** 2 + mu_m[None, None, :] ** 2
    xi2 = (beta * L) ** 2
    D = np.einsum("l,labc->abc", wl, np.exp(-(lam[:, None, None, None] + math.pi ** 2 / xi2) * s2[None]))
    D = np.where(s2 == 0, 0.0, D) * kap[:, None, None] * kap[None, :, None] * kap[None, None, :] / (math.pi * L)
    That = np.einsum("ag,bh,ck,ghk->abc", U, U, U, Qn)
    Phi = np.einsum("ag,bh,ck,abc->ghk", U, U, U, D * That)
    assert _rel(Phi, ref) < 1e-12
    # and the zeroed m = 0 entry is exactly the correction term: without it the diagonal is
    # the uncorrected sum, off by c_Lambda sum(Q)
    D0 = D.copy()
    D0[0, 0, 0] = float(np.sum(wl)) / (math.pi * L)
    Phi0 = np.einsum("ag,bh,ck,abc->ghk", U, U, U, D0 * That)
    assert np.allclose(Phi0 - Phi, c * Qn.sum() / (math.pi * L), rtol=0, atol=1e-12 * np.abs(Phi).max())


def test_error_follows_nu_to_the_order_and_reaches_the_double_floor(cloud):
    # §5.1: the overall error follows the interpolation error, O(nu^L) with nu ~ M r_c, so
    # halving the cells at a fixed order divides it by about 2^L; with equispaced nodes high
    # orders lose digits to rounding, and the ~1e-14 floor is reached with more cells instead.
    x, q, L, beta, M, ref = cloud
    cases = [(2, 8), (4, 8), (8, 8), (4, 6), (8, 6), (8, 12)]
    e = {c: _rel(lg.reciprocal(x, q, L, beta, c[0], c[1], M)["phi"], ref["phi"]) for c in cases}
    for Ln, pairs in ((8, [(2, 4), (4, 8)]), (6, [(4, 8)])):
        for a, b in pairs:
            ratio = e[(a, Ln)] / e[(b, Ln)]
            assert 2 ** Ln / 3 < ratio < 3 * 2 ** Ln, (Ln, a, b, ratio)
    assert e[(8, 12)] < 3e-13
