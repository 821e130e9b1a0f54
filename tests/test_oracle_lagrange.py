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
