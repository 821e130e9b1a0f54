"""Ranks of the two SKP constructions against the quadrature bound of §2.1.2.

Eq. estimatequad: an optimal quadrature of 1/R with |Lambda*| nodes has max error at most
16 exp(-pi sqrt(|Lambda*|)), so (ln(eps/16)/pi)^2 nodes suffice for tolerance eps.  The
cardinal-sine rule of §2.1.2 is explicit but not optimal, so its node count sits above that
figure (the paper's own example: 279 sinc nodes against 27 for a tabulated rule at 1e-14,
where the figure is 124).  The node count depends on the mesh only through the largest
argument 3 (K/2)^2, so it grows slowly with K; the two-level SVD of the B-spline influence
tensor (§2.1.1) compresses a different tensor (1/|m|^2 times the Gaussian and B-spline
factors) in the Frobenius norm, and its rank grows with K at a fixed tolerance.
"""
import math

import numpy as np
import pytest

from oracle import skp, spme


def _mode_args(K):
    m = spme.wrapped_modes(K).astype(np.float64)
    msq = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    return np.unique(msq[msq > 0])


def _bound(eps):
    return (math.log(eps / 16.0) / math.pi) ** 2


@pytest.fixture(scope="module")
def ranks():
    # (K, order, box) of the small, batched-K=48 and water workloads at their tolerance 1e-8
    out = {}
    for K, n, L in ((32, 4, 20.0), (48, 4, 55.0), (64, 4, 67.0)):
        nq, h, err = skp.sinc_search(_mode_args(K), 1e-8)
        s = skp.nkpa(spme.influence(K, n, L, 0.35), 1e-8)
        out[K] = dict(nodes=2 * nq + 1, err=err, R=s.R, r0=len(s.r1))
    return out


def test_sinc_nodes_above_optimal_rule_figure(ranks):
    for K, r in ranks.items():
        assert r["err"] <= 1e-8
        assert r["nodes"] >= _bound(1e-8), (K, r)


def test_sinc_nodes_grow_slowly_with_the_mesh(ranks):
    # K 32 -> 64 multiplies the largest argument by 4: a few nodes more, not a factor
    n32, n64 = ranks[32]["nodes"], ranks[64]["nodes"]
    assert n32 <= ranks[48]["nodes"] <= n64 <= 1.15 * n32


def test_svd_rank_grows_with_the_mesh(ranks):
    assert ranks[32]["R"] < ranks[48]["R"] < ranks[64]["R"]
    for r in ranks.values():
        assert r["r0"] < r["R"]


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-10])
def test_sinc_nodes_track_the_bound_across_tolerances(eps):
    # on the K = 32 mesh: every tolerance needs more nodes than the optimal-rule figure, and
    # tighter tolerances need more nodes
    nodes = {}
    for e in (eps, eps * 100):
        nq, _, err = skp.sinc_search(_mode_args(32), e)
        assert err <= e
        nodes[e] = 2 * nq + 1
        assert nodes[e] >= _bound(e)
    assert nodes[eps] > nodes[eps * 100]
