"""Host check of the reflection basis the error-free split uses on meshes with K % 128 == 0.

A real symmetric circulant C(k, k') = g(k - k') commutes with the reflection a <-> K - 1 - a of
its axis (no fixed point for even K), so in the basis of sums x(a) + x(K-1-a), stored at a, and
differences x(a) - x(K-1-a), stored at K - 1 - a, it is block diagonal: rows n < K/2 hold
C+(n, k) = g(n - k) + g(n + k + 1); rows n >= K/2 hold the difference block at a' = K - 1 - n
with column k standing for a = K/2 - 1 - k, C-(a', a) = g(a' - a) - g(a' + a + 1).  The layout
below is the one the library materialises; the reference is the oracle's Algorithm 2 applied
with the dense circulant factors.
"""
import numpy as np
import pytest

from oracle import skp, spme


def _folded_factor(g):
    K = g.size
    h = K // 2
    F = np.empty((K, h))
    for n in range(K):
        for k in range(h):
            if n < h:
                F[n, k] = g[(n - k) % K] + g[(n + k + 1) % K]
            else:
                ap, a = K - 1 - n, h - 1 - k
                F[n, k] = g[(ap - a) % K] - g[(ap + a + 1) % K]
    return F


def _reflect(X, axis, inverse=False):
    X = np.moveaxis(X, axis, -1).copy()
    K = X.shape[-1]
    a = np.arange(K // 2)
    lo, hi = X[..., a].copy(), X[..., K - 1 - a].copy()
    X[..., a], X[..., K - 1 - a] = lo + hi, lo - hi
    if inverse:
        X *= 0.5
    return np.moveaxis(X, -1, axis)


def _block_product(X, F):
    # contract the last axis: each output half reads only its own input half
    h = F.shape[1]
    return np.concatenate([X[..., :h] @ F[:h].T, X[..., h:] @ F[h:].T], axis=-1)


@pytest.mark.parametrize("K", [8, 16])
def test_reflection_basis_reproduces_the_skp_operator(K):
    s = skp.nkpa(spme.influence(K, 4, 11.0, 0.4), 1e-6)
    r1, g3, g2, g1 = skp.generators(s)
    Q = np.random.default_rng(K).standard_normal((K, K, K))
    ref = skp.apply(Q, s)
    Qf = _reflect(_reflect(_reflect(Q, 0), 1), 2)
    Phi = np.zeros_like(Q)
    t = 0
    for i, n_in in enumerate(r1):
        Y = _block_product(Qf, _folded_factor(g3[i]))
        for _ in range(n_in):
            Z = np.moveaxis(_block_product(np.moveaxis(Y, 1, 2), _folded_factor(g2[t])), 2, 1)
            Phi += np.moveaxis(_block_product(np.moveaxis(Z, 0, 2), _folded_factor(g1[t])), 2, 0)
            t += 1
    Phi = _reflect(_reflect(_reflect(Phi, 0, True), 1, True), 2, True)
    assert np.linalg.norm(Phi - ref) <= 1e-13 * np.linalg.norm(ref)


def test_reflection_blocks_bound_and_entries():
    # entries of the blocks are bounded by 2 max |g| (the exponent of their fixed-point digits)
    # and the two blocks together hold exactly the information of the K x K circulant
    K = 12
    g = np.random.default_rng(2).standard_normal(K)
    g = 0.5 * (g + g[(-np.arange(K)) % K])          # symmetric generator g(d) = g(-d)
    F = _folded_factor(g)
    assert np.abs(F).max() <= 2 * np.abs(g).max()
    C = g[(np.arange(K)[:, None] - np.arange(K)[None, :]) % K]
    a = np.arange(K // 2)
    P = np.zeros((K, K))
    P[a, a] = P[a, K - 1 - a] = 1.0
    P[K - 1 - a, a], P[K - 1 - a, K - 1 - a] = 1.0, -1.0
    B = P @ C @ np.linalg.inv(P)                     # the circulant in the reflection basis
    h = K // 2
    # rows and columns n < h: the sum block; n >= h: the difference block, whose stored column k
    # is basis position K - 1 - a = h + k
    np.testing.assert_allclose(B[:h, :h], F[:h], atol=1e-13)
    np.testing.assert_allclose(B[h:, h:], F[h:], atol=1e-13)
    # the off-diagonal blocks vanish
    assert np.abs(B[:h, h:]).max() < 1e-13 and np.abs(B[h:, :h]).max() < 1e-13
