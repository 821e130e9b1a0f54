"""Exact Ewald summation (oracle; test infrastructure, used only to pin the others).

§1.2, Eq. (tau) splits the Coulomb kernel with tau(R) = erf(xi R); the long-range
part is the reciprocal sum of Eq. (hexpr), the short-range part an absolutely
convergent real-space lattice sum.  With beta in 1/A, V = L^3, k = m / L:

  E_rec  = 1/(2 pi V) sum_{m != 0} exp(-pi^2 |k|^2/beta^2)/|k|^2 |S(k)|^2,
           S(k) = sum_j q_j exp(2 i pi k.x_j)
  E_real = 1/2 sum_{i,j} sum_n' q_i q_j erfc(beta |x_i - x_j + n L|) / |x_i - x_j + n L|
  E_self = -beta/sqrt(pi) sum_i q_i^2
  E_bg   = -pi (sum_i q_i)^2 / (2 V beta^2)      (neutralising background, 0 if neutral)

E_total = E_real + E_rec + E_self + E_bg does not depend on beta; that and the
Madelung constant of rock salt pin the reciprocal normalisation.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def _mode_cutoff(box: float, beta: float, eps: float) -> int:
    # exp(-pi^2 m^2 / (beta L)^2) < eps  <=>  m > beta L sqrt(-ln eps) / pi
    return int(math.ceil(beta * box * math.sqrt(-math.log(eps)) / math.pi))


def reciprocal_exact(x, q, box: float, beta: float, eps: float = 1e-18, center=None, mmax: int | None = None) -> dict:
    """Exact (mode-truncated at exp(-pi^2|k|^2/beta^2) < eps, or on the cube |m|_inf <= mmax
    when given) reciprocal Ewald sum.

    Returns E, potentials phi_i = dE/dq_i and forces F_i = -dE/dx_i."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    c = np.full(3, 0.5 * box) if center is None else np.asarray(center, dtype=np.float64)
    s = (x - c) / box + 0.5
    if mmax is None:
        mmax = _mode_cutoff(box, beta, eps)
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    e = [np.exp(2j * np.pi * np.outer(s[:, a], m)) for a in range(3)]   # (N, M)
    k2 = (m / box) ** 2
    N, M = x.shape[0], m.size
    V = box ** 3
    phi = np.zeros(N)
    F = np.zeros((N, 3))
    E = 0.0
    for i0 in range(M):
        ksq = k2[i0] + k2[:, None] + k2[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.exp(-np.pi ** 2 * ksq / beta ** 2) / ksq
        if m[i0] == 0:
            g[mmax, mmax] = 0.0
        A = (q * e[0][:, i0])[:, None] * e[1]          # (N, M1)
        S = A.T @ e[2]                                   # (M1, M2) structure factor
        E += float(np.sum(g * np.abs(S) ** 2)) / (2 * np.pi * V)
        G = g * np.conj(S)                               # (M1, M2)
        # sum_{m1,m2} G[m1,m2] exp(2 i pi (m0 s0 + m1 s1 + m2 s2)) per particle
        t = e[0][:, i0] * np.einsum("nj,jk,nk->n", e[1], G, e[2])
        phi += np.real(t) / (np.pi * V)
        # gradient of exp(2 i pi k.x) is 2 i pi k exp(...)
        t0 = e[0][:, i0] * np.einsum("nj,jk,nk->n", e[1], G, e[2]) * m[i0]
        t1 = e[0][:, i0] * np.einsum("nj,jk,nk->n", e[1] * m[None, :], G, e[2])
        t2 = e[0][:, i0] * np.einsum("nj,jk,nk->n", e[1], G, e[2] * m[None, :])
        for a, ta in enumerate((t0, t1, t2)):
            F[:, a] -= q * np.real(2j * np.pi / box * ta) / (np.pi * V)
    return dict(E=E, phi=phi, F=F)


def reciprocal_energy_cell(x, q, h, beta: float, mmax: int) -> float:
    """Exact reciprocal energy for a general (triclinic) periodic cell with cell vectors the
    columns of h: E = 1/(2 pi V) sum_{m != 0, |m|_inf <= mmax} exp(-pi^2|k|^2/beta^2)/|k|^2 |S(k)|^2
    with k = h^-T m, V = |det h| and S(k) = sum_j q_j exp(2 i pi k.x_j).  Used to pin the
    virial tensor by finite differences of a strained cell (a cubic box is h = L I)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    V = abs(float(np.linalg.det(h)))
    r = np.arange(-mmax, mmax + 1, dtype=np.float64)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k = m @ np.linalg.inv(h)                      # rows: k = h^-T m
    ksq = np.sum(k * k, axis=1)
    S = np.exp(2j * np.pi * (k @ x.T)) @ q        # (n_modes,)
    return float(np.sum(np.exp(-np.pi ** 2 * ksq / beta ** 2) / ksq * np.abs(S) ** 2)) / (2 * np.pi * V)


def reciprocal_virial_exact(x, q, box: float, beta: float, eps: float = 1e-18, center=None) -> np.ndarray:
    """Exact reciprocal virial tensor of a cubic box (modes truncated as in reciprocal_exact):
    Pi_ab = sum_{m != 0} E(m) [delta_ab - 2 (1 + pi^2|k|^2/beta^2) k_a k_b/|k|^2] with
    E(m) = exp(-pi^2|k|^2/beta^2)/|k|^2 |S(k)|^2 / (2 pi V)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    c = np.full(3, 0.5 * box) if center is None else np.asarray(center, dtype=np.float64)
    s = (x - c) / box + 0.5
    mmax = _mode_cutoff(box, beta, eps)
    r = np.arange(-mmax, mmax + 1, dtype=np.float64)
    e = [np.exp(2j * np.pi * np.outer(s[:, a], r)) for a in range(3)]
    k1 = r / box
    V = box ** 3
    Pi = np.zeros((3, 3))
    E = 0.0
    for i0 in range(r.size):
        ka = [np.full((r.size, r.size), k1[i0]), np.broadcast_to(k1[:, None], (r.size, r.size)),
              np.broadcast_to(k1[None, :], (r.size, r.size))]
        ksq = ka[0] ** 2 + ka[1] ** 2 + ka[2] ** 2
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.exp(-np.pi ** 2 * ksq / beta ** 2) / ksq
            fac = 2.0 * (1.0 + np.pi ** 2 * ksq / beta ** 2) / ksq
        if r[i0] == 0:
            g[mmax, mmax] = 0.0
            fac[mmax, mmax] = 0.0
        S = ((q * e[0][:, i0])[:, None] * e[1]).T @ e[2]
        Em = g * np.abs(S) ** 2 / (2 * np.pi * V)
        E += float(np.sum(Em))
        for a in range(3):
            for b in range(3):
                Pi[a, b] -= float(np.sum(Em * fac * ka[a] * ka[b]))
    return Pi + E * np.eye(3)


def real_space(x, q, box: float, beta: float, rcut: float) -> float:
    """E_real over all image pairs with |r| < rcut (the i = j, n = 0 term excluded)."""
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    nimg = int(math.ceil(rcut / box)) + 1
    E = 0.0
    d = x[:, None, :] - x[None, :, :]
    qq = q[:, None] * q[None, :]
    rng = range(-nimg, nimg + 1)
    for a in rng:
        for b in rng:
            for c in rng:
                r = np.linalg.norm(d + box * np.array([a, b, c], dtype=np.float64), axis=2)
                if a == 0 and b == 0 and c == 0:
                    np.fill_diagonal(r, np.inf)
                mask = r < rcut
                E += 0.5 * float(np.sum(qq[mask] * erfc(beta * r[mask]) / r[mask]))
    return E


def self_energy(q, beta: float) -> float:
    q = np.asarray(q, dtype=np.float64)
    return -beta / math.sqrt(math.pi) * float(np.dot(q, q))


def background_energy(q, box: float, beta: float) -> float:
    Q = float(np.sum(q))
    return -math.pi * Q * Q / (2.0 * box ** 3 * beta ** 2)


def total_energy(x, q, box: float, beta: float, rcut: float | None = None,
                 eps: float = 1e-18) -> float:
    """Full Ewald energy (tin-foil boundary) with real-space cutoff where erfc < eps."""
    if rcut is None:
        rcut = math.sqrt(-math.log(eps)) / beta + 1.0
    return (real_space(x, q, box, beta, rcut) + reciprocal_exact(x, q, box, beta, eps)["E"]
            + self_energy(q, beta) + background_energy(q, box, beta))
