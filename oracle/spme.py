"""Smooth particle-mesh Ewald pieces of the reciprocal path (oracle; test infrastructure).

The operator being approximated is the reciprocal Ewald kernel of §1.2,
Eq. (hexpr): H(x, y) = sum_{m != 0} alpha(|m|) exp(2 i pi <x~ - y~, m>), with
alpha(|m|) = exp(-pi^2 |m|^2 / xi^2) / |m|^2 and xi the dimensionless Ewald
parameter.  Readings fixed here (the paper gives no physical prefactor):

  * x~ is taken over the period 2 r_B = L, so xi = beta L with beta in 1/A, and
    the potential is phi(x) = (1 / (pi L)) sum_y H(x, y) q(y)
      = (1 / (pi V)) sum_{m != 0} exp(-pi^2 |k|^2 / beta^2) / |k|^2 ...,  k = m / L.
  * The m = 0 term is dropped (alpha_M(0) = 0, §2.1; tin-foil boundary).

Particle <-> mesh transfer uses cardinal B-splines (the option named in §2.2)
on a K^3 periodic mesh; the mesh operator is the circulant convolution with

  theta(d) = sum_m T(m) exp(2 i pi m.d / K),   T(m) = B(m) C(m),
  B(m) = prod_a |b(m_a)|^2,   C(m) = exp(-pi^2 |k|^2 / beta^2) / (pi V |k|^2),  C(0) = 0.

Classical PME applies it by FFT (the structure-factor factorisation of §1.2);
the paper's method applies it as a sum of Kronecker products (oracle.skp).
"""
from __future__ import annotations

import numpy as np

from . import bspline


def mesh_coords(x, box: float, K: int, center=None):
    """Mesh coordinates u = K ((x - c_B)/L + 1/2) wrapped into [0, K), split as g + f.

    A particle exactly on a cell boundary belongs to the upper cell (g = floor(u));
    u == K wraps to 0 (one cell only, as assumed in §4.2).
    """
    x = np.asarray(x, dtype=np.float64)
    c = np.full(3, 0.5 * box) if center is None else np.asarray(center, dtype=np.float64)
    u = K * ((x - c) / box + 0.5)
    u = np.mod(u, K)
    u = np.where(u >= K, u - K, u)
    g = np.floor(u).astype(np.int64)
    f = u - g
    return g, f


def spread(x, q, box: float, K: int, n: int, center=None) -> np.ndarray:
    """Charge mesh Q(k) = sum_i q_i prod_a M_n(u_ia - k_a) (periodic), the B-spline
    analogue of the interpolation matrix S_Y of §2.2, Eq. (interpkrons)."""
    g, f = mesh_coords(x, box, K, center)
    w = [bspline.weights(n, f[:, a])[0] for a in range(3)]
    q = np.asarray(q, dtype=np.float64)
    Q = np.zeros((K, K, K))
    for j0 in range(n):
        i0 = (g[:, 0] - j0) % K
        for j1 in range(n):
            i1 = (g[:, 1] - j1) % K
            w01 = q * w[0][:, j0] * w[1][:, j1]
            for j2 in range(n):
                i2 = (g[:, 2] - j2) % K
                np.add.at(Q, (i0, i1, i2), w01 * w[2][:, j2])
    return Q


def wrapped_modes(K: int) -> np.ndarray:
    """Integer mode m for each FFT index j = 0..K-1 (j for j <= K/2, j - K above)."""
    j = np.arange(K)
    return np.where(j <= K // 2, j, j - K)


def influence(K: int, n: int, box: float, beta: float) -> np.ndarray:
    """T(m) = B(m) C(m) on the FFT index grid (K, K, K); T(0) = 0."""
    m = wrapped_modes(K).astype(np.float64)
    k2 = (m / box) ** 2
    ksq = k2[:, None, None] + k2[None, :, None] + k2[None, None, :]
    bm = bspline.moduli_sq(K, n)
    B = bm[:, None, None] * bm[None, :, None] * bm[None, None, :]
    V = box ** 3
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.exp(-np.pi ** 2 * ksq / beta ** 2) / (np.pi * V * ksq)
    C[0, 0, 0] = 0.0
    return B * C


def convolve_fft(Q, T) -> np.ndarray:
    """Phi = theta * Q, theta(d) = sum_m T(m) exp(2 i pi m.d/K), via FFT (classical PME)."""
    K = Q.shape[0]
    # numpy's ifftn divides by K^3; the convolution sum carries no such factor.
    return np.real(np.fft.ifftn(T * np.fft.fftn(Q))) * float(K) ** 3


def gather(x, q, box: float, K: int, n: int, Phi, center=None):
    """phi_i = sum_k W_i(k) Phi(k) and F_i = -q_i sum_k grad W_i(k) Phi(k).

    The gradient uses dM_n/du and du/dx = K / L.  Returns (phi, F)."""
    g, f = mesh_coords(x, box, K, center)
    w, dw = zip(*[bspline.weights(n, f[:, a]) for a in range(3)])
    N = g.shape[0]
    phi = np.zeros(N)
    grad = np.zeros((N, 3))
    for j0 in range(n):
        i0 = (g[:, 0] - j0) % K
        for j1 in range(n):
            i1 = (g[:, 1] - j1) % K
            for j2 in range(n):
                i2 = (g[:, 2] - j2) % K
                P = Phi[i0, i1, i2]
                phi += w[0][:, j0] * w[1][:, j1] * w[2][:, j2] * P
                grad[:, 0] += dw[0][:, j0] * w[1][:, j1] * w[2][:, j2] * P
                grad[:, 1] += w[0][:, j0] * dw[1][:, j1] * w[2][:, j2] * P
                grad[:, 2] += w[0][:, j0] * w[1][:, j1] * dw[2][:, j2] * P
    F = -np.asarray(q, dtype=np.float64)[:, None] * grad * (K / box)
    return phi, F


def virial_influence(K: int, n: int, box: float, beta: float) -> np.ndarray:
    """T'(m) = B(m) exp(-pi^2 |k|^2/beta^2) / (pi V) on the FFT grid, T'(0) kept.

    The trace of the reciprocal virial is W = sum_m E(m) (1 - 2 pi^2 |k|^2/beta^2);
    the |k|^2 factor cancels the 1/|k|^2 of C, leaving this separable kernel."""
    m = wrapped_modes(K).astype(np.float64)
    k2 = (m / box) ** 2
    bm = bspline.moduli_sq(K, n)
    e = bm * np.exp(-np.pi ** 2 * k2 / beta ** 2)
    return e[:, None, None] * e[None, :, None] * e[None, None, :] / (np.pi * box ** 3)


def virial_tensor(Q, K: int, n: int, box: float, beta: float) -> np.ndarray:
    """Full reciprocal virial tensor of SPME (not given in the paper; the standard analytic
    derivative of the mesh energy, reading R8):

      Pi_ab = sum_{m != 0} E(m) [delta_ab - 2 (1 + pi^2 |k|^2/beta^2) k_a k_b / |k|^2],
      E(m)  = 1/2 T(m) |S(m)|^2,  S = DFT of the charge mesh,  sum_m E(m) = E,

    i.e. Pi_ab = -dE/d eps_ab under the affine strain x -> (1 + eps) x of positions and cell.
    Its trace is virial_trace()."""
    T = influence(K, n, box, beta)
    Em = 0.5 * T * np.abs(np.fft.fftn(Q)) ** 2
    k = wrapped_modes(K).astype(np.float64) / box
    ka = [k[:, None, None], k[None, :, None], k[None, None, :]]
    ksq = ka[0] ** 2 + ka[1] ** 2 + ka[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = 2.0 * (1.0 + np.pi ** 2 * ksq / beta ** 2) / ksq
    fac[0, 0, 0] = 0.0
    E = float(np.sum(Em))
    Pi = np.empty((3, 3))
    for a in range(3):
        for c in range(3):
            Pi[a, c] = (E if a == c else 0.0) - float(np.sum(Em * fac * ka[a] * ka[c]))
    return Pi


def pme(x, q, box: float, K: int, n: int, beta: float, center=None) -> dict:
    """Classical smooth PME reciprocal result (FFT route).

    Returns energy E = 1/2 sum_i q_i phi_i, potentials phi, forces F, the virial
    trace W, and the meshes Q, Phi."""
    q = np.asarray(q, dtype=np.float64)
    Q = spread(x, q, box, K, n, center)
    T = influence(K, n, box, beta)
    Phi = convolve_fft(Q, T)
    phi, F = gather(x, q, box, K, n, Phi, center)
    E = 0.5 * float(np.dot(q, phi))
    W = virial_trace(Q, E, K, n, box, beta)
    return dict(E=E, phi=phi, F=F, W=W, Q=Q, Phi=Phi)


def virial_trace(Q, E: float, K: int, n: int, box: float, beta: float) -> float:
    """W = E - (2 pi^2/beta^2) * 1/2 sum_{m != 0} T'(m) |S(m)|^2 with S the mesh DFT."""
    Tp = virial_influence(K, n, box, beta)
    S2 = np.abs(np.fft.fftn(Q)) ** 2
    s = 0.5 * float(np.sum(Tp * S2) - Tp[0, 0, 0] * S2[0, 0, 0])
    return E - 2.0 * np.pi ** 2 / beta ** 2 * s
