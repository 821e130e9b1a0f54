"""Per-cell Lagrange form of KPME (§2.2, §4.1, §4.2, Algorithm 4) — oracle, test infrastructure.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline use this module.

The periodic box (fractional coordinates s = (x - c_B)/L + 1/2 in [0, 1), reading R1) is cut
into Kc^3 cubic cells (§4.1); every cell carries the product grid of Ln equispaced interpolation
nodes per axis, t_l = -1 + 2 l/(Ln - 1) in the cell's local coordinate t in [-1, 1]
(Eq. interp1d), so the node tensor has n = Kc Ln nodes per axis (the end nodes of neighbouring
cells share a position but belong to different cells).  S_Y (Eq. sxsyfromB) holds each
particle's Ln^3 Lagrange weights on its own cell.  The reciprocal kernel on the modes
|m|_inf <= M (Eq. hexpr restricted to the cube of §2.1),

    H_M(x, y) = sum_{0 != m in [-M, M]^3} alpha(|m|) exp(2 i pi m.(s_x - s_y)),
    alpha(r) = exp(-pi^2 r^2 / xi^2) / r^2,   xi = beta L,

is approximated by S_X^* A S_Y with A(g, h) = sum_m alpha(|m|) exp(2 i pi m.(y_g - y_h)) on the
node positions y (Eq. formfinale), and the potential is phi = (1/(pi L)) H_M q (reading R2).
With the quadrature SKP of alpha_M (Eq. quaddecompalpham) the node operator is

    A = sum_l w_l A_l (x) A_l (x) A_l - c_Lambda 1 1^T,
    A_l(g, h) = sum_{m=-M}^{M} exp(-(lambda_l + pi^2/xi^2) m^2) cos(2 pi m (y_g - y_h)),

the real cosine form of §2.3 summed over the modes (the factored V*V of Eq. VtV, formed as a
dense n x n matrix), and c_Lambda = sum_l w_l multiplies sum_h Q_h = sum q (the correction
term of Eq. termbonsum).
"""
from __future__ import annotations

import math

import numpy as np

from . import ewald, skp


def lagrange_nodes(Ln: int) -> np.ndarray:
    """Equispaced nodes t_l = -1 + 2 l/(Ln - 1) on [-1, 1] (the grid of Thm. 3)."""
    return np.linspace(-1.0, 1.0, Ln)


def lagrange_basis(Ln: int, t) -> tuple[np.ndarray, np.ndarray]:
    """S_l(t) = prod_{k != l} (t - t_k)/(t_l - t_k) (Eq. interp1d) and dS_l/dt, shape (N, Ln),
    written out as the products of the definition."""
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    tn = lagrange_nodes(Ln)
    S = np.ones((t.size, Ln))
    dS = np.zeros((t.size, Ln))
    for l in range(Ln):
        for k in range(Ln):
            if k == l:
                continue
            # derivative of the product: sum over the factor that is differentiated
            term = np.full(t.size, 1.0 / (tn[l] - tn[k]))
            for j in range(Ln):
                if j != l and j != k:
                    term = term * (t - tn[j]) / (tn[l] - tn[j])
            dS[:, l] += term
            S[:, l] *= (t - tn[k]) / (tn[l] - tn[k])
    return S, dS


def node_positions(Kc: int, Ln: int) -> np.ndarray:
    """Fractional positions of the n = Kc Ln nodes of one axis: cell i, node l at
    (i + (1 + t_l)/2) / Kc."""
    tn = lagrange_nodes(Ln)
    return ((np.arange(Kc)[:, None] + 0.5 * (1.0 + tn[None, :])) / Kc).reshape(-1)


def cell_coords(x, box: float, Kc: int, center=None):
    """Cell index i (N, 3) and local coordinate t in [-1, 1] (N, 3) of every particle; a particle
    on a cell boundary belongs to the upper cell (one cell only, §4.2), s == 1 wraps to 0."""
    x = np.asarray(x, dtype=np.float64)
    c = np.full(3, 0.5 * box) if center is None else np.asarray(center, dtype=np.float64)
    s = np.mod((x - c) / box + 0.5, 1.0)
    s = np.where(s >= 1.0, s - 1.0, s)
    u = Kc * s
    i = np.floor(u).astype(np.int64)
    i = np.minimum(i, Kc - 1)
    return i, 2.0 * (u - i) - 1.0


def spread(x, q, box: float, Kc: int, Ln: int, center=None) -> np.ndarray:
    """Node charges Q = S_Y q (n^3, n = Kc Ln): q_y times its Lagrange weights on its cell's nodes."""
    i, t = cell_coords(x, box, Kc, center)
    S = [lagrange_basis(Ln, t[:, a])[0] for a in range(3)]
    q = np.asarray(q, dtype=np.float64)
    n = Kc * Ln
    Q = np.zeros((n, n, n))
    for l0 in range(Ln):
        g0 = i[:, 0] * Ln + l0
        for l1 in range(Ln):
            g1 = i[:, 1] * Ln + l1
            w01 = q * S[0][:, l0] * S[1][:, l1]
            for l2 in range(Ln):
                np.add.at(Q, (g0, g1, i[:, 2] * Ln + l2), w01 * S[2][:, l2])
    return Q


def gather(x, q, box: float, Kc: int, Ln: int, Phi, center=None):
    """phi_x = sum_g S(g, x) Phi_g (S_X^*) and F_x = -q_x grad_x phi_x (dt/dx = 2 Kc / L)."""
    i, t = cell_coords(x, box, Kc, center)
    SW = [lagrange_basis(Ln, t[:, a]) for a in range(3)]
    N = i.shape[0]
    phi = np.zeros(N)
    grad = np.zeros((N, 3))
    for l0 in range(Ln):
        g0 = i[:, 0] * Ln + l0
        for l1 in range(Ln):
            g1 = i[:, 1] * Ln + l1
            for l2 in range(Ln):
                P = Phi[g0, g1, i[:, 2] * Ln + l2]
                s0, s1, s2 = SW[0][0][:, l0], SW[1][0][:, l1], SW[2][0][:, l2]
                d0, d1, d2 = SW[0][1][:, l0], SW[1][1][:, l1], SW[2][1][:, l2]
                phi += s0 * s1 * s2 * P
                grad[:, 0] += d0 * s1 * s2 * P
                grad[:, 1] += s0 * d1 * s2 * P
                grad[:, 2] += s0 * s1 * d2 * P
    F = -np.asarray(q, dtype=np.float64)[:, None] * grad * (2.0 * Kc / box)
    return phi, F


def alpha(msq, xi: float):
    """alpha(|m|) = exp(-pi^2 |m|^2 / xi^2) / |m|^2 (Eq. hexpr), 0 at m = 0."""
    msq = np.asarray(msq, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.exp(-math.pi ** 2 * msq / xi ** 2) / msq
    return np.where(msq > 0, a, 0.0)


def apply_exact(Qn, Kc: int, Ln: int, box: float, beta: float, M: int) -> np.ndarray:
    """Phi = (1/(pi L)) A Q with A(g, h) = sum_{0 != m, |m|_inf <= M} alpha(|m|) exp(2 i pi m.(y_g - y_h)),
    through the per-axis exponential matrices (a plain definition, no SKP)."""
    y = node_positions(Kc, Ln)
    m = np.arange(-M, M + 1, dtype=np.float64)
    E = np.exp(2j * np.pi * np.outer(m, y))                   # (2M+1, n)
    Qh = np.einsum("ag,bh,ck,ghk->abc", E.conj(), E.conj(), E.conj(), Qn)
    msq = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    Ph = alpha(msq, beta * box) * Qh
    return np.real(np.einsum("ag,bh,ck,abc->ghk", E, E, E, Ph)) / (math.pi * box)


def sinc_factors(Kc: int, Ln: int, box: float, beta: float, M: int, tol: float):
    """Quadrature SKP of alpha_M (Eq. quaddecompalpham): the sinc rule of 1/|m|^2 searched over
    the arguments |m|^2 of the mode cube (§2.1.2), and the dense axis factors A_l on the nodes.
    Returns (w, A (R, n, n), c_Lambda)."""
    m = np.arange(-M, M + 1, dtype=np.float64)
    msq = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    args = np.unique(msq[msq > 0])
    nq, h, _ = skp.sinc_search(args, tol)
    w, lam = skp.sinc_rule(nq, h)
    y = node_positions(Kc, Ln)
    d = y[:, None] - y[None, :]
    xi2 = (beta * box) ** 2
    a = np.exp(-(lam[:, None] + math.pi ** 2 / xi2) * m[None, :] ** 2)       # (R, 2M+1)
    A = np.einsum("rm,mgh->rgh", a, np.cos(2 * np.pi * m[:, None, None] * d[None, :, :]))
    return w, A, float(np.sum(w))


def apply_skp(Qn, w, A, c: float, box: float) -> np.ndarray:
    """Phi = (1/(pi L)) (sum_l w_l Q x0 A_l x1 A_l x2 A_l - c_Lambda sum Q) (Algorithm 4's loop)."""
    Phi = np.zeros_like(Qn)
    for wl, Al in zip(w, A):
        Phi += wl * skp.kron_apply(Qn, Al, Al, Al)
    return (Phi - c * float(np.sum(Qn))) / (math.pi * box)


def reciprocal(x, q, box: float, beta: float, Kc: int, Ln: int, M: int, method: str = "exact",
               tol: float = 1e-10, center=None) -> dict:
    """Algorithm 4 with one cell per process merged: spread, node operator, gather.
    Returns E, phi, F, the node charges Q and the node potentials Phi."""
    q = np.asarray(q, dtype=np.float64)
    Qn = spread(x, q, box, Kc, Ln, center)
    if method == "exact":
        Phi = apply_exact(Qn, Kc, Ln, box, beta, M)
    else:
        w, A, c = sinc_factors(Kc, Ln, box, beta, M, tol)
        Phi = apply_skp(Qn, w, A, c, box)
    phi, F = gather(x, q, box, Kc, Ln, Phi, center)
    return dict(E=0.5 * float(np.dot(q, phi)), phi=phi, F=F, Q=Qn, Phi=Phi)


def direct(x, q, box: float, beta: float, M: int, center=None) -> dict:
    """The exact reciprocal sum on the mode cube |m|_inf <= M (no interpolation)."""
    return ewald.reciprocal_exact(x, q, box, beta, center=center, mmax=M)
