"""The paper's Sum-of-Kronecker-Products mesh operator (oracle; test infrastructure).

§2.1 approximates the vector of nodal values of the reciprocal influence
function on the full mode grid by a SKP; §2.3 turns each Kronecker factor into
a real operator (the cos/sin pairs of Eq. (kronw) combine, for an even factor,
into a real symmetric circulant); §2.4, Eq. (VtV) assembles
sum_lambda A^(0)(lambda) (x) A^(1)(lambda) (x) A^(2)(lambda); §3.3, Algorithm 2
applies each term as three reshaped matrix products.

With B-spline interpolation on a K^3 mesh the influence tensor is
T(m) = B(m) C(m) (oracle.spme.influence) on m in [-K/2, K/2)^3, T(0) = 0
(§2.1 and the remark after Fig. 1: zero at the unused m = 0 mode).

Index readings (the paper's are loose): I_2 matricises with rows on axis 2
(m_3), so the outer SVD's left vectors u_i are the axis-2 factors; I_1 of each
v_i puts axis 1 (m_2) on the rows, so u_ij is the axis-1 factor and v_ij the
axis-0 factor.  T is symmetric under axis permutations, so this only fixes
which mode each factor multiplies.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import spme, bspline


@dataclass
class SKP:
    """sum_r w_r a0_r (x) a1_r (x) a2_r on the FFT-ordered mode grid, minus c delta_0.

    ``outer`` / ``inner`` hold the singular values of the two SVD levels (NKPA);
    ``r1[i]`` is the number of inner terms kept for outer term i; terms are ordered
    i-major.  ``c`` is the m = 0 correction constant (0 for NKPA, c_Lambda for the
    quadrature variant)."""
    K: int
    w: np.ndarray                 # (R,)
    a0: np.ndarray                # (R, K) axis-0 factors (mode space)
    a1: np.ndarray                # (R, K)
    a2: np.ndarray                # (R, K)
    c: float = 0.0
    r1: list = field(default_factory=list)
    outer: np.ndarray | None = None
    inner: list = field(default_factory=list)
    bound: float = 0.0            # right-hand side of Eq. (estimate_svd)
    norm: float = 0.0             # ||T||_F

    @property
    def R(self) -> int:
        return int(self.w.size)

    def tensor(self) -> np.ndarray:
        """The approximated tensor sum_r w_r a0 (x) a1 (x) a2 - c delta_0."""
        T = np.einsum("r,ri,rj,rk->ijk", self.w, self.a0, self.a1, self.a2)
        T[0, 0, 0] -= self.c
        return T


def _tail(s: np.ndarray) -> np.ndarray:
    """tail[r] = sqrt(sum_{k >= r} s_k^2), with tail[len(s)] = 0."""
    t = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    return np.append(t, 0.0)


def nkpa(T: np.ndarray, tol: float) -> SKP:
    """Nearest Kronecker Product Approximation by recursive truncated SVD (§2.1.1).

    I_2(T) = U Sigma V^T (Eq. after (pb_skp)), then I_1(v_i) = U_i Sigma_i V_i^T
    (Eq. last_decomp_kron), giving T ~ sum_{i,j} s_i s_ij u_i (x) u_ij (x) v_ij.
    Ranks are chosen so that the right-hand side of Eq. (estimate_svd),
      sqrt(sum_{i>r0} s_i^2) + sum_{i<=r0} s_i sqrt(sum_{j>r1_i} s_ij^2),
    is at most tol * ||T||_F: the outer tail takes at most half of the budget
    and the rest is shared evenly by the r0 inner truncations (the inner
    tolerances are therefore smaller than the outer one, as the paper notes)."""
    K = T.shape[0]
    nrm = float(np.linalg.norm(T))
    A = T.reshape(K * K, K).T                      # I_2: rows m_3, columns (m_1, m_2)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    out_tail = _tail(s)
    budget = tol * nrm
    r0 = int(np.argmax(out_tail <= 0.5 * budget))
    if tol == 0.0:
        r0 = s.size
    inner_budget = budget - out_tail[r0]
    w, a0, a1, a2, r1s, inner = [], [], [], [], [], []
    bound = out_tail[r0]
    for i in range(r0):
        Vi = Vt[i].reshape(K, K).T                 # I_1(v_i): rows m_2, columns m_1
        Ui, si, Wti = np.linalg.svd(Vi)
        in_tail = _tail(si)
        if tol == 0.0:
            r1 = si.size
        else:
            thr = inner_budget / (r0 * s[i]) if s[i] > 0 else np.inf
            r1 = int(np.argmax(in_tail <= thr))
        bound += s[i] * in_tail[r1]
        r1s.append(r1)
        inner.append(si)
        for j in range(r1):
            w.append(s[i] * si[j])
            a0.append(Wti[j])                      # v_ij: axis 0
            a1.append(Ui[:, j])                    # u_ij: axis 1
            a2.append(U[:, i])                     # u_i : axis 2
    return SKP(K, np.asarray(w), np.asarray(a0).reshape(-1, K), np.asarray(a1).reshape(-1, K),
               np.asarray(a2).reshape(-1, K), 0.0, r1s, s, inner, float(bound), nrm)


def sinc_rule(n_quad: int, h: float):
    """Cardinal-sine quadrature of 1/R = int_0^inf exp(-tR) dt (§2.1.2):
    w_l = h / (1 + exp(-l h)), lambda_l = log(1 + exp(l h)), l = -N..N."""
    l = np.arange(-n_quad, n_quad + 1, dtype=np.float64)
    return h / (1.0 + np.exp(-l * h)), np.log1p(np.exp(l * h))


def sinc_search(args: np.ndarray, tol: float, n_max: int = 400, n_h: int = 64):
    """Smallest N_quad (and its best h) whose max relative error of
    sum_l w_l exp(-lambda_l R) against 1/R over the given arguments is <= tol.

    h is searched by brute force on a grid around pi / sqrt(2 N + 1) (§2.1.2)."""
    args = np.asarray(args, dtype=np.float64)
    for nq in range(1, n_max + 1):
        h0 = math.pi / math.sqrt(2 * nq + 1)
        best = (np.inf, h0)
        for h in h0 * np.linspace(0.5, 2.0, n_h):
            w, lam = sinc_rule(nq, h)
            approx = np.exp(-np.outer(args, lam)) @ w
            err = float(np.max(np.abs(approx * args - 1.0)))
            if err < best[0]:
                best = (err, h)
        if best[0] <= tol:
            return nq, best[1], best[0]
    raise ValueError("sinc quadrature did not reach the tolerance")


def sinc_skp(K: int, n: int, box: float, beta: float, tol: float) -> SKP:
    """Quadrature-based SKP of Eq. (quaddecompalpham) with the B-spline factor.

    T(m) = (L^2/(pi V)) B(m) exp(-pi^2 |m|^2/(beta L)^2) / |m|^2 and
    1/|m|^2 ~ sum_l w_l exp(-lambda_l |m|^2) give rank-one terms with the same
    factor a_l(m) = |b(m)|^2 exp(-(lambda_l + pi^2/(beta L)^2) m^2) on every axis,
    minus c_Lambda delta_0 with c_Lambda = (L^2/(pi V)) B(0) sum_l w_l."""
    m = spme.wrapped_modes(K).astype(np.float64)
    msq = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    args = np.unique(msq[msq > 0])
    nq, h, _ = sinc_search(args, tol)
    w, lam = sinc_rule(nq, h)
    bm = bspline.moduli_sq(K, n)
    pre = box ** 2 / (math.pi * box ** 3)
    xi2 = (beta * box) ** 2
    a = bm[None, :] * np.exp(-(lam[:, None] + math.pi ** 2 / xi2) * m[None, :] ** 2)
    c = pre * bm[0] ** 3 * float(np.sum(w))
    return SKP(K, pre * w, a.copy(), a.copy(), a.copy(), c)


def circulant(a: np.ndarray) -> np.ndarray:
    """Real circulant A(k, k') = g(k - k' mod K), g(d) = Re sum_m a(m) exp(2 i pi m d / K).

    For an even mode vector a this is the real symmetric operator that §2.3's
    cos/sin factorisation (Eqs. abelian_to_cos, kronw) produces."""
    K = a.size
    d = np.arange(K)
    g = np.real(np.exp(2j * np.pi * np.outer(d, np.arange(K)) / K) @ a)
    idx = (d[:, None] - d[None, :]) % K
    return g[idx]


def mode_product(X: np.ndarray, A: np.ndarray, axis: int) -> np.ndarray:
    """One step of Algorithm 2: reshape with rows on ``axis`` (I_p), multiply by A,
    reshape back (I_p^bullet)."""
    Xm = np.moveaxis(X, axis, 0)
    shp = Xm.shape
    Y = A @ Xm.reshape(shp[0], -1)
    return np.moveaxis(Y.reshape(shp), 0, axis)


def kron_apply(Q: np.ndarray, A0, A1, A2) -> np.ndarray:
    """(A0 (x) A1 (x) A2) vec(Q) by Algorithm 2: modes d-1, ..., 0 in turn."""
    Y = mode_product(Q, A2, 2)
    Y = mode_product(Y, A1, 1)
    return mode_product(Y, A0, 0)


def apply(Q: np.ndarray, skp: SKP) -> np.ndarray:
    """Phi = sum_r w_r Q x_0 A0_r x_1 A1_r x_2 A2_r - c sum(Q), the SKP mesh operator
    (Thm. 1 / Eq. formfinale with the correction term of Eq. termbonsum)."""
    Phi = np.zeros_like(Q)
    for r in range(skp.R):
        Phi += skp.w[r] * kron_apply(Q, circulant(skp.a0[r]), circulant(skp.a1[r]),
                                     circulant(skp.a2[r]))
    if skp.c != 0.0:
        Phi -= skp.c * float(np.sum(Q))
    return Phi


def build(K: int, n: int, box: float, beta: float, tol: float, method: str = "svd") -> SKP:
    if method == "svd":
        return nkpa(spme.influence(K, n, box, beta), tol)
    if method == "sinc":
        return sinc_skp(K, n, box, beta, tol)
    raise ValueError(method)


def reciprocal(x, q, box: float, K: int, n: int, beta: float, tol: float,
               method: str = "svd", skp: SKP | None = None, center=None) -> dict:
    """KPME reciprocal result (Algorithm 4 on one cell): spread, SKP operator,
    gather, then the correction term.  Returns E, phi, F, W and the meshes."""
    q = np.asarray(q, dtype=np.float64)
    if skp is None:
        skp = build(K, n, box, beta, tol, method)
    Q = spme.spread(x, q, box, K, n, center)
    Phi = apply(Q, skp)
    phi, F = spme.gather(x, q, box, K, n, Phi, center)
    E = 0.5 * float(np.dot(q, phi))
    W = spme.virial_trace(Q, E, K, n, box, beta)
    return dict(E=E, phi=phi, F=F, W=W, Q=Q, Phi=Phi, skp=skp)


def generator(a: np.ndarray) -> np.ndarray:
    """Real circulant generator g(d) = Re sum_m a(m) exp(2 i pi m d / K), d = 0..K-1."""
    K = a.size
    d = np.arange(K)
    return np.real(np.exp(2j * np.pi * np.outer(d, np.arange(K)) / K) @ a)


def generators(s: SKP):
    """Two-level generator form of an NKPA SKP: (r1, gen_axis2 per outer term (weight s_i),
    gen_axis1 per term (weight s_ij), gen_axis0 per term), as consumed by kpme_set_skp."""
    if not s.r1:
        raise ValueError("generators() needs the two-level (NKPA) structure")
    gen3, gen2, gen1 = [], [], []
    t = 0
    for i, r1 in enumerate(s.r1):
        gen3.append(s.outer[i] * generator(s.a2[t]))
        for j in range(r1):
            gen2.append(s.inner[i][j] * generator(s.a1[t]))
            gen1.append(generator(s.a0[t]))
            t += 1
    return np.asarray(s.r1, dtype=np.int32), np.asarray(gen3), np.asarray(gen2), np.asarray(gen1)
