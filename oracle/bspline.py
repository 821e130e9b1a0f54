"""Cardinal B-splines for particle-mesh interpolation (oracle; test infrastructure).

The paper names B-splines as the alternative particle-to-grid interpolation in
§2.2 (it cites smooth PME for them) and then works with Lagrange polynomials;
the reciprocal path here uses the B-spline option.  Definitions are the
textbook ones of smooth PME:

  M_1(u) = 1  on [0, 1),  0 elsewhere
  M_2(u) = 1 - |u - 1|  on [0, 2],  0 elsewhere
  M_n(u) = ( u M_{n-1}(u) + (n - u) M_{n-1}(u - 1) ) / (n - 1)
  M_n'(u) = M_{n-1}(u) - M_{n-1}(u - 1)
  b(m)   = exp(2 pi i (n-1) m / K) / sum_{j=0}^{n-2} M_n(j+1) exp(2 pi i m j / K)
"""
from __future__ import annotations

import numpy as np


def M(n: int, u):
    """Cardinal B-spline of order n evaluated at u (any shape), by the recursion."""
    u = np.asarray(u, dtype=np.float64)
    if n < 1:
        raise ValueError("order must be >= 1")
    if n == 1:
        return np.where((u >= 0.0) & (u < 1.0), 1.0, 0.0)
    if n == 2:
        return np.where((u >= 0.0) & (u <= 2.0), 1.0 - np.abs(u - 1.0), 0.0)
    return (u * M(n - 1, u) + (n - u) * M(n - 1, u - 1.0)) / (n - 1)


def dM(n: int, u):
    """Derivative dM_n/du = M_{n-1}(u) - M_{n-1}(u-1)."""
    return M(n - 1, u) - M(n - 1, np.asarray(u, dtype=np.float64) - 1.0)


def weights(n: int, f):
    """Weights of the n mesh points a particle touches along one axis.

    With u = g + f (g = floor(u), 0 <= f < 1) the point g - j (j = 0..n-1) gets
    M_n(f + j); returns (w, dw) with shape f.shape + (n,).
    """
    f = np.asarray(f, dtype=np.float64)[..., None]
    j = np.arange(n, dtype=np.float64)
    return M(n, f + j), dM(n, f + j)


def moduli_sq(K: int, n: int) -> np.ndarray:
    """|b(m)|^2 for m = 0..K-1 (FFT order), from the definition of b(m)."""
    m = np.arange(K, dtype=np.float64)
    j = np.arange(n - 1, dtype=np.float64)
    den = (M(n, j + 1.0)[None, :] * np.exp(2j * np.pi * np.outer(m, j) / K)).sum(axis=1)
    return 1.0 / np.abs(den) ** 2
