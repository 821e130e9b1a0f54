"""The oracle's full Ewald energy (tin-foil boundary) against brute force: the direct Coulomb sum
over every periodic image of a few charges, taken over all cells within a sphere of R box lengths
with the surface term of a spherical sample in vacuum, (2 pi / 3V) |sum_i q_i r_i|^2 (de Leeuw,
Perram and Smith), removed.  Nothing of the Ewald splitting enters the brute-force side, so this
pins the oracle's reciprocal normalisation, self term and background term at once."""
import numpy as np
import pytest

from oracle import ewald


def _sphere_sum(x, q, L, R):
    """1/2 sum_{i,j} sum_{|n| <= R, (i,n) != (j,0)} q_i q_j / |x_i - x_j + n L| (float64)."""
    r = np.arange(-R, R + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n = n[(n * n).sum(1) <= R * R]
    d = x[:, None, :] - x[None, :, :]
    qq = q[:, None] * q[None, :]
    idx = np.arange(len(q))
    E = 0.0
    for c in np.array_split(n, max(1, len(n) // 20000)):
        v = d[None] + L * c[:, None, None, :]
        rr = np.sqrt((v * v).sum(-1))
        for z in np.nonzero((c == 0).all(1))[0]:
            rr[z, idx, idx] = np.inf
        E += 0.5 * float((qq[None] / rr).sum())
    return E


@pytest.mark.parametrize("seed,L,q", [
    (3, 5.0, [1.0, -1.0, 0.5, -0.5, 0.75, -0.75]),
    (8, 7.5, [1.0, 1.0, -1.0, -1.0, 0.5, -0.25, -0.5, 0.25]),
])
def test_full_ewald_equals_spherical_lattice_sum(seed, L, q):
    rng = np.random.default_rng(seed)
    q = np.array(q)
    x = rng.uniform(0.0, L, (len(q), 3))
    E_ewald = ewald.total_energy(x, q, L, 6.0 / L)
    D = (q[:, None] * x).sum(0)
    surface = 2.0 * np.pi / (3.0 * L ** 3) * float(D @ D)
    E_sphere = _sphere_sum(x, q, L, 64)
    # the truncated spherical sums approach the limit like R^-3 (2.4e-9 at R = 64 for the first
    # configuration); a wrong normalisation, self or background term is off by O(1)
    assert abs(E_sphere - surface - E_ewald) <= 1e-8 * abs(E_ewald)
    assert abs(_sphere_sum(x, q, L, 16) - surface - E_ewald) > abs(E_sphere - surface - E_ewald)
