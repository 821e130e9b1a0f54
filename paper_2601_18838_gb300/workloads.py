"""Seeded synthetic point clouds for the reciprocal-space workloads.

This module only draws positions and charges; it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper measures on quasi-uniform synthetic point clouds in a cubic box
(§5.1, §5.2); the five workloads below stand in for those and follow that
recipe:

* ``small``   : N = 1000 charges (+1 x 500, -1 x 500), uniform in a 20 A box,
                order 4, K = 32, SKP tolerance 1e-8.
* ``water``   : 10^4 rigid 3-site molecules (O -0.834, two H +0.417,
                O-H 0.9572 A, H-O-H 104.52 deg) in a 67 A box.  Oxygens sit on a
                jittered 22^3 cubic lattice (10^4 of its sites drawn without
                replacement, jitter uniform +-0.25 A per axis), each molecule has
                a uniformly random orientation (unit quaternion), hydrogens are
                wrapped periodically.  Order 4, K = 64.
* ``mixed``   : N = 10^5 charges, a quarter each of +1, -1, +0.5, -0.5, uniform
                in a 100 A box, order 6, K = 96.
* ``batched`` : 64 independent neutral +-1 systems, N log-uniform in
                [2000, 50000] (rounded to even), box side uniform in [30, 80] A,
                K the smallest of {32, 48, 64, 96} with box/K <= 1.25 A, order 4.
* ``large``   : N = 10^6 charges +-1, uniform in a 220 A box, order 6, K = 256,
                SKP tolerance 1e-7.

Every workload uses the Ewald parameter beta = 0.35 1/A.  Seeds are
2601188380 + workload index with numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

SEED_BASE = 2601188380
BETA = 0.35


@dataclass
class System:
    """One periodic cubic system: positions (N,3) float64 in [0, L), charges (N,) float64."""
    name: str
    x: np.ndarray
    q: np.ndarray
    box: float          # side length L = 2 r_B
    K: int              # mesh points per axis
    order: int          # B-spline order n
    beta: float = BETA
    skp_tol: float = 1e-8
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def center(self):
        return (0.5 * self.box,) * 3

    @property
    def radius(self) -> float:
        return 0.5 * self.box


def _rng(idx: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + idx))


def _pm_charges(rng, n: int, values) -> np.ndarray:
    """Equal counts of each value in ``values`` (n divisible by len(values)), shuffled."""
    k = len(values)
    assert n % k == 0
    q = np.repeat(np.asarray(values, dtype=np.float64), n // k)
    rng.shuffle(q)
    return q


def uniform_system(name: str, idx: int, n: int, box: float, K: int, order: int,
                   values=(1.0, -1.0), skp_tol: float = 1e-8, rng=None) -> System:
    rng = _rng(idx) if rng is None else rng
    x = rng.uniform(0.0, box, size=(n, 3))
    q = _pm_charges(rng, n, values)
    return System(name, x, q, box, K, order, skp_tol=skp_tol)


def small() -> System:
    return uniform_system("small", 0, 1000, 20.0, 32, 4)


def _quat_rotations(rng, m: int) -> np.ndarray:
    """m uniformly distributed rotation matrices from unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random((3, m))
    a = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    w, x, y, z = d, a, b, c
    R = np.empty((m, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water(n_mol: int = 10_000, box: float = 67.0, K: int = 64, order: int = 4,
          lattice: int = 22, jitter: float = 0.25, idx: int = 1) -> System:
    rng = _rng(idx)
    sites = rng.choice(lattice ** 3, size=n_mol, replace=False)
    ijk = np.stack(np.unravel_index(sites, (lattice,) * 3), axis=1).astype(np.float64)
    a = box / lattice
    o = (ijk + 0.5) * a + rng.uniform(-jitter, jitter, size=(n_mol, 3))
    r_oh, ang = 0.9572, np.deg2rad(104.52)
    body = np.array([[r_oh * np.sin(ang / 2), 0.0, r_oh * np.cos(ang / 2)],
                     [-r_oh * np.sin(ang / 2), 0.0, r_oh * np.cos(ang / 2)]])
    R = _quat_rotations(rng, n_mol)
    h = o[:, None, :] + np.einsum("mij,hj->mhi", R, body)
    x = np.concatenate([o[:, None, :], h], axis=1).reshape(-1, 3)
    x = np.mod(x, box)
    x[x >= box] = 0.0
    q = np.tile(np.array([-0.834, 0.417, 0.417]), n_mol)
    return System("water", x, q, box, K, order, meta={"molecules": n_mol})


def mixed(n: int = 100_000) -> System:
    return uniform_system("mixed", 2, n, 100.0, 96, 6, values=(1.0, -1.0, 0.5, -0.5))


def batched(n_sys: int = 64, ks=(32, 48, 64, 96)) -> list[System]:
    rng = _rng(3)
    out = []
    for s in range(n_sys):
        n = int(round(np.exp(rng.uniform(np.log(2000), np.log(50000)))))
        n += n % 2
        box = float(rng.uniform(30.0, 80.0))
        K = next((k for k in ks if box / k <= 1.25), ks[-1])
        out.append(uniform_system(f"batched[{s}]", 3, n, box, K, 4, rng=rng))
    return out


def large(n: int = 1_000_000) -> System:
    return uniform_system("large", 4, n, 220.0, 256, 6, skp_tol=1e-7)


def lagrange(n: int = 20_000) -> System:
    """The per-cell Lagrange form (§4.1): 2e4 charges +-1 in a 30 A box, beta = 0.1/A (xi = 3),
    modes |m|_inf <= 4, 8 cells of 8 equispaced nodes per axis (64 nodes), quadrature SKP 1e-12,
    node operator in mode space."""
    s = uniform_system("lagrange", 5, n, 30.0, 64, 8, skp_tol=1e-12)
    s.beta = 0.1
    s.meta = {"interp": "lagrange_modes", "modes": 4, "cells": 8}
    return s


def by_name(name: str):
    return {"small": small, "water": water, "mixed": mixed, "batched": batched, "large": large,
            "lagrange": lagrange}[name]()


def random_system(n: int, box: float, K: int, order: int, seed: int, beta: float = BETA,
                  skp_tol: float = 1e-8) -> System:
    """Small seeded +-1 system for parity tests at reduced sizes.

    Charges alternate +1, -1 before shuffling, so the system is neutral when n is
    even and carries a net charge of +1 when n is odd.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(0.0, box, size=(n, 3))
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    rng.shuffle(q)
    return System(f"random[{seed}]", x, q, box, K, order, beta=beta, skp_tol=skp_tol)
