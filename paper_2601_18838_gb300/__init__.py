"""GB300-native reciprocal-space Kroneckerised Particle Mesh Ewald.

The compute path is the CUDA library ``libkpme.so`` (C ABI in ``include/kpme.h``);
this package is its thin Python binding:

* ``Plan``                 one periodic problem (box, mesh K, B-spline order, beta,
                           SKP factors, arithmetic) — ``kpme_plan`` and friends.
* ``reciprocal_energy``    differentiable energy (torch.autograd.Function).
* ``reciprocal_potential`` differentiable potentials at targets x of sources (y, q).
* ``workloads``            seeded synthetic point clouds.
"""
from ._binding import Plan, Batch, KpmeError, PRECISIONS, EXPORTS, lib  # noqa: F401
from .autograd import reciprocal_energy, reciprocal_potential  # noqa: F401
