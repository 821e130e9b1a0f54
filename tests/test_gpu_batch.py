"""Batched evaluation of independent systems (uneven N, box and K) by one graph launch,
checked system by system against single-plan evaluations and against the float64 SKP oracle
(potentials, forces, energy and virial trace of every non-empty system)."""
import numpy as np
import pytest

from oracle import skp
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu


def _systems():
    specs = [(1200, 31.0, 32), (0, 40.0, 32), (2501, 47.0, 48), (777, 22.0, 32), (4000, 66.0, 64), (1999, 35.0, 32),
             (3001, 52.0, 48)]
    return [wl.random_system(n, L, K, 4, seed=1000 + i) for i, (n, L, K) in enumerate(specs)]


def test_batch_matches_single_plans_and_oracle():
    torch = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    from paper_2601_18838_gb300 import Batch, Plan
    systems = _systems()
    batch = Batch([dict(box=s.box, K=s.K, order=s.order, beta=s.beta, skp_tol=s.skp_tol, max_n=max(s.n, 1))
                   for s in systems])
    ranks = batch.build_skp()
    offsets = np.cumsum([0] + [s.n for s in systems])
    x = dev(torch, np.concatenate([s.x for s in systems]))
    q = dev(torch, np.concatenate([s.q for s in systems]))
    out = batch.energy_forces(x, q, offsets, virial=True)
    again = batch.energy_forces(x, q, offsets, virial=True)   # graph replay
    E, F, P = host(out["energy"]), host(out["forces"]), host(out["dEdq"])
    np.testing.assert_allclose(host(again["energy"]), E, rtol=1e-6)
    for i, s in enumerate(systems):
        a, b = offsets[i], offsets[i + 1]
        if s.n == 0:
            assert E[i] == 0.0
            continue
        plan = Plan(s.box, s.K, s.order, s.beta, precision="bf16x10", skp_tol=s.skp_tol, max_n=s.n)
        R, _ = plan.build_skp()
        assert R == ranks[i]
        ref = plan.energy_forces(dev(torch, s.x), dev(torch, s.q))
        assert abs(E[i] - ref["energy"].item()) < 1e-6 * abs(ref["energy"].item())
        assert rel(P[a:b], host(ref["dEdq"])) < 1e-6
        assert rel(F[a:b], host(ref["forces"])) < 1e-6
    # every non-empty system (K = 32, 48 and 64, even and odd n) against the float64 SKP oracle
    W = host(out["virial"])
    for i, s in enumerate(systems):
        if s.n == 0:
            continue
        a, b = offsets[i], offsets[i + 1]
        o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
        r = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
        e_phi, e_f = rel(P[a:b], r["phi"]), rel(F[a:b], r["F"])
        e_E, e_W = abs(E[i] - r["E"]) / abs(r["E"]), abs(W[i] - r["W"]) / abs(r["W"])
        print(f"batched system {i} (K={s.K}, n={s.n}): phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e} W {e_W:.2e}")
        assert e_phi < 1e-6 and e_f < 1e-5 and e_E < 1e-6 and e_W < 1e-5
