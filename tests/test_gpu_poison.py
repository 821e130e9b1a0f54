"""No kernel reads plan scratch it has not written: with KPME_POISON=1 every device allocation
of a plan starts as 0xFF bytes (NaN in floats, -1 in integers), and every path must still match
the float64 oracle at its bar."""
import numpy as np
import pytest

from oracle import skp
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    return t


@pytest.mark.parametrize("K,n,L,prec,tile,fused", [
    (32, 1001, 18.0, "fp64", 0, 1),       # float64 form, cell-sorted spreading
    (32, 1001, 18.0, "bf16x10", 0, 1),    # fused stages 2-3, cell-sorted particles
    (64, 3001, 40.0, "bf16x10", -1, 0),   # tensor-memory A per stage, no cell sort
    (48, 2050, 30.0, "bf16x10", -1, 1),   # shared-memory A kernel (digit planes)
    (128, 5003, 90.0, "bf16x10", 0, 1),   # reflection basis, tile-staged particles
    (64, 3001, 40.0, "fp32", -1, 1),      # CUDA-core float32 stages
])
def test_poisoned_scratch_does_not_change_results(torch, monkeypatch, K, n, L, prec, tile, fused):
    monkeypatch.setenv("KPME_POISON", "1")
    from paper_2601_18838_gb300 import Plan
    s = wl.random_system(n, L, K, 4, seed=K + n + 3)
    plan = Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    plan.set_skp(*skp.generators(o))
    plan.set_tune(tile, fused, 2)   # tile 0 keeps the plan's cell-sorted default
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    for _ in range(2):   # the second call replays the captured graph on the same scratch
        out = plan.energy_forces(dev(torch, s.x), dev(torch, s.q), virial=True)
        e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
        e_W = abs(out["virial"].item() - ref["W"]) / abs(ref["W"])
        bar = 1e-12 if prec == "fp64" else 2e-6
        assert np.isfinite(e_phi) and e_phi < bar and e_f < 10 * bar and e_W < 10 * bar, (e_phi, e_f, e_W)
    plan.close()


def test_poisoned_batch(torch, monkeypatch):
    monkeypatch.setenv("KPME_POISON", "1")
    from paper_2601_18838_gb300 import Batch
    systems = [wl.random_system(1200, 31.0, 32, 4, seed=41), wl.random_system(2501, 47.0, 48, 4, seed=42)]
    batch = Batch([dict(box=s.box, K=s.K, order=s.order, beta=s.beta, skp_tol=s.skp_tol, max_n=s.n)
                   for s in systems])
    batch.build_skp()
    offsets = np.cumsum([0] + [s.n for s in systems])
    x = dev(torch, np.concatenate([s.x for s in systems]))
    q = dev(torch, np.concatenate([s.q for s in systems]))
    out = batch.energy_forces(x, q, offsets, virial=True)
    P = host(out["dEdq"])
    for i, s in enumerate(systems):
        o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
        r = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
        assert rel(P[offsets[i]:offsets[i + 1]], r["phi"]) < 1e-6
    batch.close()
