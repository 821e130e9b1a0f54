"""The 10^6-charge box (220 A, order 6, K = 256, SKP tolerance 1e-7) at full size against the
float64 SKP oracle (Algorithm 4 with the oracle's own two-level SVD at the same tolerance),
the binding comparison: the oracle's factors installed on the GPU isolate the arithmetic
error; the GPU's own SKP build is checked against the same oracle; classical FFT-PME is the
extra reference the SKP approximates to its compression tolerance."""
import numpy as np
import pytest

from oracle import skp, spme
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    s = wl.large()
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    return torch, s, o, ref


def _errors(out, ref):
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(out["energy"].item() - ref["E"]) / abs(ref["E"])
    e_W = abs(out["virial"].item() - ref["W"]) / abs(ref["W"])
    return e_phi, e_f, e_E, e_W


@pytest.mark.parametrize("prec", ["bf16x10", "fp32"])
def test_large_box_oracle_factors(setup, prec):
    torch, s, o, ref = setup
    from paper_2601_18838_gb300 import Plan
    plan = Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)
    plan.set_skp(*skp.generators(o))
    out = plan.energy_forces(dev(torch, s.x), dev(torch, s.q), virial=True)
    e_phi, e_f, e_E, e_W = _errors(out, ref)
    print(f"large {prec} (oracle SKP, R={o.R}): phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e} W {e_W:.2e}")
    assert e_phi < 1e-6 and e_f < 1e-5 and e_E < 1e-6 and e_W < 1e-5
    plan.close()


def test_large_box_gpu_build(setup):
    torch, s, o, ref = setup
    from paper_2601_18838_gb300 import Plan
    plan = Plan(s.box, s.K, s.order, s.beta, precision="bf16x10", skp_tol=s.skp_tol, max_n=s.n)
    R, err = plan.build_skp()
    assert err <= s.skp_tol and R == o.R
    x, q = dev(torch, s.x), dev(torch, s.q)
    out = plan.energy_forces(x, q, virial=True)
    e_phi, e_f, e_E, e_W = _errors(out, ref)
    pme = spme.pme(s.x, s.q, s.box, s.K, s.order, s.beta)
    p_phi = rel(host(out["dEdq"]), pme["phi"])
    print(f"large bf16x10 (GPU SKP, R={R}, err {err:.2e}): vs SKP oracle phi {e_phi:.2e} F {e_f:.2e} "
          f"E {e_E:.2e} W {e_W:.2e} | vs FFT-PME phi {p_phi:.2e}")
    assert e_phi < 1e-6 and e_f < 1e-5 and e_E < 1e-6 and e_W < 1e-5
    assert p_phi < 2e-6
    # charge conservation of the float32 mesh at full size (rounding of K^3 values)
    Q = host(plan.spread(x, q))
    assert abs(Q.sum() - s.q.sum()) < 1e-6 * np.abs(Q).sum()
    plan.close()
