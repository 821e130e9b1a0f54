"""The 10^6-charge box (220 A, order 6, K = 256, SKP tolerance 1e-7) at full size: the GPU
builds its own SKP and the result is compared with the oracle's classical FFT-PME (the SKP
approximates it to the compression tolerance), plus size-independent invariants."""
import numpy as np
import pytest

from oracle import spme
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu


def test_large_box_against_fft_pme():
    torch = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    from paper_2601_18838_gb300 import Plan
    s = wl.large()
    plan = Plan(s.box, s.K, s.order, s.beta, precision="bf16x10", skp_tol=s.skp_tol, max_n=s.n)
    R, err = plan.build_skp()
    assert err <= s.skp_tol
    x, q = dev(torch, s.x), dev(torch, s.q)
    out = plan.energy_forces(x, q, virial=True)
    ref = spme.pme(s.x, s.q, s.box, s.K, s.order, s.beta)
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(out["energy"].item() - ref["E"]) / abs(ref["E"])
    e_W = abs(out["virial"].item() - ref["W"]) / abs(ref["W"])
    print(f"large: R={R} skp err {err:.2e} | vs FFT-PME phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e} W {e_W:.2e}")
    assert e_phi < 2e-6 and e_f < 1e-5 and e_E < 2e-6 and e_W < 2e-6
    # charge conservation of the float32 mesh at full size (rounding of K^3 values)
    Q = host(plan.spread(x, q))
    assert abs(Q.sum() - s.q.sum()) < 1e-6 * np.abs(Q).sum()
