"""Error paths under host-side fault injection (KPME_FAULT, read when a plan is made).  Nothing
here makes the GPU fault: allocations fail on the host, the plan handle is spoiled on the host,
the device status word is raised from the host, and the shortened wait budget makes the
kernels' bounded waits give up, after which they let their copies and MMAs in flight complete,
release tensor memory and return (the context stays usable)."""
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


def _plan(s, prec="bf16x10"):
    from paper_2601_18838_gb300 import Plan
    return Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)


def _healthy(torch, s):
    # a plan made without faults works afterwards and matches the oracle
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol)
    p = _plan(s)
    p.build_skp()
    out = p.energy_forces(dev(torch, s.x), dev(torch, s.q))
    assert rel(host(out["dEdq"]), ref["phi"]) < 1e-6
    p.close()


def test_allocation_failure_reports_oom(torch, monkeypatch):
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(500, 16.0, 32, 4, seed=3)
    monkeypatch.setenv("KPME_FAULT", "alloc")
    with pytest.raises(KpmeError, match="out of device memory"):
        _plan(s)
    # a later allocation: the plan is made, its SKP installation fails
    hit = False
    for n in (8, 12, 16, 24):
        monkeypatch.setenv("KPME_FAULT", f"alloc:{n}")
        try:
            p = _plan(s)
        except KpmeError as e:
            assert "out of device memory" in str(e)
            continue
        try:
            p.build_skp()
        except KpmeError as e:
            assert "out of device memory" in str(e)
            hit = True
        p.close()
    assert hit
    monkeypatch.delenv("KPME_FAULT")
    _healthy(torch, s)


def test_corrupted_plan_handle_is_rejected(torch, monkeypatch):
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(500, 16.0, 32, 4, seed=4)
    monkeypatch.setenv("KPME_FAULT", "plan")
    p = _plan(s)
    with pytest.raises(KpmeError, match="invalid argument.*corrupted plan handle"):
        p.build_skp()
    with pytest.raises(KpmeError, match="invalid argument"):
        p.energy_forces(dev(torch, s.x), dev(torch, s.q))
    p.close()
    monkeypatch.delenv("KPME_FAULT")
    _healthy(torch, s)


def test_raised_status_word_reports_timeout_once(torch, monkeypatch):
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(500, 16.0, 32, 4, seed=5)
    monkeypatch.setenv("KPME_FAULT", "timeout")
    p = _plan(s)
    monkeypatch.delenv("KPME_FAULT")
    with pytest.raises(KpmeError, match="timed out"):
        p.build_skp()          # the build ran; the raised word is reported at its end
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol)
    out = p.energy_forces(dev(torch, s.x), dev(torch, s.q))
    assert rel(host(out["dEdq"]), ref["phi"]) < 1e-6
    p.close()


@pytest.mark.parametrize("K,L", [(64, 40.0), (128, 80.0)])
def test_device_waits_give_up_and_the_plan_recovers(torch, monkeypatch, K, L):
    # K = 64: stage 1 and the fused stages 2-3; K = 128: all three stages with A in tensor memory
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(2001, L, K, 4, seed=K)
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    monkeypatch.setenv("KPME_FAULT", "budget:1")
    p = _plan(s)
    monkeypatch.delenv("KPME_FAULT")
    p.set_skp(*skp.generators(o))
    x, q = dev(torch, s.x), dev(torch, s.q)
    p.energy_forces(x, q)                      # the kernels give up on the device
    torch.cuda.synchronize()                   # ... and return: the stream completes
    with pytest.raises(KpmeError, match="timed out"):
        p.energy_forces(x, q)                  # reported by the next call
    out = p.energy_forces(x, q)                # the production budget again
    assert rel(host(out["dEdq"]), ref["phi"]) < 1e-6 and rel(host(out["forces"]), ref["F"]) < 1e-5
    p.close()
    _healthy(torch, wl.random_system(500, 16.0, 32, 4, seed=6))
