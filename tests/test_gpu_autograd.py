"""Differentiation: the autograd.Function's adjoint (derivative B-splines in the gather)
against central finite differences of the GPU energy and against the oracle's forces."""
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


def _plan(s, prec):
    from paper_2601_18838_gb300 import Plan
    return Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)


def test_autograd_matches_adjoint_and_finite_differences(torch):
    from paper_2601_18838_gb300 import reciprocal_energy
    s = wl.random_system(96, 14.0, 32, 6, seed=31)
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    plan = _plan(s, "fp64")
    plan.set_skp(*skp.generators(o))
    x = dev(torch, s.x).requires_grad_(True)
    q = dev(torch, s.q).requires_grad_(True)
    E = reciprocal_energy(x, q, plan)
    E.backward()
    out = plan.energy_forces(x.detach(), q.detach())
    # a second call sums the charge mesh in another atomic order: equal to rounding
    np.testing.assert_allclose(host(x.grad), -host(out["forces"]), rtol=0, atol=1e-12 * np.abs(host(x.grad)).max())
    np.testing.assert_allclose(host(q.grad), host(out["dEdq"]), rtol=0, atol=1e-12 * np.abs(host(q.grad)).max())
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    assert rel(-host(x.grad), ref["F"]) < 1e-11
    assert abs(E.item() - ref["E"]) < 1e-12 * abs(ref["E"])
    # central differences of the GPU float64 energy, h = 1e-4 A
    h = 1e-4
    for i, a in [(0, 0), (17, 1), (95, 2)]:
        xp, xm = s.x.copy(), s.x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        Ep = plan.energy_forces(dev(torch, xp), dev(torch, s.q))["energy"].item()
        Em = plan.energy_forces(dev(torch, xm), dev(torch, s.q))["energy"].item()
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - x.grad[i, a].item()) < 1e-7 * np.abs(host(x.grad)).max()
    # dE/dq by a central difference is exact for a quadratic energy
    for i in (3, 50):
        qp, qm = s.q.copy(), s.q.copy()
        qp[i] += 0.5
        qm[i] -= 0.5
        fd = (plan.energy_forces(dev(torch, s.x), dev(torch, qp))["energy"].item()
              - plan.energy_forces(dev(torch, s.x), dev(torch, qm))["energy"].item())
        assert abs(fd - q.grad[i].item()) < 1e-11 * max(1.0, abs(fd))


def test_mixed_charges_forces_tensor_path(torch):
    # 10^5 charges (+-1, +-0.5), 100 A box, order 6, K = 96: forces through the adjoint
    # of the error-free split path against the float64 oracle
    from paper_2601_18838_gb300 import reciprocal_energy
    s = wl.mixed()
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    plan = _plan(s, "bf16x10")
    plan.set_skp(*skp.generators(o))
    x = dev(torch, s.x).requires_grad_(True)
    q = dev(torch, s.q).requires_grad_(True)
    E = reciprocal_energy(x, q, plan)
    E.backward()
    e_f, e_phi = rel(-host(x.grad), ref["F"]), rel(host(q.grad), ref["phi"])
    print(f"mixed bf16x10: F {e_f:.2e} phi {e_phi:.2e} E {abs(E.item() - ref['E']) / abs(ref['E']):.2e}")
    assert e_f < 1e-5 and e_phi < 1e-6


@pytest.mark.parametrize("method", ["svd", "sinc"])
def test_potential_autograd_matches_oracle(torch, method):
    # p = potentials at targets x of charges q at sources y (§1.1); L = sum(g p)
    from oracle import spme
    from paper_2601_18838_gb300 import Plan, reciprocal_potential
    s = wl.random_system(96, 14.0, 32, 6, seed=41)
    rng = np.random.default_rng(5)
    xt = rng.uniform(-2.0, 16.0, (40, 3))
    g = rng.normal(size=40)
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol, method=method)
    plan = Plan(s.box, s.K, s.order, s.beta, precision="fp64", skp_tol=s.skp_tol, max_n=s.n, skp_method=method)
    if method == "svd":
        plan.set_skp(*skp.generators(o))
    else:
        plan.build_skp()
    y = dev(torch, s.x).requires_grad_(True)
    q = dev(torch, s.q).requires_grad_(True)
    x = dev(torch, xt).requires_grad_(True)
    p = reciprocal_potential(y, q, x, plan)
    (p * dev(torch, g)).sum().backward()

    def pot(ys, qs, xs):
        Phi = skp.apply(spme.spread(ys, qs, s.box, s.K, s.order), o)
        return spme.gather(xs, np.zeros(len(xs)), s.box, s.K, s.order, Phi)[0]

    assert rel(host(p), pot(s.x, s.q, xt)) < 1e-11
    # dL/dq: the adjoint problem (charges g at the targets, potentials at the sources)
    assert rel(host(q.grad), pot(xt, g, s.x)) < 1e-11
    # dL/dx and dL/dy: central differences of the float64 oracle, h = 1e-4 A
    h = 1e-4
    L0 = lambda ys, xs: float(np.dot(g, pot(ys, s.q, xs)))
    gx, gy = host(x.grad), host(y.grad)
    for i, a in [(0, 0), (21, 1), (39, 2)]:
        xp, xm = xt.copy(), xt.copy()
        xp[i, a] += h
        xm[i, a] -= h
        fd = (L0(s.x, xp) - L0(s.x, xm)) / (2 * h)
        assert abs(fd - gx[i, a]) < 1e-7 * np.abs(gx).max()
    for j, a in [(2, 0), (50, 2), (95, 1)]:
        yp, ym = s.x.copy(), s.x.copy()
        yp[j, a] += h
        ym[j, a] -= h
        fd = (L0(yp, xt) - L0(ym, xt)) / (2 * h)
        assert abs(fd - gy[j, a]) < 1e-7 * np.abs(gy).max()
