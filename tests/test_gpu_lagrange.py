"""The per-cell Lagrange form of KPME on the GPU (KPME_INTERP_LAGRANGE) against the oracle:
node charges and gathering, the quadrature SKP over the mode cube, and energies / potentials /
forces, against the oracle's exact node operator and the direct sum on the same modes."""
import numpy as np
import pytest

from oracle import lagrange as lg
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu

L_BOX, BETA, M = 20.0, 0.15, 4


@pytest.fixture(scope="module")
def torch():
    t = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    return t


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L_BOX, (n, 3))
    q = rng.choice([-1.0, 1.0], n)
    return x, q - q.mean()


def _plan(prec, Kc, Ln, max_n, tol=1e-12):
    from paper_2601_18838_gb300 import Plan
    return Plan(L_BOX, Kc * Ln, Ln, BETA, precision=prec, skp_tol=tol, skp_method="sinc", max_n=max_n,
                interp="lagrange", modes=M)


@pytest.mark.parametrize("Kc,Ln", [(4, 16), (8, 8), (16, 4), (6, 12)])
def test_lagrange_spread_and_gather_match_oracle(torch, Kc, Ln):
    x, q = _cloud(301, Kc)
    plan = _plan("fp64", Kc, Ln, 301)
    Q = host(plan.spread(dev(torch, x), dev(torch, q)))
    Qr = lg.spread(x, q, L_BOX, Kc, Ln)
    assert np.abs(Q - Qr).max() <= 1e-12 * np.abs(Qr).max()
    rng = np.random.default_rng(1)
    Phi = rng.standard_normal(Q.shape)
    phi, F = plan.gather(dev(torch, x), dev(torch, q), dev(torch, Phi))
    phi_r, F_r = lg.gather(x, q, L_BOX, Kc, Ln, Phi)
    assert rel(host(phi), phi_r) < 1e-12 and rel(host(F), F_r) < 1e-12


@pytest.mark.parametrize("prec,Kc,Ln", [("fp64", 4, 16), ("fp64", 8, 8), ("fp64", 6, 12), ("fp32", 8, 8),
                                         ("fp32", 16, 4)])
def test_lagrange_crowded_boundary_and_empty_cells(torch, prec, Kc, Ln):
    """One cell holding several chunks of particles, particles on cell corners (the upper cell owns
    them, decided in float64 alike on both sides), and mostly empty cells."""
    rng = np.random.default_rng(11)
    h = L_BOX / Kc
    crowd = rng.uniform(0.0, h, (150, 3)) + h * np.array([1.0, 2.0, 0.0])
    corners = np.repeat(h * np.arange(Kc, dtype=np.float64)[:, None], 3, axis=1)
    x = np.vstack([crowd, corners, rng.uniform(0.0, L_BOX, (20, 3))])
    q = rng.choice([-1.0, 1.0], len(x))
    plan = _plan(prec, Kc, Ln, len(x))
    tol = 1e-12 if prec == "fp64" else 1e-4
    Q = host(plan.spread(dev(torch, x), dev(torch, q)))
    Qr = lg.spread(x, q, L_BOX, Kc, Ln)
    assert np.abs(Q - Qr).max() <= tol * np.abs(Qr).max()
    Phi = rng.standard_normal(Q.shape)
    phi, F = plan.gather(dev(torch, x), dev(torch, q), dev(torch, Phi))
    phi_r, F_r = lg.gather(x, q, L_BOX, Kc, Ln, Phi)
    assert rel(host(phi), phi_r) < tol and rel(host(F), F_r) < tol


# Equispaced nodes: at Ln = 16 the weights reach ~1e3 with cancelling signs (the Lebesgue
# constant), which float32 node charges do not survive; the float forms are used with Ln <= 8
# and the FP64 form carries the high orders (the paper's "relatively small orders" in double).
@pytest.mark.parametrize("prec,Kc,Ln,tol,tol_f", [("fp64", 4, 16, 3e-9, 1e-7), ("fp64", 8, 8, 1e-12, 1e-11),
                                                 ("fp32", 8, 8, 5e-5, 2e-4), ("fp32", 16, 4, 2e-5, 1e-4),
                                                 ("bf16x10", 8, 8, 5e-6, 5e-5), ("bf16x10", 16, 4, 2e-6, 2e-5)])
def test_lagrange_energy_forces_match_oracle(torch, prec, Kc, Ln, tol, tol_f):
    x, q = _cloud(500, 7)
    plan = _plan(prec, Kc, Ln, 500)
    R, err = plan.build_skp()
    assert R > 0 and err <= 1e-12
    out = plan.energy_forces(dev(torch, x), dev(torch, q))
    ref = lg.reciprocal(x, q, L_BOX, BETA, Kc, Ln, M)            # exact node operator
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(out["energy"].item() - ref["E"]) / abs(ref["E"])
    print(f"lagrange {prec} Kc={Kc} Ln={Ln}: R={R} phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e}")
    assert e_phi < tol and e_f < tol_f and e_E < tol
    if prec == "fp64":
        # and the interpolation error against the direct sum on the same modes (Thm. 3)
        d = lg.direct(x, q, L_BOX, BETA, M)
        assert rel(host(out["dEdq"]), d["phi"]) < (1e-8 if Ln >= 12 else 1e-6)


def test_lagrange_non_neutral_charges_use_the_correction(torch):
    x, q = _cloud(200, 3)
    q = q + 0.25
    plan = _plan("fp64", 4, 16, 200)
    plan.build_skp()
    out = plan.energy_forces(dev(torch, x), dev(torch, q))
    ref = lg.reciprocal(x, q, L_BOX, BETA, 4, 16, M)
    assert rel(host(out["dEdq"]), ref["phi"]) < 1e-9
    assert plan.skp_c() > 0


def test_lagrange_rejects_what_it_does_not_support(torch):
    from paper_2601_18838_gb300._binding import KpmeError
    x, q = _cloud(50, 5)
    plan = _plan("fp64", 4, 16, 50)
    plan.build_skp()
    with pytest.raises(KpmeError):
        plan.energy_forces(dev(torch, x), dev(torch, q), virial=True)
    with pytest.raises(KpmeError):
        plan.virial_tensor(dev(torch, x), dev(torch, q))
    with pytest.raises(KpmeError):   # the B-spline form's parameters are checked as before
        from paper_2601_18838_gb300 import Plan
        Plan(L_BOX, 64, 16, BETA, precision="fp64", skp_method="svd", interp="lagrange", modes=M)


def test_lagrange_autotune_keeps_results(torch):
    """The autotuner times Lagrange plans without a virial and keeps the results unchanged."""
    x, q = _cloud(2000, 9)
    plan = _plan("bf16x10", 8, 8, 2000)
    plan.build_skp()
    xd, qd = dev(torch, x), dev(torch, q)
    t = plan.autotune(xd, qd)
    assert t["ms_per_eval"] > 0
    out = plan.energy_forces(xd, qd)
    ref = lg.reciprocal(x, q, L_BOX, BETA, 8, 8, M)
    assert rel(host(out["dEdq"]), ref["phi"]) < 2e-5 and rel(host(out["forces"]), ref["F"]) < 1e-4


def _plan_modes(prec, Kc, Ln, max_n, tol=1e-12):
    from paper_2601_18838_gb300 import Plan
    return Plan(L_BOX, Kc * Ln, Ln, BETA, precision=prec, skp_tol=tol, skp_method="sinc", max_n=max_n,
                interp="lagrange_modes", modes=M)


# The mode-space form evaluates the same quadrature operator (its sum over the terms collapsed
# into one diagonal) in float64; the float forms round only the node charges and potentials.
@pytest.mark.parametrize("prec,Kc,Ln,tol,tol_f", [("fp64", 4, 16, 3e-9, 1e-7), ("fp64", 8, 8, 1e-12, 1e-11),
                                                 ("fp64", 6, 12, 1e-10, 1e-9), ("fp32", 8, 8, 2e-6, 3e-5),
                                                 ("bf16x10", 8, 8, 2e-6, 3e-5), ("bf16x10", 16, 4, 2e-6, 3e-5)])
def test_lagrange_modes_match_oracle(torch, prec, Kc, Ln, tol, tol_f):
    x, q = _cloud(500, 7)
    plan = _plan_modes(prec, Kc, Ln, 500)
    R, err = plan.build_skp()
    assert R > 0 and err <= 1e-12 and plan.skp_c() == 0.0
    out = plan.energy_forces(dev(torch, x), dev(torch, q))
    ref = lg.reciprocal(x, q, L_BOX, BETA, Kc, Ln, M)            # exact node operator
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(out["energy"].item() - ref["E"]) / abs(ref["E"])
    print(f"lagrange_modes {prec} Kc={Kc} Ln={Ln}: R={R} phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e}")
    assert e_phi < tol and e_f < tol_f and e_E < tol
    if prec == "fp64" and Ln == 8:
        # the same quadrature summed term by term (the oracle's Algorithm 4 loop)
        sk = lg.reciprocal(x, q, L_BOX, BETA, Kc, Ln, M, method="sinc", tol=1e-12)
        assert rel(host(out["dEdq"]), sk["phi"]) < 1e-13 and rel(host(out["forces"]), sk["F"]) < 1e-12


def test_lagrange_modes_non_neutral_autotune_and_potential(torch):
    x, q = _cloud(300, 4)
    q = q + 0.25                                                  # the m = 0 mode is not in the cube sum
    plan = _plan_modes("fp64", 4, 16, 300)
    plan.build_skp()
    xd, qd = dev(torch, x), dev(torch, q)
    plan.autotune(xd, qd)
    out = plan.energy_forces(xd, qd)
    ref = lg.reciprocal(x, q, L_BOX, BETA, 4, 16, M)
    assert rel(host(out["dEdq"]), ref["phi"]) < 3e-9
    # potentials at other points (a second cell sort of the targets)
    t = np.random.default_rng(5).uniform(0.0, L_BOX, (77, 3))
    p = plan.potential(xd, qd, dev(torch, t))
    Qn = lg.spread(x, q, L_BOX, 4, 16)
    Phi = lg.apply_exact(Qn, 4, 16, L_BOX, BETA, M)
    p_r, _ = lg.gather(t, np.zeros(len(t)), L_BOX, 4, 16, Phi)
    assert rel(host(p), p_r) < 3e-9


@pytest.mark.parametrize("Kc,Ln,Mm", [(2, 4, 7), (2, 4, 9), (3, 6, 8)])
def test_lagrange_modes_more_modes_than_nodes(torch, Kc, Ln, Mm):
    """Mode rows r = 2M + 1 above the node count of an axis, and above the grouped kernels'
    register budget (M > 7: one launch per transform)."""
    from paper_2601_18838_gb300 import Plan
    x, q = _cloud(120, 13)
    plan = Plan(L_BOX, Kc * Ln, Ln, BETA, precision="fp64", skp_tol=1e-12, skp_method="sinc", max_n=120,
                interp="lagrange_modes", modes=Mm)
    plan.build_skp()
    out = plan.energy_forces(dev(torch, x), dev(torch, q))
    ref = lg.reciprocal(x, q, L_BOX, BETA, Kc, Ln, Mm)
    assert rel(host(out["dEdq"]), ref["phi"]) < 1e-10 and rel(host(out["forces"]), ref["F"]) < 1e-9
