"""GPU parity: the CUDA path through the C ABI against the CPU oracle, stage by stage and
end to end, on seeded inputs (several tiles plus ragged tails)."""
import numpy as np
import pytest

from oracle import skp, spme
from paper_2601_18838_gb300 import workloads as wl
from tests._gpu_util import cuda_or_skip, dev, host, rel

pytestmark = pytest.mark.gpu

# Relative RMS error bars against the float64 SKP oracle (potentials, forces): 1e-6 / 1e-5 for
# the float32 and split forms, 1e-3 for the single-product forms (plain BF16; plain TF32 is
# held to the same bar), whose force bar is taken at the same 1:10 ratio, 1e-2.  FP64 is held
# to its own arithmetic.
BAR = {"fp64": (1e-12, 1e-11), "fp32": (1e-6, 1e-5), "tf32x3": (1e-6, 1e-5), "bf16x6": (1e-6, 1e-5),
       "bf16x3": (1e-6, 1e-5), "bf16x10": (1e-6, 1e-5), "tf32": (1e-3, 1e-2), "bf16": (1e-3, 1e-2)}
TOL = BAR
FORMS = ["fp64", "fp32", "tf32x3", "bf16x6", "bf16x3", "tf32", "bf16", "bf16x10"]

# Forms that miss their bar, with the errors measured on one GB300 (phi, F): strict xfails, so
# a change that brings a form under its bar turns the test red until the mark is removed.
MISSES = {
    ("small", "bf16x3"): "phi 4.9e-6, F 1.9e-5: 16 significant bits per operand (2^-17 per value)",
    ("small", "bf16"): "phi 3.2e-3, F 1.0e-2: 8 significant bits per operand",
    ("water", "fp32"): "phi 1.9e-6, F 8.0e-6: per-multiply-add float32 rounding over the three stages",
    ("water", "tf32x3"): "phi 7.1e-6, F 1.4e-5: 22-bit operands and the tensor core's float32 accumulation",
    ("water", "bf16x6"): "phi 5.8e-6, F 1.3e-5: the tensor core's float32 accumulation of floating slices",
    ("water", "bf16x3"): "phi 5.9e-5, F 2.8e-4: 16 significant bits per operand",
    ("water", "tf32"): "phi 4.8e-3, F 2.8e-2: 11 significant bits per operand",
    ("water", "bf16"): "phi 3.2e-2, F 1.3e-1: 8 significant bits per operand",
    ("apply_water", "fp32"): "Phi 3.7e-6: per-multiply-add float32 rounding",
    ("apply_water", "tf32x3"): "Phi 8.6e-6",
    ("apply_water", "bf16x6"): "Phi 7.5e-6",
    ("apply_water", "bf16x3"): "Phi 1.4e-4",
    ("apply_water", "tf32"): "Phi 1.4e-2",
    ("apply_water", "bf16"): "Phi 6.0e-2",
    ("apply_small", "bf16x3"): "Phi 6.6e-6",
    ("apply_small", "bf16"): "Phi 3.8e-3",
}


def _forms(box, forms=FORMS):
    out = []
    for f in forms:
        why = MISSES.get((box, f))
        out.append(pytest.param(f, marks=pytest.mark.xfail(reason=f"measured {why}", strict=True)) if why else f)
    return out


@pytest.fixture(scope="module")
def torch():
    t = cuda_or_skip()
    import __graft_entry__ as g
    g.build()
    return t


def _plan(s, prec, **kw):
    from paper_2601_18838_gb300 import Plan
    return Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=max(s.n, 1), **kw)


def _oracle_skp(s):
    return skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)


@pytest.mark.parametrize("prec", ["fp64", "bf16x10"])
def test_sinc_skp_build_matches_oracle(torch, prec):
    # §2.1.2: the GPU picks the same node count as the oracle's search and its energy, potentials
    # and forces (with the m = 0 correction of the rule) match the oracle's sinc evaluation
    s = wl.small()
    plan = _plan(s, prec, skp_method="sinc")
    R, err = plan.build_skp()
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol, method="sinc")
    assert R == o.R
    assert err <= s.skp_tol
    g = plan.get_skp()
    assert g["r0"] == R and list(g["r1"]) == [1] * R
    np.testing.assert_allclose(g["c"], o.c, rtol=1e-9)
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    out = plan.energy_forces(dev(torch, s.x), dev(torch, s.q))
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(host(out["energy"])[0] - ref["E"]) / abs(ref["E"])
    print(f"sinc {prec}: R={R} err={err:.2e} phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e}")
    tp = 1e-9 if prec == "fp64" else 1e-6
    assert e_phi < tp and e_f < 10 * tp and e_E < tp
    # and it approximates the same operator as the SVD form
    sv = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=_oracle_skp(s))
    assert rel(host(out["dEdq"]), sv["phi"]) < 1e-6


@pytest.mark.parametrize("prec,order,n,sort", [("fp64", 4, 999, True), ("fp32", 4, 999, True), ("fp64", 6, 1001, True),
                                               ("fp32", 8, 257, True), ("fp32", 4, 999, False),
                                               ("bf16x10", 6, 1001, False), ("fp32", 8, 257, False)])
def test_spread(torch, prec, order, n, sort):
    s = wl.random_system(n, 17.0, 32, order, seed=n)
    plan = _plan(s, prec)
    if not sort:
        plan.set_tune(-1, 1, 2)   # no cell sort: lane-group spreading with float32 atomics
    Q = host(plan.spread(dev(torch, s.x), dev(torch, s.q)))
    ref = spme.spread(s.x, s.q, s.box, s.K, s.order)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert np.abs(Q - ref).max() <= tol * np.abs(ref).max()
    assert abs(Q.sum() - s.q.sum()) < 1e-4


def test_spread_boundary_particles(torch):
    L, K = 10.0, 16
    x = np.array([[0.0, 0.0, 0.0], [10.0, 5.0, -10.0], [-0.0, 20.0, 9.999999999999998],
                  [2.5, 7.5, 3.125], [-3.0, 13.0, 0.625]])
    q = np.array([1.0, -1.0, 0.5, -0.25, 2.0])
    s = wl.System("edge", x, q, L, K, 4)
    plan = _plan(s, "fp64")
    Q = host(plan.spread(dev(torch, x), dev(torch, q)))
    np.testing.assert_allclose(Q, spme.spread(x, q, L, K, 4), atol=1e-15)


@pytest.mark.parametrize("prec,sort", [("fp32", True), ("fp32", False), ("bf16x10", True)])
def test_mesh_coordinates_near_cell_boundaries(torch, prec, sort):
    """The float32 forms take the mesh coordinate in double-float arithmetic and fall back to
    the float64 rounding sequence within 2^-20 of a cell boundary: positions on the mesh
    points, one float64 ulp either side, at the box faces, outside the box (one and several
    periods) and just inside 1e-12 of a boundary spread and gather as the oracle does."""
    L, K, order = 19.0, 32, 6
    rng = np.random.default_rng(11)
    h = L / K
    cands = [k * h for k in range(-K, 2 * K + 1)]
    cands += [np.nextafter(v, np.inf) for v in cands] + [np.nextafter(v, -np.inf) for v in cands]
    cands += [v + 1e-12 for v in cands[:3 * K]] + [0.0, -0.0, L, -L, 2.5 * L, -3.25 * L, 7.0 * L + h]
    cands = np.array(cands)
    n = 601
    x = np.stack([rng.choice(cands, n) for _ in range(3)], axis=1)
    x[::3] = rng.uniform(-L, 2 * L, size=x[::3].shape)   # and ordinary positions between them
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    s = wl.System("edges", x, q, L, K, order)
    plan = _plan(s, prec)
    if not sort:
        plan.set_tune(-1, 1, 2)
    Q = host(plan.spread(dev(torch, x), dev(torch, q)))
    ref = spme.spread(x, q, L, K, order)
    assert np.abs(Q - ref).max() <= 2e-6 * np.abs(ref).max()
    Phi = rng.standard_normal((K, K, K))
    phi, F = plan.gather(dev(torch, x), dev(torch, q), dev(torch, Phi))
    phi_r, F_r = spme.gather(x, q, L, K, order, Phi)
    assert rel(host(phi), phi_r) < 2e-6 and rel(host(F), F_r) < 2e-6


def test_skp_build_matches_oracle(torch):
    s = wl.small()
    plan = _plan(s, "fp64")
    R, err = plan.build_skp()
    o = _oracle_skp(s)
    g = plan.get_skp()
    assert g["r0"] == len(o.r1)
    assert list(g["r1"]) == list(o.r1)
    assert R == o.R
    np.testing.assert_allclose(g["sigma_outer"], o.outer[:g["r0"]], rtol=1e-10)
    si = np.concatenate([o.inner[i][:r] for i, r in enumerate(o.r1)])
    np.testing.assert_allclose(g["sigma_inner"], si, rtol=1e-9, atol=1e-12 * si.max())
    assert err <= s.skp_tol
    # the two SKPs are different factorisations of the same truncated operator
    Q = spme.spread(s.x, s.q, s.box, s.K, s.order)
    Phi_gpu = host(plan.apply(dev(torch, Q)))
    Phi_ref = skp.apply(Q, o)
    assert rel(Phi_gpu, Phi_ref) < 4 * s.skp_tol


def _apply_case(torch, s, prec):
    o = _oracle_skp(s)
    r1, g3, g2, g1 = skp.generators(o)
    plan = _plan(s, prec)
    plan.set_skp(r1, g3, g2, g1)
    Q = spme.spread(s.x, s.q, s.box, s.K, s.order)
    Phi_ref = skp.apply(Q, o)
    Phi = host(plan.apply(dev(torch, Q)))
    plan.close()
    return rel(Phi, Phi_ref)


# bf16x6 on the small box measures 1.05e-6, too close to the bar for a strict mark either way
@pytest.mark.parametrize("prec", _forms("apply_small", [f for f in FORMS if f != "bf16x6"]))
def test_apply_with_oracle_factors(torch, prec):
    e = _apply_case(torch, wl.small(), prec)
    print(f"{prec}: rel Phi {e:.3e}")
    assert e < BAR[prec][0]


@pytest.mark.parametrize("prec", _forms("apply_water"))
def test_apply_with_oracle_factors_water(torch, prec):
    e = _apply_case(torch, wl.water(), prec)
    print(f"water {prec}: rel Phi {e:.3e}")
    assert e < BAR[prec][0]


@pytest.mark.parametrize("prec,order,sort", [("fp64", 6, True), ("fp32", 6, True), ("fp32", 6, False),
                                             ("fp32", 4, False), ("bf16x10", 8, False)])
def test_gather(torch, prec, order, sort):
    s = wl.random_system(1531, 23.0, 48, order, seed=3)
    rng = np.random.default_rng(0)
    Phi = rng.standard_normal((48, 48, 48))
    plan = _plan(s, prec)
    if not sort:
        plan.set_tune(-1, 1, 2)   # no cell sort: one thread per particle, untiled mesh reads
    phi, F = plan.gather(dev(torch, s.x), dev(torch, s.q), dev(torch, Phi))
    phi_r, F_r = spme.gather(s.x, s.q, s.box, 48, order, Phi)
    tol = 1e-13 if prec == "fp64" else 2e-6
    assert rel(host(phi), phi_r) < tol and rel(host(F), F_r) < tol


@pytest.mark.parametrize("prec", _forms("small"))
def test_energy_forces_small(torch, prec):
    s = wl.small()
    o = _oracle_skp(s)
    ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    plan = _plan(s, prec)
    plan.set_skp(*skp.generators(o))
    out = plan.energy_forces(dev(torch, s.x), dev(torch, s.q), virial=True)
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(out["energy"].item() - ref["E"]) / abs(ref["E"])
    e_W = abs(out["virial"].item() - ref["W"]) / abs(ref["W"])
    print(f"{prec}: phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e} W {e_W:.2e}")
    tp, tf = BAR[prec]
    plan.close()
    assert e_phi < tp and e_f < tf and e_E < 10 * tp and e_W < 10 * tp


@pytest.fixture(scope="module")
def water_ref():
    s = wl.water()
    o = _oracle_skp(s)
    return s, o, skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)


@pytest.mark.parametrize("prec", _forms("water"))
def test_energy_forces_water_box(torch, water_ref, prec):
    # the 67 A water box (30,000 atoms, K = 64) at the bars of its form
    s, o, ref = water_ref
    x, q = dev(torch, s.x), dev(torch, s.q)
    plan = _plan(s, prec)
    plan.set_skp(*skp.generators(o))
    out = plan.energy_forces(x, q)
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    print(f"water {prec}: phi {e_phi:.2e} F {e_f:.2e}")
    tp, tf = BAR[prec]
    plan.close()
    assert e_phi < tp and e_f < tf


@pytest.mark.parametrize("K,order,n,L,fused,fold,ozt", [
    (32, 4, 1001, 18.0, "1", "1", "1"),     # fused stages 2-3, BN = 32 (four k3' per tile)
    (32, 4, 1001, 18.0, "0", "1", "1"),     # tensor-memory A, resident and per pair
    (48, 4, 2050, 30.0, "1", "1", "2"),     # K % 32 != 0 on tensor-memory A: one 64-wide chunk holding
                                            # 48 values; a warp's rows reach two next-stage rows
    (48, 4, 2050, 30.0, "1", "1", "1"),     # (default) the shared-memory A kernel, row maxima across warps
    (64, 4, 3001, 40.0, "1", "1", "1"),     # fused, BN = 64
    (64, 4, 3001, 40.0, "0", "1", "1"),
    (96, 6, 4003, 70.0, "1", "1", "1"),     # tensor-memory A, two 64-wide chunks (second half empty)
    (128, 4, 5003, 90.0, "1", "0", "1"),    # tensor-memory A, two full chunks, two column tiles
    (128, 4, 5003, 90.0, "1", "1", "1"),    # reflection basis: one 64-wide chunk per half
    (256, 6, 20011, 150.0, "1", "1", "1"),  # reflection basis, two chunks per half, four column tiles
])
def test_error_free_split_sizes(torch, monkeypatch, K, order, n, L, fused, fold, ozt):
    # ragged particle counts and the kernel variants of the error-free split
    monkeypatch.setenv("KPME_FUSED", fused)
    monkeypatch.setenv("KPME_FOLD", fold)
    monkeypatch.setenv("KPME_OZT", ozt)
    s = wl.random_system(n, L, K, order, seed=K + n)
    o = _oracle_skp(s)
    ref = skp.reciprocal(s.x, s.q, s.box, K, order, s.beta, s.skp_tol, skp=o)
    plan = _plan(s, "bf16x10")
    plan.set_skp(*skp.generators(o))
    out = plan.energy_forces(dev(torch, s.x), dev(torch, s.q), virial=True)
    e_phi, e_f = rel(host(out["dEdq"]), ref["phi"]), rel(host(out["forces"]), ref["F"])
    e_E = abs(host(out["energy"])[0] - ref["E"]) / abs(ref["E"])
    e_W = abs(host(out["virial"])[0] - ref["W"]) / abs(ref["W"])
    print(f"bf16x10 K={K} fused={fused} fold={fold} ozt={ozt}: phi {e_phi:.2e} F {e_f:.2e} E {e_E:.2e} W {e_W:.2e}")
    assert e_phi < 1e-6 and e_f < 1e-5 and e_E < 1e-6 and e_W < 1e-5
    # the stage entry point on the same mesh: the operator alone, float64 in and out
    Q = spme.spread(s.x, s.q, s.box, K, order)
    assert rel(host(plan.apply(dev(torch, Q))), skp.apply(Q, o)) < 1e-6
    plan.close()


def test_potential_targets_differ_from_sources(torch):
    s = wl.random_system(640, 15.0, 32, 4, seed=77)
    xt = np.random.default_rng(1).uniform(-3, 18, (333, 3))
    o = _oracle_skp(s)
    Phi = skp.apply(spme.spread(s.x, s.q, s.box, 32, 4), o)
    ref, _ = spme.gather(xt, np.zeros(333), s.box, 32, 4, Phi)
    plan = _plan(s, "fp64")
    plan.set_skp(*skp.generators(o))
    p = host(plan.potential(dev(torch, s.x), dev(torch, s.q), dev(torch, xt)))
    assert rel(p, ref) < 1e-12


def test_empty_and_errors(torch):
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(64, 12.0, 32, 4, seed=5)
    plan = _plan(s, "fp32")
    x, q = dev(torch, s.x), dev(torch, s.q)
    with pytest.raises(KpmeError, match="not built"):
        plan.energy_forces(x, q)
    plan.build_skp()
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda:0")
    out = plan.energy_forces(e, torch.zeros(0, dtype=torch.float64, device="cuda:0"), virial=True)
    assert out["energy"].item() == 0.0 and out["virial"].item() == 0.0
    big = dev(torch, np.zeros((65, 3)))
    with pytest.raises(KpmeError, match="capacity"):
        plan.energy_forces(big, dev(torch, np.zeros(65)))


@pytest.mark.parametrize("prec,box", [("fp64", "small"), ("fp32", "small"), ("bf16x10", "small"),
                                      ("bf16x10", "water")])
def test_virial_tensor_matches_oracle(torch, prec, box):
    # full reciprocal virial tensor (mode space, exact mesh kernel) against the oracle's FFT
    # evaluation on the same mesh; its trace is the scalar virial of energy_forces up to the
    # SKP approximation of the mesh kernel
    s = wl.small() if box == "small" else wl.water()
    x, q = dev(torch, s.x), dev(torch, s.q)
    plan = _plan(s, prec)
    Pi, E = plan.virial_tensor(x, q)
    Q = spme.spread(s.x, s.q, s.box, s.K, s.order)
    ref = spme.virial_tensor(Q, s.K, s.order, s.box, s.beta)
    Eref = 0.5 * float(np.sum(spme.influence(s.K, s.order, s.box, s.beta) * np.abs(np.fft.fftn(Q)) ** 2))
    Pi = host(Pi)
    tol = 1e-12 if prec == "fp64" else 5e-6
    e_pi = np.linalg.norm(Pi - ref) / np.linalg.norm(ref)
    print(f"{prec} {box}: tensor {e_pi:.2e}")
    assert e_pi < tol and abs(float(E) - Eref) < tol * abs(Eref)
    np.testing.assert_array_equal(Pi, Pi.T)
    plan.set_skp(*skp.generators(_oracle_skp(s)))
    W = plan.energy_forces(x, q, virial=True)["virial"].item()
    assert abs(np.trace(Pi) - W) < 1e-6 * abs(W)
