"""kpme_save_skp / kpme_load_skp: an SKP stored by one plan and installed in another gives the
same evaluation, and files that do not fit the plan are refused with a message."""
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


def _plan(s, prec, K=None, box=None):
    from paper_2601_18838_gb300 import Plan
    return Plan(box or s.box, K or s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)


@pytest.mark.parametrize("prec,method", [("fp64", "svd"), ("bf16x10", "svd"), ("bf16x10", "sinc")])
def test_saved_skp_reproduces_the_evaluation(torch, tmp_path, prec, method):
    from paper_2601_18838_gb300 import Plan
    s = wl.random_system(1500, 21.0, 32, 4, seed=5)
    mk = lambda: Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n, skp_method=method)
    a = mk()
    a.build_skp()
    path = tmp_path / "skp.bin"
    a.save_skp(path)
    b = mk()
    b.load_skp(path)
    ga, gb = a.get_skp(), b.get_skp()
    for k in ("r1", "gen3", "gen2", "gen1"):
        np.testing.assert_array_equal(np.asarray(ga[k]), np.asarray(gb[k]))
    assert ga["c"] == gb["c"]
    x, q = dev(torch, s.x), dev(torch, s.q)
    oa, ob = a.energy_forces(x, q, virial=True), b.energy_forces(x, q, virial=True)
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert rel(host(ob["dEdq"]), host(oa["dEdq"])) < tol and rel(host(ob["forces"]), host(oa["forces"])) < tol
    # and the loaded plan still matches the float64 SKP oracle of the same system
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol, method=method) if method == "sinc" else \
        skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    r = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
    assert rel(host(ob["dEdq"]), r["phi"]) < (1e-7 if prec == "fp64" else 1e-6)
    a.close()
    b.close()


def test_load_refuses_files_that_do_not_fit(torch, tmp_path):
    from paper_2601_18838_gb300 import KpmeError
    s = wl.random_system(800, 21.0, 32, 4, seed=6)
    a = _plan(s, "bf16x10")
    a.build_skp()
    good = tmp_path / "good.bin"
    a.save_skp(good)
    cases = {}
    cases["other K"] = _plan(s, "bf16x10", K=48)
    cases["other box"] = _plan(s, "bf16x10", box=22.0)
    for why, p in cases.items():
        with pytest.raises(KpmeError, match="differs"):
            p.load_skp(good)
        p.close()
    b = _plan(s, "bf16x10")
    short = tmp_path / "short.bin"
    short.write_bytes(good.read_bytes()[:200])
    with pytest.raises(KpmeError, match="short"):
        b.load_skp(short)
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not an skp at all" * 4)
    with pytest.raises(KpmeError, match="not an SKP file"):
        b.load_skp(junk)
    with pytest.raises(KpmeError, match="cannot open"):
        b.load_skp(tmp_path / "missing.bin")
    b.load_skp(good)   # the plan is still usable after the refusals
    out = b.energy_forces(dev(torch, s.x), dev(torch, s.q))
    assert np.isfinite(out["energy"].item())
    a.close()
    b.close()
