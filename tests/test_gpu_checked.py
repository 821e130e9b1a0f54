"""The checked build (libkpme_debug.so: every index of the particle and mesh kernels checked
against its buffer, a failed check reported by the next call as an error naming the kernel)
runs the particle paths cleanly and gives the release build's results.  It runs in a child
process, since a process loads one build of the library."""
import os
import subprocess
import sys
import textwrap

import pytest

from tests._gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np, torch
    from oracle import skp
    from paper_2601_18838_gb300 import Plan, Batch, _binding, workloads as wl
    assert _binding.LIB_PATH.endswith("libkpme_debug.so"), _binding.LIB_PATH
    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    cases = [(32, 1001, 18.0, 4, "bf16x10", 0), (32, 1001, 18.0, 4, "bf16x10", -1),
             (64, 3001, 40.0, 6, "fp32", 0), (64, 3001, 40.0, 4, "bf16x10", -1),
             (128, 5003, 90.0, 4, "bf16x10", 0), (32, 999, 17.0, 4, "fp64", 0)]
    for K, n, L, order, prec, tile in cases:
        s = wl.random_system(n, L, K, order, seed=K + n)
        plan = Plan(s.box, s.K, s.order, s.beta, precision=prec, skp_tol=s.skp_tol, max_n=s.n)
        o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
        plan.set_skp(*skp.generators(o))
        plan.set_tune(tile, 1, 2)
        x, q = torch.tensor(s.x, device="cuda"), torch.tensor(s.q, device="cuda")
        for _ in range(2):   # a failed check of the first call is reported by the second
            out = plan.energy_forces(x, q, virial=True)
        ref = skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o)
        e = rel(out["dEdq"].cpu().numpy(), ref["phi"])
        assert e < (1e-12 if prec == "fp64" else 2e-6), (K, prec, tile, e)
        phi, F = plan.gather(x, q, torch.randn(K, K, K, dtype=torch.float64, device="cuda"))
        plan.energy_forces(x, q)   # reports a failed check of the stage calls above
        plan.close()
        print("checked", K, prec, tile, f"{{e:.2e}}", flush=True)
    systems = [wl.random_system(1200, 31.0, 32, 4, seed=41), wl.random_system(2501, 47.0, 48, 4, seed=42)]
    b = Batch([dict(box=s.box, K=s.K, order=s.order, beta=s.beta, skp_tol=s.skp_tol, max_n=s.n) for s in systems])
    b.build_skp()
    off = np.cumsum([0] + [s.n for s in systems])
    x = torch.tensor(np.concatenate([s.x for s in systems]), device="cuda")
    q = torch.tensor(np.concatenate([s.q for s in systems]), device="cuda")
    for _ in range(2):
        b.energy_forces(x, q, off, virial=True)
    torch.cuda.synchronize()
    b.close()
    print("checked batch", flush=True)
""")


def test_checked_build_runs_the_particle_paths_cleanly():
    cuda_or_skip()
    from paper_2601_18838_gb300 import build as b
    b.build(debug=True)
    env = dict(os.environ, KPME_LIB="debug")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900)
    print(r.stdout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("checked") == 7
