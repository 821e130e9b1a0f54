"""bench.py on the host: the reference arm (the float64 oracle timed on the host cores) prints
the contract's JSON line, and every workload the bench names exists."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_every_bench_workload_is_defined():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_18838_gb300 import workloads
    for name in bench.WORKLOAD_TEXT:
        if name != "batched":   # a list of systems, built by the batched runner
            s = workloads.by_name(name)
            assert s.n > 0 and s.K > 0


def test_measured_records_follow_their_kernels():
    """The DRAM-traffic and tensor-activity records of bench.py carry the digest of the kernel
    sources they were measured on: a record reports only while its own workload's kernels are
    unchanged and its launch split matches, and the 10^6-charge box's digest does not cover the
    fused kernel it never runs."""
    sys.path.insert(0, ROOT)
    import bench
    assert "gemm_ozf.cu" not in bench.SKP_SOURCES["large"]
    for (w, prec), rec in bench.SKP_TRAFFIC.items():
        ok = rec["digest"] == bench._skp_digest(w)
        assert (bench._skp_traffic(w, prec, rec["launches"]) is not None) == ok
        assert bench._skp_traffic(w, prec, rec["launches"] + 1) is None
    assert bench._skp_traffic("large", "fp32", 4) is None
