"""Benchmark: reciprocal evaluations per second of the tensor-core SKP path on GB300.

One step = one reciprocal evaluation of the whole path (spread, SKP mode products,
gather of potentials and forces, float64 energy and virial) for the 10^6-charge box
(220 A, B-spline order 6, K = 256, SKP tolerance 1e-7), the largest single-GPU
workload; the water box (10^4 rigid 3-site molecules, K = 64) is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x10]
                    [--workload large|water|small|mixed|lagrange|batched] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica on its
own GPU (the path has no data-parallel split for one system); ``value`` is the
evaluations of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reciprocal evals/s + TFLOP/s at ≤1e-6 rel err: tensor-core SKP vs FP64 form"
WORKLOAD_TEXT = {
    "water": "water box: 10^4 rigid 3-site molecules (30,000 atoms), L=67 A, B-spline order 4, K=64, "
             "beta=0.35/A, SKP tol 1e-8",
    "small": "1000 charges +-1, L=20 A, order 4, K=32, beta=0.35/A, SKP tol 1e-8",
    "mixed": "1e5 charges (+-1, +-0.5), L=100 A, order 6, K=96, beta=0.35/A, SKP tol 1e-8",
    "large": "1e6 charges +-1, L=220 A, order 6, K=256, beta=0.35/A, SKP tol 1e-7",
    "batched": "64 independent neutral +-1 systems, N log-uniform in [2000, 50000], box 30-80 A, "
               "K in {32, 48, 64} (box/K <= 1.25 A), order 4, one graph launch per evaluation",
    "lagrange": "per-cell Lagrange form: 2e4 charges +-1, L=30 A, beta=0.1/A, modes |m|_inf <= 4, "
                "8^3 cells of 8^3 equispaced nodes (64 per axis), quadrature SKP 1e-12, no virial; node "
                "operator in mode space (the terms' sum as one diagonal)",
}
DTYPE = {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "tf32x3": "tf32", "bf16": "bf16", "bf16x3": "bf16",
         "bf16x6": "bf16", "bf16x10": "bf16"}


# DRAM bytes (read + write) per launch of the SKP mode-product kernels, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, averaged over the launches of one evaluation),
# with the digest of the kernel sources the counters were taken on: a changed kernel reports
# null until it is captured again.
SKP_TRAFFIC = {
    # profiles/dram_traffic_water_k64_bf16x10.md: mp_ozt_kernel 1,513,984 B + mp_ozf_kernel
    # 19,318,784 B (reads; 0 B written: Y and Phi stay in L2), 2 launches per evaluation
    ("water", "bf16x10"): {"digest": "8b97809330ffdde9", "launches": 2,
                           "bytes_per_launch": (1513984 + 19318784) / 2},
    # profiles/launches_large_k256_bf16x10.md: one evaluation's stage 1 (93,060,608 B read +
    # 880,000,000 B written), stage 2 (1,066,170,880 + 11,189,232,384), stage 3 (11,840,929,792
    # + 277,398,784) and the unfold of Phi (67,126,272 + 4,329,472): 4 launches
    ("large", "bf16x10"): {"digest": "c442ea68c11a0123", "launches": 4,
                           "bytes_per_launch": (93060608 + 880000000 + 1066170880 + 11189232384 + 11840929792
                                                + 277398784 + 67126272 + 4329472) / 4},
}
# the sources of the stage kernels each workload runs (the digest of a record covers these)
SKP_SOURCES = {"water": ("gemm_ozf.cu", "gemm_ozt.cu", "tc_common.cuh"), "large": ("gemm_ozt.cu", "tc_common.cuh")}


def _skp_digest(workload="water"):
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_18838_gb300", "csrc")
    for name in SKP_SOURCES.get(workload, SKP_SOURCES["water"]):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _skp_traffic(workload, precision, launches):
    """Counted DRAM bytes per stage launch, or None once the kernels or the launch split changed."""
    rec = SKP_TRAFFIC.get((workload, precision))
    if not rec or rec["digest"] != _skp_digest(workload) or rec["launches"] != launches:
        return None
    return rec["bytes_per_launch"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _system(name):
    from paper_2601_18838_gb300 import workloads
    return getattr(workloads, name)()


def _oracle_eval(s):
    """The oracle's evaluation of workload s and its plan-time build (returns (build_s, eval, skp))."""
    t0 = time.perf_counter()
    if s.meta.get("interp", "bspline").startswith("lagrange"):
        from oracle import lagrange as lg
        Kc, M = s.meta["cells"], s.meta["modes"]
        fac = lg.sinc_factors(Kc, s.order, s.box, s.beta, M, s.skp_tol)

        def ev():
            Qn = lg.spread(s.x, s.q, s.box, Kc, s.order)
            Phi = lg.apply_skp(Qn, *fac, s.box)
            phi, F = lg.gather(s.x, s.q, s.box, Kc, s.order, Phi)
            return {"phi": phi, "F": F}
        return time.perf_counter() - t0, ev, None
    from oracle import skp
    o = skp.build(s.K, s.order, s.box, s.beta, s.skp_tol)
    return (time.perf_counter() - t0,
            lambda: skp.reciprocal(s.x, s.q, s.box, s.K, s.order, s.beta, s.skp_tol, skp=o), o)


# Full oracle evaluations are timed while one takes at most this many seconds (estimated from
# the work: particles x stencil points and Kronecker terms x K^4); larger workloads are
# timed on a bounded sample of the same evaluation and scaled to one evaluation.
FULL_EVAL_LIMIT_S = 10.0


def _oracle_sample(s, o):
    """One bounded sample of the oracle's evaluation of workload s, scaled to a full
    evaluation: spreading and gathering of the first n_p particles (scaled by N / n_p), the
    SKP operator of Algorithm 2 on the first r_s Kronecker terms (scaled by R / r_s), and the
    virial trace in full.  Returns (estimated seconds per evaluation, description)."""
    import numpy as np
    from oracle import skp, spme
    n_p = min(s.n, 40_000)
    r_s = min(o.R, 4)
    x, q = s.x[:n_p], s.q[:n_p]
    sub = skp.SKP(o.K, o.w[:r_s], o.a0[:r_s], o.a1[:r_s], o.a2[:r_s], 0.0)
    t0 = time.perf_counter()
    Qp = spme.spread(x, q, s.box, s.K, s.order)
    t1 = time.perf_counter()
    Phi = skp.apply(Qp, sub)
    t2 = time.perf_counter()
    spme.gather(x, q, s.box, s.K, s.order, Phi)
    t3 = time.perf_counter()
    spme.virial_trace(Qp, 0.0, s.K, s.order, s.box, s.beta)
    t4 = time.perf_counter()
    est = ((t1 - t0) + (t3 - t2)) * s.n / n_p + (t2 - t1) * o.R / r_s + (t4 - t3)
    desc = (f"spreading and gathering of {n_p} of the {s.n} charges (time x {s.n / n_p:.0f}), the SKP "
            f"operator on {r_s} of its {o.R} Kronecker terms (time x {o.R / r_s:.2f}), the virial trace in "
            f"full; float64 numpy oracle")
    return est, desc


def _full_eval_estimate_s(s):
    # numpy oracle on the host: ~1.5e7 stencil updates/s for spreading plus gathering and
    # ~2e11 flop/s for the dense mode products (6 R K^4 at the rank the tolerance gives)
    R = 50 if s.K <= 64 else 170
    return s.n * s.order ** 3 / 1.5e7 + 6 * R * float(s.K) ** 4 / 2e11


def cpu_baseline(s, budget_s: float = 20.0, max_evals: int = 5, gpu_out=None) -> dict:
    """The float64 oracle (as it stands) on the host cores: full reciprocal evaluations of
    the same workload, as many as fit in the budget (at least one), or, where one full
    evaluation would take longer than FULL_EVAL_LIMIT_S, bounded samples of it scaled to one
    evaluation (repeated while the budget lasts)."""
    t_build, ev, o = _oracle_eval(s)
    cores = os.cpu_count()
    if o is not None and _full_eval_estimate_s(s) > FULL_EVAL_LIMIT_S:
        n, t, ests = 0, 0.0, []
        while n < max_evals and (n == 0 or t < budget_s):
            a = time.perf_counter()
            est, desc = _oracle_sample(s, o)
            t += time.perf_counter() - a
            ests.append(est)
            n += 1
        est = sorted(ests)[len(ests) // 2]
        return {"value": 1.0 / est, "unit": "evals/s", "cores": cores, "kind": "oracle",
                "sample": f"median of {n} samples: {desc} (SKP build {t_build:.1f} s not timed; numpy's BLAS "
                          f"threads for the mode products, one thread for spreading and gathering)"}
    n, t, ref = 0, 0.0, None
    while n < max_evals and (n == 0 or t < budget_s):
        a = time.perf_counter()
        ref = ev()
        t += time.perf_counter() - a
        n += 1
    res = {"value": n / t, "unit": "evals/s", "cores": cores, "kind": "oracle",
           "sample": f"{n} full float64 oracle evaluations (numpy) of the {s.name} workload "
                     f"(SKP build {t_build:.1f} s not timed)"}
    if gpu_out is not None:
        import numpy as np
        phi, F = gpu_out
        res["accuracy_vs_oracle"] = {
            "phi_rel_rms": float(np.linalg.norm(phi - ref["phi"]) / np.linalg.norm(ref["phi"])),
            "F_rel": float(np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"])),
        }
    return res


def run_reference(args):
    """The reference arm: the float64 oracle as it stands on the host cores, the same workload
    and metric.  A step is one full evaluation, or, for workloads whose full evaluation takes
    longer than FULL_EVAL_LIMIT_S, one bounded sample scaled to an evaluation."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    s = _system(args.workload)
    _, ev, o = _oracle_eval(s)
    sampled = o is not None and _full_eval_estimate_s(s) > FULL_EVAL_LIMIT_S
    if sampled:
        for _ in range(args.warmup):
            _oracle_sample(s, o)
        total, desc = 0.0, ""
        for _ in range(args.steps):
            est, desc = _oracle_sample(s, o)
            total += est
        dt = total
        sample = f"per step: {desc}"
    else:
        for _ in range(args.warmup):
            ev()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ev()
        dt = time.perf_counter() - t0
        sample = f"{args.steps} full float64 oracle evaluations per timed region"
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_TEXT[args.workload]},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _init_dist(dev):
    ws, _, _ = _dist()
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("nccl", device_id=dev)
    return dist


def run_batched(args):
    """All systems of the batched workload per step (one graph launch per rank); value in
    system-evaluations per second.  Under torchrun the systems are sharded across the ranks
    by estimated cost (no data-path collective; only the timing is combined, max over
    ranks), so the work per GPU stays fixed as N grows ("scaling": "weak")."""
    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = _init_dist(dev)
    from paper_2601_18838_gb300 import build as _build
    if rank == 0:
        _build.build()
    if pg:
        pg.barrier()
    from paper_2601_18838_gb300 import Batch
    from paper_2601_18838_gb300 import shard, workloads
    systems = workloads.batched()
    parts = shard.partition_lpt([shard.system_cost(s.K, s.n) for s in systems], ws)
    mine = [systems[i] for i in parts[rank]]
    ms = 0.0
    ranks = []
    tuned = 0
    clocks = None
    if mine:
        batch = Batch([dict(box=s.box, K=s.K, order=s.order, beta=s.beta, skp_tol=s.skp_tol, max_n=s.n)
                       for s in mine], precision=args.precision)
        ranks = batch.build_skp()
        offsets = np.cumsum([0] + [s.n for s in mine])
        x = torch.tensor(np.concatenate([s.x for s in mine]), device=dev)
        q = torch.tensor(np.concatenate([s.q for s in mine]), device=dev)
        tuned = 0 if args.no_autotune else batch.autotune(x, q, offsets, cache=args.tune_cache)   # per class
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            batch.energy_forces(x, q, offsets, virial=True)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = ClockSampler(local)
    clk.start()
    if mine:
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.energy_forces(x, q, offsets, virial=True)
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    # end to end through the public API: the step's positions and charges from pinned host
    # memory, the batch, then forces, potentials, energies and virials back to pinned host memory
    e_ms = 0.0
    h2d = d2h = 0
    if mine:
        xh, qh = x.cpu().pin_memory(), q.cpu().pin_memory()
        xd, qd = torch.empty_like(x), torch.empty_like(q)
        n_tot = int(offsets[-1])
        Fh = torch.empty((n_tot, 3), dtype=torch.float64).pin_memory()
        Ph = torch.empty(n_tot, dtype=torch.float64).pin_memory()
        Eh = torch.empty((2, len(mine)), dtype=torch.float64).pin_memory()
        h2d, d2h = n_tot * 32, n_tot * 32 + 16 * len(mine)

        def e2e_step():
            xd.copy_(xh, non_blocking=True)
            qd.copy_(qh, non_blocking=True)
            o = batch.energy_forces(xd, qd, offsets, virial=True)
            Fh.copy_(o["forces"], non_blocking=True)
            Ph.copy_(o["dEdq"], non_blocking=True)
            Eh[0].copy_(o["energy"], non_blocking=True)
            Eh[1].copy_(o["virial"], non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            e_ms += a.elapsed_time(b)
    if pg:
        t = torch.tensor([ms, e_ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms, e_ms = t[0].item(), t[1].item()
    n_sys = len(systems)
    # useful flops: 6 R K^4 per system (its Kronecker terms' three dense mode products), over
    # the whole batch evaluation (particle work and reductions included: the batch is one
    # graph launch, so its kernels are not timed apart)
    useful = sum(6.0 * r * float(s.K) ** 4 for r, s in zip(ranks, mine))
    peak, peak_note, _ = _tensor_peak(args.precision)
    roof = None
    if mine and ms > 0:
        ach = useful / (ms / args.steps * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "the whole batch evaluation (one graph launch: every system's "
                "spreading, SKP mode products, gathering and reductions)", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "peak_source": peak_note,
                "work": "useful flops sum over this rank's systems of 6 R K^4 per evaluation",
                "flops_per_step": useful}
    cb = None
    if rank == 0 and mine and not args.no_cpu_baseline:
        # the float64 oracle on a sample of this rank's systems (four spread over its list),
        # one full evaluation each; value in system-evaluations per second
        sample = mine[::max(1, len(mine) // 4)][:4]
        t_eval = 0.0
        for s in sample:
            _, ev, _ = _oracle_eval(s)
            a = time.perf_counter()
            ev()
            t_eval += time.perf_counter() - a
        cb = {"value": len(sample) / t_eval, "unit": "system-evals/s", "cores": os.cpu_count(), "kind": "oracle",
              "sample": f"one full float64 oracle evaluation each of {len(sample)} of the {len(mine)} systems "
                        f"(K = {', '.join(str(s.K) for s in sample)}; n = {', '.join(str(s.n) for s in sample)}), "
                        f"mean time per system (SKP builds not timed)"}
    line = {"metric": METRIC, "value": n_sys * args.steps / (ms * 1e-3), "unit": "system-evals/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE.get(args.precision, args.precision),
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["batched"], "precision": args.precision, "systems": n_sys,
                       "particles": int(sum(s.n for s in systems)), "skp_ranks_rank0": [int(r) for r in ranks],
                       "autotune": {"systems_timed_rank0": int(tuned) if mine else 0},
                       "parallelism": f"systems sharded over {ws} ranks (longest processing time first)"
                       if ws > 1 else "single GPU",
                       "l2": "flushed between steps (256 MB write outside the timed events)"},
            "roofline": roof,
            "e2e": {"value": n_sys * args.steps / (e_ms * 1e-3), "unit": "system-evals/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h} if e_ms > 0 else None,
            "cpu_baseline": cb, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if mine:
        batch.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def _tensor_peak(precision):
    """Dense tensor peak for the precision's MMA kind: the measured bf16 burst figure (a step of
    this bench is milliseconds long, far from the seconds-long power-capped loop of the
    sustained figure), halved for tf32 (the nominal ratio)."""
    peaks, src = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    note = f"{src} bf16_tflops (burst)"
    if precision.startswith("tf32"):
        peak, note = peak / 2.0, note + " x 1/2 (tf32 nominal ratio)"
    return peak, note, peaks


def _measure(args, name, steps, warmup, ctx, headline):
    """Time `steps` evaluations of workload `name` through one plan (warm-ups first, L2
    flushed before each step, CUDA events on the launching stream), then the same steps with
    the library's per-step events, and (headline only) the end-to-end and FP64-form runs."""
    import numpy as np
    import torch
    from paper_2601_18838_gb300 import Plan
    pg, dev, rank, ws, local = ctx
    s = _system(name)
    if headline and args.skp_tol is not None:
        s.skp_tol = args.skp_tol
    stream = torch.cuda.current_stream()
    lag = s.meta.get("interp", "bspline").startswith("lagrange")
    extra = dict(interp=s.meta["interp"], modes=s.meta["modes"], skp_method="sinc") if lag else {}
    plan = Plan(s.box, s.K, s.order, s.beta, precision=args.precision, skp_tol=s.skp_tol, max_n=s.n, **extra)
    vir = not lag   # the per-cell form has no virial
    R, skp_err = plan.build_skp()
    info = plan.info()
    x = torch.tensor(s.x, device=dev)
    q = torch.tensor(s.q, device=dev)
    # launch configuration picked by timing (before any timed step)
    tune = {"tile": None, "autotune": "off"} if args.no_autotune else plan.autotune(x, q, cache=args.tune_cache)
    out = {"energy": torch.empty(1, dtype=torch.float64, device=dev),
           "forces": torch.empty((s.n, 3), dtype=torch.float64, device=dev),
           "dEdq": torch.empty(s.n, dtype=torch.float64, device=dev),
           "virial": torch.empty(1, dtype=torch.float64, device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def step():
        plan.energy_forces(x, q, forces=True, dEdq=True, virial=vir, out=out)

    def timed(nsteps, profile=False):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        plan.set_profiling(profile)
        plan.get_profile(reset=True)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        prof = plan.get_profile(reset=True)
        plan.set_profiling(False)
        return sum(a.elapsed_time(b) for a, b in evs), prof

    def max_over_ranks(v):
        if not pg:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return t.item()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local) if headline else None
    if clk:
        clk.start()
    ms_total, _ = timed(steps)
    clocks = clk.stop() if clk else None
    ms_total = max_over_ranks(ms_total)
    ms_step = ms_total / steps
    res = {"workload": name, "value": ws * steps / (ms_total * 1e-3), "unit": "evals/s", "ms_per_step": ms_step,
           "clocks": clocks, "skp_rank": R, "skp_r0": info["r0"], "skp_rel_err": skp_err,
           "autotune": ({k: tune[k] for k in ("tile", "fused", "split", "ms_per_eval")}
                        if not args.no_autotune else "off")}

    # per-kernel timing (same steps, library events on the launching stream)
    _, prof = timed(steps, profile=True)
    res["profile_ms_per_step"] = {k: v[0] / steps for k, v in prof.items()}
    res["launches_per_step"] = sum(v[1] for v in prof.values()) / steps
    K = s.K
    skp_ms = sum(prof[k][0] for k in ("skp_stage1", "skp_stage2", "skp_stage3")) / steps
    skp_launches = sum(prof[k][1] for k in ("skp_stage1", "skp_stage2", "skp_stage3")) / steps
    tensor = args.precision in ("bf16", "tf32", "bf16x3", "tf32x3", "bf16x6", "bf16x10")
    peak, peak_note, peaks = _tensor_peak(args.precision)
    useful = info["flops_useful"]          # 6 R K^4 per evaluation
    executed = info["flops_executed"]      # MMA flops the split form issues
    kname = ("SKP mode products, error-free split on tcgen05 (mp_ozt_kernel stage 1, mp_ozf_kernel fused "
             "stages 2-3 for K = 32/64; mp_ozt/mp_oz_kernel stages 1-3 otherwise)" if args.precision == "bf16x10"
             else "mp_tc_kernel (SKP mode products, tcgen05)")
    roof = None
    if tensor and skp_ms > 0:
        ach = useful / (skp_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": kname, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": _skp_traffic(name, args.precision, skp_launches),
                "peak_source": peak_note,
                "work": "useful flops 6 R K^4 per evaluation (the three dense mode products of every Kronecker "
                        "term); the split form issues more on the tensor pipe (see executed)",
                "flops_per_step": useful, "ms_per_step": skp_ms, "launches_per_step": skp_launches,
                "ms_per_launch": skp_ms / max(skp_launches, 1)}
        ex = executed / (skp_ms * 1e-3) / 1e12
        res["executed"] = {"flops_per_step": executed, "TFLOP/s": ex, "frac_of_peak": ex / peak,
                           "note": "bf16 MMA flops issued per evaluation: digit products of the split "
                                   "(10 per multiply for bf16x10) over the two-level term structure "
                                   "(r0 + 2R) 2 K^4 (K^4 per fold half on folded meshes)"}
        res["tensor_pipe_active"] = _tensor_active(name, args.precision)
    if lag and s.meta["interp"] == "lagrange_modes":
        # the node operator in mode space on the CUDA cores: double-float multiply-adds on the
        # float32 pipe (float forms) or float64 (FP64 form)
        if args.precision == "fp64":
            alu_peak, src = 1250.0, "nominal FP64 rate of a GB300 (1.25 TFLOP/s)"
        else:
            # 152 SMs x 128 float32 lanes x 2070 MHz, 15 float32 instructions per double-float
            # multiply-add (df_mul + df_add), 2 flops per multiply-add
            alu_peak = 152 * 128 * 2.07 / 15 * 2
            src = "float32 pipe (152 SMs x 128 lanes x 2070 MHz) / 15 instructions per double-float multiply-add"
        ach = executed / (skp_ms * 1e-3) / 1e9 if skp_ms > 0 else None
        roof = {"bound": "alu", "kernel": "modes_axis_df_kernel / modes_mid_df_kernel (mode-space node operator: "
                                          "three forward and three backward transforms, the diagonal fused)",
                "achieved": ach, "peak": alu_peak, "unit": "GFLOP/s", "frac": (ach / alu_peak) if ach else None,
                "traffic": None, "peak_source": src,
                "flops_per_step": executed, "ms_per_step": skp_ms, "launches_per_step": skp_launches,
                "ms_per_launch": skp_ms / max(skp_launches, 1)}
    res["roofline"] = roof
    res["tflops_useful"] = useful / (ms_step * 1e-3) / 1e12
    # spreading and gathering against HBM: algorithmic bytes per evaluation (positions and
    # charges in float64, the float32 mesh written or read once, potentials and forces out)
    hbm = peaks.get("hbm_gbs", 6800.0)
    mesh_b = 4 * K ** 3
    part = {}
    for kn, nbytes in (("spread", s.n * 32 + mesh_b), ("gather", mesh_b + s.n * 32 + s.n * 32)):
        ms_k = prof[kn][0] / steps if kn in prof else 0.0
        gbs = nbytes / (ms_k * 1e-3) / 1e9 if ms_k > 0 else None
        part[kn] = {"bytes_per_eval": nbytes, "ms_per_eval": ms_k, "GB/s": gbs, "frac_hbm": (gbs / hbm) if gbs else None}
    part["hbm_peak_gbs"] = hbm
    if not lag and ("spread" in prof or "gather" in prof):
        # the bound of the B-spline kernels is the rate of their n^3 float32 updates (atomics)
        # and stencil reads per particle, not their bytes: measured live, same pattern
        from paper_2601_18838_gb300._binding import measure_update_rate
        rates = measure_update_rate(K, s.order, min(s.n, 1 << 20))
        sorted_path = tune.get("tile") not in (-1, None) or tune.get("autotune") == "off"
        upd = s.n * s.order ** 3
        for kn, peak_k, what in (("spread", "shared_atomic" if sorted_path else "global_atomic",
                                  "float32 atomic adds of the stencils (tile region in shared memory)" if sorted_path
                                  else "float32 atomic adds of the stencils into the mesh in device memory"),
                                 ("gather", "read", "stencil reads of the float32 mesh, one thread per particle")):
            ms_k = part[kn]["ms_per_eval"]
            if ms_k > 0:
                ach = upd / (ms_k * 1e-3)
                part[kn]["roofline"] = {"bound": "atomics" if kn == "spread" else "loads", "achieved": ach,
                                        "peak": rates[peak_k], "unit": "updates/s" if kn == "spread" else "reads/s",
                                        "frac": ach / rates[peak_k] if rates[peak_k] else None,
                                        "work": f"n order^3 = {upd} per evaluation: {what}",
                                        "peak_source": "kpme_measure_update_rate (same access pattern, live)"}
    part["note"] = ("per-cell Lagrange: spread = counting sort by cell (clear, count, scan, scatter) + one CTA "
                    "per cell writing its Ln^3 node block once (no atomics), gather = one CTA per cell with the "
                    "block in shared memory, one warp per particle"
                    if lag else
                    "no cell sort (autotuned): spread = mesh clear + lane-group spreading with float32 atomics "
                    "into the L2-resident mesh, gather = one thread per particle"
                    if tune.get("tile") == -1 else
                    "spread includes the cell sort (count, scan, scatter); gather reads the sorted records")
    res["particle_kernels"] = part

    if headline:
        # end to end through the public API with host buffers
        xh = torch.tensor(s.x).pin_memory()
        qh = torch.tensor(s.q).pin_memory()
        Fh = torch.empty((s.n, 3), dtype=torch.float64).pin_memory()
        ph = torch.empty(s.n, dtype=torch.float64).pin_memory()
        Eh = torch.empty(2, dtype=torch.float64).pin_memory()
        xd = torch.empty_like(x)
        qd = torch.empty_like(q)

        def e2e_step():
            xd.copy_(xh, non_blocking=True)
            qd.copy_(qh, non_blocking=True)
            plan.energy_forces(xd, qd, forces=True, dEdq=True, virial=vir, out=out)
            Fh.copy_(out["forces"], non_blocking=True)
            ph.copy_(out["dEdq"], non_blocking=True)
            Eh[0:1].copy_(out["energy"], non_blocking=True)
            if vir:
                Eh[1:2].copy_(out["virial"], non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            e_ms += a.elapsed_time(b)
        e_ms = max_over_ranks(e_ms)
        res["e2e"] = {"value": ws * steps / (e_ms * 1e-3), "unit": "evals/s", "h2d_bytes_per_step": s.n * 32,
                      "d2h_bytes_per_step": s.n * 32 + (16 if vir else 8)}

        # FP64 GPU form at the same SKP (the baseline the tensor path must beat)
        if args.fp64_steps > 0:
            plan.set_precision("fp64")
            step()
            torch.cuda.synchronize()
            f_ms, _ = timed(args.fp64_steps)
            res["fp64_form"] = {"value": args.fp64_steps / (f_ms * 1e-3), "unit": "evals/s",
                                "ms_per_step": f_ms / args.fp64_steps, "steps": args.fp64_steps}
            plan.set_precision(args.precision)

    if rank == 0:
        step()
        torch.cuda.synchronize()
        res["_gpu_out"] = (out["dEdq"].cpu().numpy(), out["forces"].cpu().numpy())
    res["_system"] = s
    plan.close()
    return res


# ncu tensor-pipe activity of the SKP kernels (sm__pipe_tensor_cycles_active, % of active
# cycles, one capture per kernel) with the digest of the kernel sources it was taken on.
SKP_TENSOR_ACTIVE = {
    # profiles/mp_ozf_kernel_water_k64_bf16x10.md
    ("water", "bf16x10"): {"digest": "8b97809330ffdde9",
                           "pct": {"mp_ozf_kernel<64>": 32.3, "mp_ozt_kernel<64, 8, 1> (stage 1)": 12.6}},
    # profiles/mp_ozt_kernel_large_k256_bf16x10.md (16-term groups of the same kernels; mean of
    # the captured launches: stage 1 59.7, stage 2 60.7 / 55.1, stage 3 59.1 / 59.2)
    ("large", "bf16x10"): {"digest": "c442ea68c11a0123",
                           "pct": {"mp_ozt_kernel<128, 4, 1> (stages 1, 2)": 58.5,
                                   "mp_ozt_kernel<128, 4, 0> (stage 3)": 59.1}},
}


def _tensor_active(workload, precision):
    rec = SKP_TENSOR_ACTIVE.get((workload, precision))
    if not rec or rec["digest"] != _skp_digest(workload):
        return None
    return {"pct_of_active_cycles": rec["pct"], "source": "ncu sm__pipe_tensor_cycles_active (profiles/)"}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="bf16x10")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed evaluations of the FP64 GPU form (default 1 for the 10^6-charge box, else 5)")
    ap.add_argument("--no-water", action="store_true", help="skip the water box reported beside the headline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plan's default launch configuration")
    ap.add_argument("--skp-tol", type=float, default=None,
                    help="override the workload's SKP tolerance (a smaller SKP, for profiling captures of the "
                         "same kernels on less device memory; not a benchmark setting)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file: a matching entry is applied without timing, a new choice is "
                         "appended (a profiling run then repeats the configuration of the plain run)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    if args.fp64_steps is None:
        args.fp64_steps = 1 if args.workload == "large" else 5
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)

    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = _init_dist(dev)
    from paper_2601_18838_gb300 import build as _build
    if rank == 0:
        _build.build()
    if pg:
        pg.barrier()
    ctx = (pg, dev, rank, ws, local)
    m = _measure(args, args.workload, args.steps, args.warmup, ctx, headline=True)
    water = None
    if args.workload != "water" and not args.no_water:
        w = _measure(args, "water", max(args.steps, 20), args.warmup, ctx, headline=False)
        water = {k: w[k] for k in ("value", "unit", "ms_per_step", "roofline", "executed", "tensor_pipe_active",
                                   "particle_kernels", "profile_ms_per_step", "skp_rank", "autotune") if k in w}
        water["workload"] = WORKLOAD_TEXT["water"]
        if rank == 0 and not args.no_cpu_baseline:
            water["cpu_baseline"] = cpu_baseline(w["_system"], budget_s=10.0, max_evals=3, gpu_out=w["_gpu_out"])
    if rank == 0:
        cb = None if args.no_cpu_baseline else cpu_baseline(m["_system"], gpu_out=m["_gpu_out"])
        line = {
            "metric": METRIC, "value": m["value"], "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE.get(args.precision, args.precision), "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "precision": args.precision,
                       "skp_rank": m["skp_rank"], "skp_r0": m["skp_r0"], "skp_rel_err": m["skp_rel_err"],
                       "autotune": m["autotune"],
                       "l2": "flushed between steps (256 MB write outside the timed events)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "tflops_useful": m["tflops_useful"], "roofline": m["roofline"], "executed": m.get("executed"),
            "tensor_pipe_active": m.get("tensor_pipe_active"),
            "particle_kernels": m["particle_kernels"], "e2e": m.get("e2e"),
            "gpu_launches": int(round(m["launches_per_step"] * args.steps)),
            "fp64_form": m.get("fp64_form"), "clocks": m["clocks"], "cpu_baseline": cb,
            "profile_ms_per_step": m["profile_ms_per_step"], "water_box": water,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
