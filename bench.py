"""Throughput of the hybrid DH step (Sec. 2, Eq. 5 and the procedure of
Sec. 2.3) on one GB300, printed as one JSON line.

A bench "step" is one full step of the integrator (both kicks with the fused
encounter search, Kepler drift, rigorous test, sets, Hermite, drifts) over the
whole workload. Default workload: the 16384-body disk (4 planets + 16380
planetesimals of 1e-10, seed 1, tau = P(a=5)/40) with the mixed-precision
kick; --prec fp64 runs the plain FP64 kick instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                  [--impl ours|reference] [--workload NAME]

--impl reference times the plain FP64 CPU oracle (the only reference this
method has here) on the host cores, on the same workload (a bounded sample
above 32768 bodies). With several GPUs (torchrun) a single disk's step is
split over them (contiguous row blocks, NCCL all-gathers between the phases;
strong scaling), while the ensemble's ranks integrate batches of their own
(weak scaling); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "disk_16384": ("disk_16384", "16384-body disk: 4 planets + 16380 planetesimals (1e-10), seed 1"),
    "disk_260": ("disk_260", "260-body disk: 4 planets + 256 planetesimals (1e-9), seed 0"),
    "disk_262144": ("disk_262144", "262144-body embryo disk: 64 embryos (1e-6) + 262080 planetesimals (1e-11), seed 2"),
    "ensemble_512": ("ensemble", "512 systems, N uniform 64-4096: 2 planets (1e-3 at a=1, 1.6) + planetesimals (1e-9), seed 3"),
}
METRIC = "particle-steps/s"
# E_Kep alone on massless test particles: a "step" is one Kepler drift of
# every particle; the learned guess is compared with the standard one
# the whole-system Hermite (Sec. 2.3, last paragraph): every step of these
# switches (two Jupiter-mass planets 0.8 AU apart)
WHOLE_WORKLOADS = {
    "planet_encounter_16384": (16381, "two Jupiter-mass planets at a = 5 and 5.6 AU, 0.12 rad "
                                      "apart, + 16381 planetesimals (1e-9, a 8-14 AU), seed 9; "
                                      "whole_hermite = 1"),
}
KEPLER_WORKLOADS = {
    "kepler_1m": "1,048,576 massless test particles about a unit star: a log-uniform 0.5-50, "
                 "e uniform 0-0.9, seed 4; tau = P(a=5)/40; E_Kep only",
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _workload(name):
    from paper_1007_3458_gb300 import workloads as W
    fn, desc = WORKLOADS[name]
    return getattr(W, fn)(), desc


def rank_workload(name, rank, world, **kw):
    """The workload one rank integrates. The ensemble's systems are independent
    problems: with several ranks each rank draws its own batch of the same
    shape (seed 3 + 1000 rank; rank 0 keeps the reference batch), so the work
    per GPU is fixed (weak scaling) and no data crosses ranks. A single system
    is the same on every rank: its step is split over the ranks (run_split)."""
    from paper_1007_3458_gb300 import workloads as W
    fn, desc = WORKLOADS[name]
    if fn == "ensemble" and world > 1:
        kw = dict(kw, seed=kw.get("seed", 3) + 1000 * rank)
        return getattr(W, fn)(**kw), desc + f" (rank {rank}: seed {kw['seed']})"
    return getattr(W, fn)(**kw), desc


def sum_over_ranks(x, device="cpu"):
    """Sum of x over the ranks of the default process group (x with one
    rank): the units all ranks processed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x, device="cpu"):
    """Largest x over the ranks of the default process group (x itself with
    one rank): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 4 + k and r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# FP64-pipe warp instructions of one k_kepler launch on the 1,048,576 test
# particles (ncu sm__inst_executed_pipe_fp64.sum), per (solver, guess, source
# digest of kepler.cu + mlp.cuh)
KEPLER_FP64_WARP_INST = {
    ("newton32", "standard", "52815e32767a71e8"): 12070789,
    ("newton", "standard", "52815e32767a71e8"): 23102409,
}

# DRAM bytes (read + written) per launch of the mixed kick, from one ncu
# capture of each workload's kick after autotuning (dram__bytes_read.sum +
# dram__bytes_write.sum, the mean over the launches of the first steps, both
# kinds of kick where the step has both); keyed by (workload, rows per CTA, j-splits, digest of the
# kick's source at the capture), since the partial-sum slots written grow
# with the splits. A shape or a kick source not captured reports null (the
# capture commands sit with the ncu summaries under profiles/).
KICK_DRAM_BYTES = {
    ("disk_16384", 256, 64, "3d6b39905dba5b88"): 9.17e5,
    ("disk_16384", 256, 128, "3d6b39905dba5b88"): 1.24e6,
    ("disk_262144", 256, 64, "3d6b39905dba5b88"): 2.35e7,
    ("disk_262144", 512, 64, "3d6b39905dba5b88"): 1.85e7,
}


def probe_peaks(q, dev, reps=5):
    """Measured FMA throughput of this GPU (qym_probe_fma: long chains of
    independent FFMA, packed FFMA2 and DFMA on every SM, CUDA events): the
    best of `reps` launches of each after one untimed launch, with the SM
    clock sampled meanwhile. The FP32 pipe peak is the larger of the scalar
    and the packed figure."""
    out = {}
    with ClockSampler(dev) as clk:
        for name, kind, iters in (("ffma", 0, 1 << 17), ("ffma2", 1, 1 << 16),
                                  ("dfma", 2, 1 << 12)):
            q.qym_probe_fma(kind, iters)
            best = max(q.qym_probe_fma(kind, iters)[0] for _ in range(reps))
            out[name] = best
    out["fp32"] = max(out["ffma"], out["ffma2"])
    out["clocks"] = clk.summary()
    out["how"] = ("qym_probe_fma: 4 x SMs CTAs of 256 threads, 8 independent FMA chains per "
                  "thread, best of %d launches (CUDA events)" % reps)
    return out


def source_digest(*names):
    """sha256 (first 16 hex digits) of kernel sources, so that a DRAM traffic
    figure captured for one version of a kernel is not reported for another."""
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1007_3458_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(w, n_max=8192):
    """The oracle on a bounded sample of the workload: returns (one_step,
    bodies, scale, description, sample_bodies). one_step() advances the sample
    by one whole step; a step of the full workload costs `scale` times that. A
    batch is sampled by whole systems (its first 8, stepped one after
    another); beyond n_max bodies a single disk is sampled by a random subset
    of the same disk (one oracle step costs ~N^2 pair evaluations: two kicks
    and the all-pairs encounter test), its time scaled by (N/n)^2."""
    import oracle as O
    O.build()
    from paper_1007_3458_gb300 import workloads as W
    prm = O.params(eps_H=w.eps_H)
    if w.nsys > 1:
        rows = [(int(w.offsets[s]), int(w.offsets[s + 1])) for s in range(min(w.nsys, 8))]
        st = {}
        for a, b in rows:
            st[a] = (w.q[a:b].copy(), O.helio_to_dh(w.m[a:b], w.v[a:b]))

        def one_step():
            for a, b in rows:
                qq, vv = st[a]
                r = O.step(w.m[a:b], qq, vv, [0, b - a], w.tau, 1, prm)
                st[a] = (r.q, r.v)
        nb = sum(b - a - 1 for a, b in rows)
        return one_step, nb, 1.0, f"the first {len(rows)} systems ({nb} bodies)", nb
    n_full = w.n_bodies
    n_s = min(n_full, n_max)
    ws = w if n_s == n_full else W.subsample(w, n_s, seed=0)
    st = [ws.q.copy(), O.helio_to_dh(ws.m, ws.v)]

    def one_step():
        r = O.step(ws.m, st[0], st[1], ws.offsets, w.tau, 1, prm)
        st[0], st[1] = r.q, r.v
    if n_s == n_full:
        return one_step, n_full, 1.0, "the whole workload", n_full
    return (one_step, n_full, (n_full / n_s) ** 2,
            f"a {n_s}-body random subsample of the disk, time scaled by (N/n)^2 to the "
            f"{n_full}-body disk", n_s)


def cpu_baseline(w, threads=1, max_seconds=20.0, n_max=8192):
    """The oracle's particle-steps/s on a bounded sample (oracle_sample), whole
    steps until about max_seconds have passed (at most 50), on `threads`
    threads (its loops over bodies; results identical for any count)."""
    import oracle as O
    one_step, nb, scale, what, ns = oracle_sample(w, n_max)
    O.set_threads(threads)
    try:
        t0 = time.perf_counter()
        steps = 0
        while steps < 1 or (time.perf_counter() - t0 < max_seconds and steps < 50):
            one_step()
            steps += 1
        raw = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    dt = raw * scale
    return {"value": nb * steps / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"{steps} steps of {what} (plain FP64 oracle, "
                      + ("single thread)" if threads == 1 else f"its body loops on {threads} threads)"),
            "sample_value": ns * steps / raw, "scaled": scale != 1.0}


def run_reference_kepler(args):
    """The oracle's Kepler drift of test particles, single thread, on a
    bounded sample (the first 20000 particles per step): W untimed drifts, then
    K timed ones."""
    import oracle as O
    from paper_1007_3458_gb300 import workloads as W
    O.build()
    qq, vv, dt = W.test_particles(1 << 20, seed=4)
    cores = host_cores()
    m = 100000 * cores
    solver = 1 if args.solver == "newton" else 0
    O.set_threads(cores)
    for _ in range(args.warmup):
        O.kepler_drift(qq[:m], vv[:m], 1.0, dt, solver=solver)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.kepler_drift(qq[:m], vv[:m], 1.0, dt, solver=solver)
    cdt = time.perf_counter() - t0
    O.set_threads(1)
    value = m * args.steps / cdt
    cb = {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
          "sample": f"first {m} particles, {args.steps} timed drifts after {args.warmup} untimed, "
                    f"standard guess (plain FP64 oracle, its body loop on {cores} threads)"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * len(qq) / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "description": KEPLER_WORKLOADS[args.workload],
                       "solver": args.solver, "guess": "standard", "l2": "n/a (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference(args):
    """The reference arm: the oracle on the host cores (its loops over bodies
    on every core; results identical to one thread), on this arm's workload
    and metric. W untimed steps, then K timed steps, each a step of the whole
    workload up to 32768 bodies, else of a random subsample scaled by (N/n)^2
    (oracle_sample)."""
    import oracle as O
    ws, rank = _dist()
    if rank != 0:
        return 0
    if args.workload in KEPLER_WORKLOADS:
        return run_reference_kepler(args)
    w, desc = _workload(args.workload)
    t_all = time.perf_counter()
    cores = host_cores()
    one_step, nb, scale, what, ns = oracle_sample(w, 32768)
    O.set_threads(cores)
    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    raw = time.perf_counter() - t0
    O.set_threads(1)
    dt = raw * scale
    value = nb * args.steps / dt
    cb = {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
          "sample": f"{args.steps} timed steps (after {args.warmup} untimed) of {what} "
                    f"(plain FP64 oracle, its body loops on {cores} threads)",
          "sample_value": ns * args.steps / raw}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "description": desc, "kick": "fp64",
                       "l2": "n/a (CPU)",
                       "sampling": ("none: every step is a step of the whole workload"
                                    if scale == 1.0 else
                                    f"each step is a step of a {ns}-body subsample; time scaled "
                                    f"by (N/n)^2 = {scale:.4g}"),
                       "sample_bodies": ns},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line))
    return 0


def precision_compare(q, torch, w, args, dev):
    """The paper's FP64 kick beside the FP32-compensated one on the same
    workload: each runs 2 untimed steps, then S timed steps from there; reported
    are its particle-steps/s and the relative energy change over those steps
    (the largest and the median over the systems), and for one system the mixed kick's
    per-particle |a - a_FP64| / |a_FP64| at the mixed run's final positions."""
    S = 2 if w.n_bodies > 100000 else max(1, min(args.steps, 20))
    out = {"steps": S}
    qfin = None
    for name, prec in (("mixed", q.QYM_KICK_MIXED), ("fp64", q.QYM_KICK_FP64)):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, device=dev,
                           l2_flush_bytes=256 << 20, eps_H=w.eps_H)
        if args.autotune:
            q.qym_autotune(sim.ctx)
        stream = torch.cuda.ExternalStream(q.qym_get_stream(sim.ctx))
        sim.step(w.tau, 2)
        E0 = np.asarray(sim.energy(), dtype=np.float64)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(w.tau, S)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        E1 = np.asarray(sim.energy(), dtype=np.float64)
        rel_e = np.abs(E1 - E0) / np.abs(E0)
        out[name] = {"value": w.n_bodies * S / (ms / 1e3), "ms_per_step": ms / S,
                     "energy_rel_err": float(np.max(rel_e)),
                     "energy_rel_err_median": float(np.median(rel_e))}
        if name == "mixed":
            qfin = sim.state()[0]
        sim.close()
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    if w.nsys == 1:
        rows = len(w.m)
        md = torch.tensor(w.m, dtype=torch.float64, device="cuda")
        qd = torch.tensor(np.ascontiguousarray(qfin.T), dtype=torch.float64, device="cuda")
        acc = {}
        for name, prec in (("mixed", q.QYM_KICK_MIXED), ("fp64", q.QYM_KICK_FP64)):
            ad = torch.empty_like(qd)
            work = torch.empty(q.qym_accel_workspace_bytes(rows, prec), dtype=torch.uint8,
                               device="cuda")
            q.qym_accel_dev(rows, md, qd, ad, 1.0, prec, work)
            torch.cuda.synchronize()
            acc[name] = ad.cpu().numpy().T[1:]
        n = np.linalg.norm(acc["fp64"], axis=1)
        rel = np.linalg.norm(acc["mixed"] - acc["fp64"], axis=1) / n
        out["accel_rel_err_max"] = float(rel.max())
        out["accel_rel_err_p99"] = float(np.percentile(rel, 99))
    return out


def run_split(args):
    """One system's step split over the job's GPUs (paper_1007_3458_gb300.split):
    every rank holds the whole disk and computes its block of rows; the
    exchanges between the phases go through NCCL all-gathers. The total work
    is fixed whatever the number of GPUs (strong scaling). --split 1 runs this
    path on one GPU too."""
    import torch
    import torch.distributed as dist
    ws, rank = _dist()
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29517")
        dist.init_process_group("nccl", rank=rank, world_size=ws)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import paper_1007_3458_gb300 as q
    from paper_1007_3458_gb300 import split as SP
    q.build()
    w, desc = _workload(args.workload)
    if w.nsys != 1:
        raise SystemExit("the split step is for a single system")
    prec = q.QYM_KICK_MIXED if args.prec == "mixed" else q.QYM_KICK_FP64
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, device=dev, eps_H=w.eps_H)
    if args.autotune:
        q.qym_autotune(sim.ctx)
    eng = SP.GpuEngine(sim, rank, ws)
    run = SP.SplitRun(eng, SP.TorchComm())
    run.step(w.tau, max(args.warmup, 3))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        dist.barrier()
        torch.cuda.synchronize()

    # timed region: K steps, each after writing 256 MB (L2 is 129 MB), host
    # time around them with the device synchronised on both sides, max over ranks
    with ClockSampler(dev) as clk:
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            run.step(w.tau, 1)
        barrier()
        ms = 1e3 * (time.perf_counter() - t0)
    ms = max_over_ranks(ms, "cuda")
    st = sim.stats()
    nb = w.n_bodies
    value = nb * args.steps / (ms / 1e3)
    lo, hi = eng.own
    k1_ms, pairs_all = q.qym_time_kick(sim.ctx, 1, 10)
    k2_ms, _ = q.qym_time_kick(sim.ctx, 0, 10)
    own_pairs = (hi - lo) * (nb - 1)
    kick_ms = 0.5 * (k1_ms + k2_ms)
    probe = probe_peaks(q, dev)
    achieved = 20.0 * own_pairs / (kick_ms / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "k_kick_mixed" if prec else "k_kick_fp64",
            "achieved": achieved, "peak": probe["fp32"] if prec else probe["dfma"],
            "unit": "TFLOP/s", "traffic": None, "peak_probe": probe,
            "convention": "20 flop per ordered pair of this rank's rows, mean of the searching "
                          "and the plain kick"}
    roof["frac"] = achieved / roof["peak"]
    # end to end: the state from pinned host memory, one split step, back
    q0h, v0h = sim.state()
    qh = torch.empty(q0h.shape, dtype=torch.float64, pin_memory=True).numpy()
    vh = torch.empty(v0h.shape, dtype=torch.float64, pin_memory=True).numpy()
    qh[:] = q0h
    vh[:] = v0h
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(qh, vh)
        run.step(w.tau, 1)
        qh, vh = q.qym_get_state(sim.ctx, qh, vh)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda")
    e2e = {"value": nb * e2e_steps / e2e_s, "unit": METRIC,
           "h2d_bytes_per_step": int(qh.nbytes + vh.nbytes),
           "d2h_bytes_per_step": int(qh.nbytes + vh.nbytes), "steps": e2e_steps,
           "what": "qym_set_state + one split step + qym_get_state per step on every rank"}
    sim.close()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    cb = None
    if ws == 1:
        # the oracle on every host core (its loops over bodies; the same bits
        # as one thread), and beside it on one thread
        cb = cpu_baseline(w, host_cores(), max_seconds=args.cpu_seconds, n_max=32768)
        cb["single_thread"] = cpu_baseline(w, 1, max_seconds=args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "fp32-pair/f64-state" if prec else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "kick": args.prec,
                       "parallelism": f"one system split over {ws} GPU(s): contiguous row "
                                      "blocks, NCCL all-gathers between the phases",
                       "tau": w.tau, "bodies": nb, "eps_H": w.eps_H, "own_rows": [lo, hi],
                       "l2": "flushed: 256 MB written before every step, inside the timed region",
                       "timing": "host clock around K one-step runs, device synchronised on "
                                 "both sides, max over ranks"},
            "stats": st, "gpu_launches": int(st["launches"]) * args.steps,
            "roofline": roof, "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cb}
    print(json.dumps(line))
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    ws, rank = _dist()
    if args.split or (ws > 1 and WORKLOADS[args.workload][0] != "ensemble"):
        return run_split(args)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import paper_1007_3458_gb300 as q
    q.build()
    w, desc = rank_workload(args.workload, rank, ws)
    prec = q.QYM_KICK_MIXED if args.prec == "mixed" else q.QYM_KICK_FP64
    # every step starts by writing 256 MB (twice the 129 MB L2), inside the
    # timed region, so no step reuses the previous step's lines
    search = {"binned": q.QYM_SEARCH_BINNED, "fused": q.QYM_SEARCH_FUSED,
              "auto": q.QYM_SEARCH_AUTO, "escape": q.QYM_SEARCH_ESCAPE}[args.search]
    sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, device=dev,
                       l2_flush_bytes=256 << 20, eps_H=w.eps_H, merge_kicks=args.merge_kicks,
                       search=search, hermite_cluster=args.hermite_cluster)
    if args.shape:
        q.qym_set_kick_shape(sim.ctx, *[int(x) for x in args.shape.split(",")])
    elif args.autotune:
        q.qym_autotune(sim.ctx)
    if args.kick_only:
        # a few launches of the kick kernels alone (for a profiler capture)
        q.qym_time_kick(sim.ctx, 1, 2)
        q.qym_time_kick(sim.ctx, 0, 2)
        torch.cuda.synchronize()
        sim.close()
        return 0
    stream = torch.cuda.ExternalStream(q.qym_get_stream(sim.ctx))
    # warm-up (also captures the step graph)
    sim.step(w.tau, max(args.warmup, 3))
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K steps inside one call, events on the context's stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        barrier()
        e0.record(stream)
        sim.step(w.tau, args.steps)
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    st = sim.stats()
    nb = w.n_bodies
    nb_all = sum_over_ranks(nb, "cuda")
    value = nb_all * args.steps / (ms / 1e3)
    pairs = w.pairs_per_kick()
    gpair = 2 * sum_over_ranks(pairs, "cuda") * args.steps / (ms / 1e3) / 1e9

    # dominant kernel: the all-pairs kick, timed alone on the same stream
    reps = 20
    k1_ms, _ = q.qym_time_kick(sim.ctx, 1, reps)
    k2_ms, _ = q.qym_time_kick(sim.ctx, 0, reps)
    # the step's two kicks: with the binned search both are plain; with the
    # fused one the first carries the search
    sim_search = sim.effective_params().search
    binned = sim_search == q.QYM_SEARCH_BINNED
    kick_ms = k2_ms if binned else 0.5 * (k1_ms + k2_ms)
    achieved = 20.0 * pairs / (kick_ms / 1e3) / 1e12
    clocks = clk.summary()
    probe = probe_peaks(q, dev)
    peak = probe["fp32"] if prec else probe["dfma"]
    digest = source_digest("kick.cu")
    roof = {"bound": "alu", "kernel": "k_kick_mixed" if prec else "k_kick_fp64",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": "measured (qym_probe_fma, %s)" % ("FP32 FMA pipe" if prec else "FP64"),
            "peak_probe": probe,
            "traffic": (KICK_DRAM_BYTES.get((args.workload, st["kick_tile_i"], st["kick_tile_splits"],
                                             digest)) if prec else None),
            "traffic_unit": "bytes per launch (ncu)", "kick_source_digest": digest,
            "convention": ("20 flop per ordered pair over the plain kick's launch time (the "
                           "binned search leaves both kicks of a step plain)" if binned else
                           "20 flop per ordered pair over the mean launch time of the searching "
                           "and the plain kick"),
            "kick_ms_with_search": k1_ms, "kick_ms_plain": k2_ms,
            "frac_with_search": 20.0 * pairs / (k1_ms / 1e3) / 1e12 / peak,
            "frac_plain": 20.0 * pairs / (k2_ms / 1e3) / 1e12 / peak,
            "gpair_per_s_kernel": pairs / (kick_ms / 1e3) / 1e9,
            "kick_shape": {"rows_per_cta": st["kick_tile_i"], "splits": st["kick_tile_splits"]}}

    # E_Dft alone (the momentum reduction and the drift with the kick's packs)
    # against HBM; the state is put back
    edft = edft_roofline(q, sim, w)

    # end to end through the C ABI with host buffers: per step, the state goes
    # host -> device (qym_set_state), one step, device -> host (qym_get_state),
    # the state in pinned host memory
    q0h, v0h = sim.state()
    qh = torch.empty(q0h.shape, dtype=torch.float64, pin_memory=True).numpy()
    vh = torch.empty(v0h.shape, dtype=torch.float64, pin_memory=True).numpy()
    qh[:] = q0h
    vh[:] = v0h
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(qh, vh)
        sim.step(w.tau, 1)
        qh, vh = q.qym_get_state(sim.ctx, qh, vh)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda")
    e2e = {"value": nb_all * e2e_steps / e2e_s, "unit": METRIC,
           "h2d_bytes_per_step": int(qh.nbytes + vh.nbytes),
           "d2h_bytes_per_step": int(qh.nbytes + vh.nbytes),
           "steps": e2e_steps,
           "what": "qym_set_state + qym_step(tau, 1) + qym_get_state per step, pinned host state"}
    sim.close()
    # the same steps with the two kicks between steps merged into one (an exact
    # rewrite, reported beside the paper's two kicks per step)
    merged = None
    if not args.merge_kicks and args.merged_too:
        sm = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, device=dev,
                          l2_flush_bytes=256 << 20, eps_H=w.eps_H, merge_kicks=1, search=search)
        if args.autotune:
            q.qym_autotune(sm.ctx)
        sms = torch.cuda.ExternalStream(q.qym_get_stream(sm.ctx))
        sm.step(w.tau, max(args.warmup, 3))
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(sms)
        sm.step(w.tau, args.steps)
        f1.record(sms)
        barrier()
        mms = max_over_ranks(f0.elapsed_time(f1), "cuda")
        sst = sm.stats()
        merged = {"value": nb_all * args.steps / (mms / 1e3), "ms_per_step": mms / args.steps,
                  "kicks_per_step": 1, "launches": int(sst["launches"]),
                  "candidates": int(sst["candidates"]), "encounters": int(sst["encounters"]),
                  "rescans": int(sst["rescans"]), "hermite_steps_max": int(sst["hermite_steps_max"])}
        sm.close()
    # the same steps with the other encounter search (binned after the drift /
    # fused into the first kick), for comparison
    other = None
    if args.search_too:
        alt = q.QYM_SEARCH_FUSED if binned else q.QYM_SEARCH_BINNED
        so = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, device=dev,
                          l2_flush_bytes=256 << 20, eps_H=w.eps_H, merge_kicks=args.merge_kicks,
                          search=alt)
        if args.autotune:
            q.qym_autotune(so.ctx)
        sos = torch.cuda.ExternalStream(q.qym_get_stream(so.ctx))
        so.step(w.tau, max(args.warmup, 3))
        barrier()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(sos)
        so.step(w.tau, args.steps)
        g1.record(sos)
        barrier()
        oms = max_over_ranks(g0.elapsed_time(g1), "cuda")
        ost = so.stats()
        other = {"search": "fused" if alt == q.QYM_SEARCH_FUSED else "binned",
                 "value": nb_all * args.steps / (oms / 1e3), "ms_per_step": oms / args.steps,
                 "candidates": int(ost["candidates"]), "encounters": int(ost["encounters"]),
                 "rescans": int(ost["rescans"]), "launches": int(ost["launches"]),
                 "hermite_steps_max": int(ost["hermite_steps_max"])}
        so.close()
    precision = None
    if args.precision_too and ws == 1 and prec == q.QYM_KICK_MIXED:
        precision = precision_compare(q, torch, w, args, dev)
    if rank != 0:
        return 0
    cb = None
    if ws == 1:
        # the oracle on every host core (its loops over bodies; the same bits
        # as one thread), and beside it on one thread
        cb = cpu_baseline(w, host_cores(), max_seconds=args.cpu_seconds, n_max=32768)
        cb["single_thread"] = cpu_baseline(w, 1, max_seconds=args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32-pair/f64-state" if prec else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "kick": args.prec,
                       "search": {q.QYM_SEARCH_BINNED: "binned", q.QYM_SEARCH_ESCAPE: "escape"}.get(
                           sim_search, "fused"),
                       "parallelism": ("independent batches per rank" if ws > 1 and
                                       WORKLOADS[args.workload][0] == "ensemble" else
                                       "replicas" if ws > 1 else "single GPU"),
                       "tau": w.tau, "bodies": nb, "eps_H": w.eps_H,
                       "l2": "flushed: 256 MB written at the start of every step, inside the timed region"},
            "gpair_per_s": gpair, "stats": st, "gpu_launches": int(st["launches"]),
            "kicks_per_step": 1 if args.merge_kicks else 2, "merged_kicks": merged,
            "other_search": other,
            "precision": precision,
            "roofline": roof, "edft": edft, "clocks": clocks, "e2e": e2e, "cpu_baseline": cb}
    print(json.dumps(line))
    return 0


def run_sweep(args):
    """Sensitivity of the step to the Hill factors (Sec. 3.3: a_E sets the
    encounter detection radius, a_H the transition radius r_crit): for each
    pair, the same K steps from the workload's initial state, with the relative
    energy change over them, the particle-steps/s and the encounter work."""
    import torch
    import paper_1007_3458_gb300 as q
    q.build()
    w, desc = rank_workload(args.workload, 0, 1)
    a_Es = [float(x) for x in args.sweep_a_e.split(",")]
    a_Hs = [float(x) for x in args.sweep_a_h.split(",")]
    points = []
    for aE in a_Es:
        for aH in a_Hs:
            sim = q.Simulation(w.m, w.q, w.v, w.offsets, eps_H=w.eps_H, a_E=aE, a_H=aH)
            stream = torch.cuda.ExternalStream(q.qym_get_stream(sim.ctx))
            E0 = np.asarray(sim.energy(), dtype=np.float64)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(w.tau, args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            E1 = np.asarray(sim.energy(), dtype=np.float64)
            st = sim.stats()
            sim.close()
            points.append({"a_E": aE, "a_H": aH,
                           "energy_rel_err": float(np.max(np.abs(E1 - E0) / np.abs(E0))),
                           "value": w.n_bodies * args.steps / (ms / 1e3),
                           "encounters": int(st["encounters"]), "sets": int(st["sets"]),
                           "max_set": int(st["max_set"]), "hermite_steps": int(st["hermite_steps"]),
                           "status_bits": int(st["status_bits"])})
    print(json.dumps({"metric": "energy error and particle-steps/s against a_E, a_H",
                      "unit": METRIC, "steps": args.steps, "data": "synthetic",
                      "config": {"workload": args.workload, "description": desc, "kick": "mixed",
                                 "tau": w.tau, "eps_H": w.eps_H},
                      "points": points}))
    return 0


# E_Dft's algorithmic bytes per row: the reduction reads m and v (32 B); the
# drift reads Q and writes it (48 B) and writes the kick's float packs (32 B)
EDFT_MOMENTUM_BYTES = 32
EDFT_DRIFT_BYTES = 80


def edft_roofline(q, sim, w, reps=20):
    """E_Dft (Sec. 2, Eq. 2) timed alone through qym_time_drift (CUDA events on
    the context's stream, the state put back): achieved GB/s of its two
    launches against the measured HBM copy bandwidth."""
    mom_ms, drift_ms = q.qym_time_drift(sim.ctx, w.tau, reps)
    rows = len(w.m)
    peak, which = hbm_peak_gbs()
    out = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": which, "rows": rows}
    for name, ms, bpr in (("momentum", mom_ms, EDFT_MOMENTUM_BYTES),
                          ("drift", drift_ms, EDFT_DRIFT_BYTES)):
        gbs = rows * bpr / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "bytes_per_row": bpr, "achieved": gbs, "frac": gbs / peak}
    return out


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_whole(args):
    """Steps that switch to the whole-system Hermite (whole.cu): time per step
    (the host drives the block steps and reads the sets back each step, so
    the step is timed on the host clock around synchronised calls), block
    steps per step, and the energy error beside the hybrid step's."""
    import torch
    import paper_1007_3458_gb300 as q
    from paper_1007_3458_gb300 import workloads as W
    q.build()
    npl, desc = WHOLE_WORKLOADS[args.workload]
    w = W.planet_encounter(n_planetesimals=npl, name=args.workload)
    prec = q.QYM_KICK_MIXED if args.prec == "mixed" else q.QYM_KICK_FP64
    out = {}
    for label, wh in (("whole", 1), ("hybrid", 0)):
        sim = q.Simulation(w.m, w.q, w.v, w.offsets, kick_prec=prec, eps_H=w.eps_H,
                           whole_hermite=wh)
        E0 = sim.energy()[0]
        sim.step(w.tau, args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(w.tau, args.steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = sim.stats()
        E1 = sim.energy()[0]
        sim.close()
        out[label] = {"ms_per_step": 1e3 * dt / args.steps,
                      "value": len(w.m[1:]) * args.steps / dt,
                      "whole_steps": int(st["whole_steps"]),
                      "hermite_block_steps": int(st["hermite_steps"]),
                      "us_per_block_step": (1e6 * dt / st["hermite_steps"]
                                            if wh and st["hermite_steps"] else None),
                      "launches": int(st["launches"]),
                      "energy_error_after": abs(E1 / E0 - 1.0), "status": int(st["status_bits"])}
    head = out["whole"]
    line = {"metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (whole-system Hermite)", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "tau": w.tau,
                       "kick": args.prec, "timing": "host clock around synchronised qym_step "
                       "calls (the switch reads the sets back every step)"},
            "compare": out, "gpu_launches": head["launches"]}
    print(json.dumps(line))
    return 0


def run_kepler(args):
    """E_Kep of 1,048,576 test particles (Appendix): timed drifts with the
    standard and the learned starting guess."""
    import torch
    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.cuda.current_device()
    import paper_1007_3458_gb300 as q
    from paper_1007_3458_gb300 import guess as G
    from paper_1007_3458_gb300 import workloads as W
    q.build()
    solver = {"newton": q.QYM_SOLVER_NEWTON, "newton32": q.QYM_SOLVER_NEWTON32,
              "laguerre": q.QYM_SOLVER_LAGUERRE}[args.solver]
    t_train = time.perf_counter()
    if args.train:
        wts, losses, nrows = G.train_default()
    else:
        # standard guess only (a quick run, e.g. for a profiler capture)
        wts, losses, nrows = np.zeros(q.QYM_MLP_NW, np.float32), np.zeros(100, np.float32), 0
        args.guess = "standard"
    t_train = time.perf_counter() - t_train
    qq, vv, dt = W.test_particles(1 << 20, seed=4)
    n = len(qq)
    q0 = torch.from_numpy(np.ascontiguousarray(qq.T)).cuda()
    v0 = torch.from_numpy(np.ascontiguousarray(vv.T)).cuda()
    q1, v1 = torch.empty_like(q0), torch.empty_like(v0)
    wd = torch.from_numpy(wts).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def drift(guess, x=None, it=None, st=None, slv=None):
        q.qym_kepler_drift_dev(n, q0, v0, q1, v1, 1.0, dt, solver if slv is None else slv, guess,
                               wd if guess == q.QYM_GUESS_MLP else None, 50, x_out=x,
                               iters=it, status=st)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    res = {}
    # the headline (solver, guess) first, then the other solvers and guesses
    # for comparison, each timed the same way
    solvers = {"newton": q.QYM_SOLVER_NEWTON, "newton32": q.QYM_SOLVER_NEWTON32,
               "laguerre": q.QYM_SOLVER_LAGUERRE}
    guesses = (("standard", q.QYM_GUESS_STANDARD), ("learned", q.QYM_GUESS_MLP))
    arms = [(args.solver, args.guess)]
    if args.compare:
        arms += [(sn, gn) for sn in ("newton32", "newton", "laguerre") for gn, _ in guesses
                 if (sn, gn) != arms[0] and (args.train or gn == "standard")]
    for sname, name in arms:
        guess = dict(guesses)[name]
        slv = solvers[sname]
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        drift(guess, it=it, st=st, slv=slv)
        for _ in range(args.warmup):
            drift(guess, slv=slv)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with ClockSampler(dev) as clk:
            barrier()
            for a, b in ev:
                flush.fill_(1)          # L2 flushed between timed drifts (outside the events)
                a.record(stream)
                drift(guess, slv=slv)
                b.record(stream)
            barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        itn = it.cpu().numpy()
        res[f"{sname}/{name}"] = {"value": n * args.steps * ws / (ms / 1e3),
                                  "ms_per_step": ms / args.steps,
                                  "iterations_mean": float(itn.mean()),
                                  "iterations_max": int(itn.max()),
                                  "status": int(st.item()), "clocks": clk.summary()}
    head = res[f"{args.solver}/{args.guess}"]
    # the guess trained on planetary-system logs alone (no test particles):
    # Newton iterations (FP64) on the test particles, where it extrapolates,
    # and on a held-out disk of the same kind as its training disk
    variants = None
    if args.train and args.compare:
        t1 = time.perf_counter()
        w_disk, l_disk, n_disk = G.train_disk_only()
        t1 = time.perf_counter() - t1
        wdd = torch.from_numpy(w_disk).cuda()

        def iters(qq_, vv_, dt_, weights, guess):
            m_ = len(qq_)
            a0 = torch.from_numpy(np.ascontiguousarray(qq_.T)).cuda()
            b0 = torch.from_numpy(np.ascontiguousarray(vv_.T)).cuda()
            a1, b1 = torch.empty_like(a0), torch.empty_like(b0)
            it_ = torch.empty(m_, dtype=torch.int32, device="cuda")
            st_ = torch.zeros(1, dtype=torch.int32, device="cuda")
            q.qym_kepler_drift_dev(m_, a0, b0, a1, b1, 1.0, dt_, q.QYM_SOLVER_NEWTON, guess,
                                   weights, 50, iters=it_, status=st_)
            torch.cuda.synchronize()
            return float(it_.float().mean().item()), int(st_.item())

        hq, hv, htau = G.heldout_disk()
        variants = {"disk_only": {"rows": n_disk, "train_seconds": t1,
                                  "loss_first": float(l_disk[:10].mean()),
                                  "loss_last": float(l_disk[-100:].mean())},
                    "newton_iterations": {}}
        for label, (a_, b_, d_) in (("test_particles", (qq, vv, dt)),
                                    ("heldout_disk", (hq, hv, htau))):
            variants["newton_iterations"][label] = {
                "standard": iters(a_, b_, d_, None, q.QYM_GUESS_STANDARD),
                "learned_default": iters(a_, b_, d_, wd, q.QYM_GUESS_MLP),
                "learned_disk_only": iters(a_, b_, d_, wdd, q.QYM_GUESS_MLP)}
    # end to end through the C ABI with host buffers: the state goes host ->
    # device, one drift, device -> host
    hq = torch.from_numpy(np.ascontiguousarray(qq.T)).pin_memory()
    hv = torch.from_numpy(np.ascontiguousarray(vv.T)).pin_memory()
    oq, ov = torch.empty_like(hq).pin_memory(), torch.empty_like(hv).pin_memory()
    g_head = q.QYM_GUESS_MLP if args.guess == "learned" else q.QYM_GUESS_STANDARD
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        q0.copy_(hq, non_blocking=True)
        v0.copy_(hv, non_blocking=True)
        drift(g_head)
        oq.copy_(q1, non_blocking=True)
        ov.copy_(v1, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    nbytes = int(hq.numel() * 8 + hv.numel() * 8)
    e2e = {"value": n * e2e_steps * ws / e2e_s, "unit": METRIC, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
           "what": "pinned H2D of (q, v) + qym_kepler_drift_dev + D2H of (q1, v1) per step"}
    # roofline of k_kepler: bound by FP64 issue, not by its 96 bytes per
    # particle (read q0, v0, write q1, v1, float64 x 3 each). Achieved = the
    # FP64-pipe instructions ncu counted for one launch of this source (x 32
    # lanes: issue slots, divergent lanes included) over the live launch
    # time; peak = the DFMA instruction rate measured by qym_probe_fma.
    peak_gbs, which = hbm_peak_gbs()
    hbm = 96.0 * n / (head["ms_per_step"] / 1e3) / 1e9
    kdig = source_digest("kepler.cu", "mlp.cuh")
    fp64_inst = KEPLER_FP64_WARP_INST.get((args.solver, args.guess, kdig))
    pk = probe_peaks(q, dev)
    dfma_rate = pk["dfma"] / 2.0 * 1e3          # 1e9 FP64 thread-instructions/s
    achieved = fp64_inst * 32 / (head["ms_per_step"] / 1e3) / 1e9 if fp64_inst else None
    roof = {"bound": "alu", "kernel": "k_kepler<%s>" % ("true" if args.guess == "learned" else "false"),
            "achieved": achieved, "peak": dfma_rate, "unit": "G FP64 instr/s",
            "frac": achieved / dfma_rate if achieved else None,
            "peak_source": "measured (qym_probe_fma DFMA: %.3f TFLOP/s)" % pk["dfma"],
            "fp64_warp_instructions_per_launch": fp64_inst, "kepler_source_digest": kdig,
            "convention": ("FP64-pipe warp instructions of one launch (ncu "
                           "sm__inst_executed_pipe_fp64.sum, this source) x 32 over the live launch "
                           "time, against the measured DFMA thread-instruction rate; null when the "
                           "source has changed since the count was taken"),
            "traffic": None,
            "hbm": {"achieved": hbm, "peak": peak_gbs, "unit": "GB/s", "frac": hbm / peak_gbs,
                    "peak_source": which, "bytes_per_particle": 96}}
    if rank != 0:
        return 0
    cb = None
    if ws == 1:
        import oracle as O
        O.build()
        cores = host_cores()
        O.set_threads(cores)
        m2 = 200000
        t0 = time.perf_counter()
        O.kepler_drift(qq[:m2], vv[:m2], 1.0, dt, solver=0 if args.solver == "laguerre" else 1)
        cdt = time.perf_counter() - t0
        O.set_threads(1)
        cb = {"value": m2 / cdt, "unit": METRIC, "cores": cores, "kind": "oracle",
              "sample": f"first {m2} particles, one drift, standard guess (plain FP64 oracle, "
                        f"its body loop on {cores} threads)"}
        m = 20000
        t0 = time.perf_counter()
        O.kepler_drift(qq[:m], vv[:m], 1.0, dt, solver=0 if args.solver == "laguerre" else 1)
        cdt = time.perf_counter() - t0
        cb["single_thread"] = {"value": m / cdt, "unit": METRIC, "cores": 1, "kind": "oracle",
                               "sample": f"first {m} particles, one drift, standard guess (plain "
                                         "FP64 oracle, single thread)"}
    line = {"metric": METRIC, "value": head["value"], "unit": METRIC, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (bf16/f32 guess network)" if args.guess == "learned" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": KEPLER_WORKLOADS[args.workload],
                       "solver": args.solver, "guess": args.guess, "particles": n, "tau": dt,
                       "l2": "flushed: 256 MB written before every timed drift, outside the events",
                       "training": {"rows": nrows, "seconds": t_train,
                                    "loss_first": float(losses[:10].mean()),
                                    "loss_last": float(losses[-100:].mean())}},
            "compare": res, "guess_training_variants": variants,
            "gpu_launches": args.steps, "roofline": roof,
            "clocks": head["clocks"], "e2e": e2e, "cpu_baseline": cb}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="disk_16384",
                    choices=sorted(WORKLOADS) + sorted(KEPLER_WORKLOADS) + sorted(WHOLE_WORKLOADS))
    ap.add_argument("--guess", default="standard", choices=["standard", "learned"],
                    help="kepler_1m: the starting guess of the headline number")
    ap.add_argument("--compare", type=int, default=1,
                    help="kepler_1m: also time the other solvers and guesses")
    ap.add_argument("--solver", default="newton32", choices=["newton", "newton32", "laguerre"],
                    help="kepler_1m: Kepler solver (newton32: FP32 Newton steps, then FP64 Laguerre)")
    ap.add_argument("--hermite-cluster", type=int, default=0, choices=[0, 2, 4, 8],
                    help="CTAs per cluster for the large encounter sets (0: the library's choice)")
    ap.add_argument("--merge-kicks", type=int, default=0,
                    help="1: one kick of tau between steps (exact rewrite of the paper's two)")
    ap.add_argument("--merged-too", type=int, default=1,
                    help="also time the merged-kick step and report it under merged_kicks")
    ap.add_argument("--sweep", action="store_true",
                    help="run the a_E x a_H sensitivity sweep instead (one JSON line)")
    ap.add_argument("--sweep-a-e", default="1,1.5,2,2.5,3,4,6")
    ap.add_argument("--sweep-a-h", default="0.5,1,2")
    ap.add_argument("--precision-too", type=int, default=1,
                    help="also run the FP64 kick and report both kicks' energy error (and the "
                         "mixed kick's acceleration error) under precision")
    ap.add_argument("--train", type=int, default=1,
                    help="kepler_1m: train the guess network first (0: standard guess only)")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--search", default="auto", choices=["auto", "binned", "fused", "escape"],
                    help="close-encounter search: binned after the drift, fused into the kick, "
                         "the paper's escape-velocity sweep (fused into the kick), or the "
                         "library's choice for the workload")
    ap.add_argument("--shape", default="",
                    help="threads,ipt,splits: the kick's launch shape instead of autotuning")
    ap.add_argument("--search-too", type=int, default=1,
                    help="also time the other encounter search and report it under other_search")
    ap.add_argument("--split", type=int, default=0,
                    help="1: a single system's step split over the job's GPUs even on one GPU "
                         "(with several GPUs a single system always is)")
    ap.add_argument("--kick-only", action="store_true",
                    help="launch only the kick kernels a few times (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in KEPLER_WORKLOADS:
        return run_kepler(args)
    if args.workload in WHOLE_WORKLOADS:
        return run_whole(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
