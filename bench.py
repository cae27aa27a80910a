#!/usr/bin/env python3
"""Throughput of QFactor-Sample instantiation on GB300: converged
instantiations per second at cost <= 1e-8, and the sweep's HBM bandwidth
against the measured peak.

Workload (default): n = 12 qubits, brick wall of 17 two-qubit U(4) gates
(three half-layers), target built from Haar-random gates in the same
structure, M = 32 orthonormal training states, 32 multistarts, complex64
sweeps with FP64 SVD, master gates, cost check and refinement, tol 1e-8,
at most 500 sweeps.  One step = one full instantiation of one target (a new
target per step).  Inputs are synthetic and seeded (the paper's benchmark
circuits are not available); the B list (512 MiB) exceeds L2, so no flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank instantiates its own targets (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged instantiations/s at cost<=1e-8"
UNIT = "instantiations/s"

WORKLOADS = {
    # name: (factory name, precision, description)
    "brick_n12": ("brick_n12", 1, "n=12 brick wall 17 gates, M=32, 32 starts, complex64 sweeps + FP64 SVD/refine/check"),
    "brick_n8": ("brick_n8", 0, "n=8 brick wall 28 gates, M=16, 16 starts, FP64"),
    "chain_n3": ("chain_n3", 0, "n=3 chain of 4 gates, M=4, 1 start, FP64, tol 1e-10"),
    "uneven_blocks": ("uneven_blocks", 1, "4096 problems, n uniform in {3,4,5}, 2-10 nearest-neighbour gates, "
                      "M=2^(n-1), 8 starts, complex64 sweeps + FP64 check/refine, one persistent launch"),
    "qf_vs_qfs": ("qf_vs_qfs", 0, "full-unitary QFactor vs QFactor-Sample with double-and-restart, n = 3..10"),
    "states_ablation": ("states_ablation", 0, "Haar vs computational-basis training states (Appendix D): "
                        "smallest M that generalises and double-and-restart, brick walls n = 6, 8, 10"),
    "learned": ("learned", 1, "learned warm start: 4-qubit 6-gate structure, MLP 256-3x1024-192 trained on "
                "method-generated pairs; 65536 fresh targets, predicted start then 8 random starts as fallback"),
}
HW_BAD = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def _problem(kind, seed):
    from paper_2405_12866_gb300 import workloads as w
    fac = getattr(w, WORKLOADS[kind][0])
    return fac(target_seed=seed) if kind != "chain_n3" else w.chain_n3(target_seed=seed + 1)


# ------------------------------------------------------------- env / ranks

def dist_env():
    from paper_2405_12866_gb300.ranks import dist_env as _env
    return _env()


class Clocks:
    """nvidia-smi clock and throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        import tempfile
        self.path = os.environ.get("QFS_CLOCKS_CSV",
                                   os.path.join(tempfile.gettempdir(), f"qfs_clocks_rank{device_index}.csv"))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak(sustained=True):
    """Dense bf16 tensor peak (TFLOP/s) and its source."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in d else "bf16_tflops"
        return float(d[key]), "measured (" + key + ")"
    except Exception:
        return (1700.0 if sustained else 1900.0), "fallback"


KERNEL_SOURCES = {
    "k_sweep_df": ("sweep_df.cu", "polar4.cuh", "qfs_common.cuh", "qfs_kernels.h"),
    "k_batch_sweep": ("batch.cu", "polar4.cuh", "qfs_common.cuh", "qfs_kernels.h"),
    "k_backward_q4": ("kernels_sweep.cu", "polar4.cuh", "qfs_common.cuh", "qfs_kernels.h"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2405_12866_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic_record(kernel, workload):
    """DRAM bytes per launch of a kernel on a workload from the committed ncu
    summary (profiles/traffic.json), used only while the kernel's sources are
    unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("source_sha256") != kernel_source_hash(kernel) or rec.get("bench_workload") != workload:
        return None
    return rec.get("dram_bytes_per_launch")


# --------------------------------------------------------- oracle baseline

def _oracle_start_sweeps(args):
    """Worker (spawned): `sweeps` oracle sweeps of one start; returns seconds."""
    UPsi, Psi, G, pairs, n, sweeps = args
    from oracle import qfs_oracle as o
    t = time.perf_counter()
    for _ in range(sweeps):
        G = o.sweep(UPsi, Psi, G, pairs, n).gates
    return time.perf_counter() - t


def oracle_sample(kind, seed, pool=None, cores=None):
    """Time the oracle on a bounded sample of one target of the workload:
    U Psi once and one sweep of every start, the starts in parallel over
    host processes.  Returns the seconds of each part."""
    from oracle import qfs_oracle as o  # noqa: F401  (imported where it runs)
    p = _problem(kind, seed)
    Psi, G0 = p.samples(), p.init_gates()
    t0 = time.perf_counter()
    UPsi = p.U @ Psi
    t_pre = time.perf_counter() - t0
    t1 = time.perf_counter()
    pool.map(_oracle_start_sweeps, [(UPsi, Psi, G0[s], p.pairs, p.n, 1) for s in range(p.S)])
    t_sw = time.perf_counter() - t1
    return {"seconds_precompute": t_pre, "seconds_per_sweep_all_starts": t_sw, "name": p.name, "starts": p.S}


def golden_runs(kind):
    """The oracle's own full runs of this workload (tests/golden), written by
    oracle/make_golden.py: mean sweeps per instantiation, converged
    fraction, the number of targets and their seeds."""
    path = os.path.join(ROOT, "tests", "golden", f"{kind}_oracle_runs.json")
    try:
        runs = json.load(open(path))
    except Exception:
        return None
    sw = [r["sweeps"] for r in runs.values()]
    conv = [r["converged"] for r in runs.values()]
    return {"sweeps": float(np.mean(sw)), "converged": float(np.mean(conv)), "targets": len(sw),
            "seeds": sorted(int(k) for k in runs)}


def oracle_rate(samples, g):
    """Converged instantiations/s of the oracle extrapolated from timed
    samples: per target, U Psi + (mean sweeps per instantiation of the
    oracle's own full runs) x (one sweep of all starts), times the converged
    fraction of those runs."""
    t_inst = float(np.mean([x["seconds_precompute"] + x["seconds_per_sweep_all_starts"] * g["sweeps"]
                            for x in samples]))
    return g["converged"] / t_inst, t_inst


def oracle_note(g, n_samples, cores):
    return (f"extrapolated: per timed target, U Psi once + 1 sweep of all starts on {cores} host processes; "
            f"x {g['sweeps']:.2f} sweeps/instantiation and x converged fraction {g['converged']:.2f}, both "
            f"from the oracle's own full runs of {g['targets']} targets of this workload (seeds "
            f"{g['seeds'][0]}..{g['seeds'][-1]}); {n_samples} target(s) timed")


# ---------------------------------------------------------------- arms

def run_reference(args):
    """The oracle on the workload's timed targets (the same seeds as our
    arm's timed steps), one bounded sample per step."""
    from paper_2405_12866_gb300.ranks import target_seeds, warmup_seeds
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count()
    g = golden_runs(args.workload) or {"sweeps": 100.0, "converged": 1.0, "targets": 0, "seeds": [0]}
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for sd in warmup_seeds(0, args.warmup):
            oracle_sample(args.workload, sd, pool=pool, cores=cores)
        t0 = time.perf_counter()
        samples = [oracle_sample(args.workload, sd, pool=pool, cores=cores) for sd in target_seeds(0, args.steps)]
        wall = time.perf_counter() - t0
    value, t_inst = oracle_rate(samples, g)
    note = oracle_note(g, len(samples), cores)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][2], "parallelism": "host processes over starts",
                       "step": "one bounded sample per timed target: U Psi + one sweep of all starts",
                       "extrapolation": note, "seconds_per_instantiation_extrapolated": t_inst},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": note},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import qfs
    if rank == 0 or world == 1:
        qbuild.build()
    if world > 1:
        dist.barrier()
    qfs.lib()
    kind = args.workload
    prec = WORKLOADS[kind][1]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = qfs.Context(local, stream.cuda_stream)

    # Inputs of every step, generated on the host and made resident before
    # timing: the timed targets (seeds 0..K*T-1 of this rank) and separate
    # warm-up targets.  With --targets-per-call T > 1 a step is one call that
    # instantiates T targets together (their starts share the sweep launches).
    TPC = 1 if args.restart_doubling else max(1, args.targets_per_call)
    from paper_2405_12866_gb300.ranks import combine, target_seeds, warmup_seeds
    probs_t = [_problem(kind, seed) for seed in target_seeds(rank, args.steps * TPC)]
    probs_w = [_problem(kind, seed) for seed in warmup_seeds(rank, args.warmup * TPC)]
    first = probs_t[0]
    L, S, M, n = first.L, first.S, first.M, first.n

    def upload(probs):
        out = []
        for i in range(0, len(probs), TPC):
            grp = probs[i:i + TPC]
            out.append((torch.from_numpy(np.stack([p.U for p in grp])).to(dev),
                        torch.from_numpy(np.stack([p.samples() for p in grp])).to(dev),
                        torch.from_numpy(np.ascontiguousarray(np.stack([p.init_gates() for p in grp]))).to(dev)))
        return out

    dev_t, dev_w = upload(probs_t), upload(probs_w)
    out = torch.zeros((TPC, L, 4, 4), dtype=torch.complex128, device=dev)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=first.max_sweeps, dist_tol=first.tol,
                             precision=prec, start_groups=args.start_groups,
                             restart_doubling=1 if args.restart_doubling else 0, concurrent_targets=args.slots)

    def step(probs, dev_in, i):
        if args.restart_doubling:
            # double-and-restart draws its training states itself (host target)
            prm.seed = probs[i].seed
            return [ctx.instantiate(n, first.pairs, probs[i].U, prm)]
        U, Psi, G0 = dev_in[i]
        if TPC == 1:
            return [ctx.instantiate_dev(n, first.pairs, U[0], Psi[0], G0[0], prm, out[0])]
        return ctx.instantiate_many_dev(n, first.pairs, U, Psi, G0, prm, out)

    for i in range(args.warmup):
        step(probs_w, dev_w, i)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    # Timed region: K steps, kernel launches counted, no per-launch events.
    clocks = Clocks(local)
    clocks.start()
    ctx.profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    results = [r for i in range(args.steps) for r in step(probs_t, dev_t, i)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = ctx.profile_read(-1)["launches"]
    conv = sum(r.converged for r in results)
    sweeps = [r.sweeps for r in results]
    (ms_all,), (conv_all, launches_all) = combine([ms], [conv, launches], dev)
    value = conv_all / (ms_all / 1e3)

    # End to end through the public host-pointer API on the same K targets:
    # pinned host inputs, H2D of target, samples and initial gates inside
    # the call, D2H of the gates and costs.
    e2e = None
    if args.e2e:
        hin = []
        for i in range(0, len(probs_t), TPC):
            grp = probs_t[i:i + TPC]
            hin.append(tuple(torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
                             for x in (np.stack([p.U for p in grp]), np.stack([p.samples() for p in grp]),
                                       np.stack([p.init_gates() for p in grp]))))
        # One untimed call through the same host API on a warm-up target
        # (its first use sizes the context's workspace for the host copy of
        # the target), as the device path is warmed up above.
        pw = probs_w[0] if probs_w else probs_t[0]
        if args.restart_doubling:
            prm.seed = pw.seed
            ctx.instantiate(n, first.pairs, pw.U, prm)
        elif TPC == 1:
            ctx.instantiate(n, first.pairs, pw.U, prm, pw.samples(), pw.init_gates())
        else:
            grp = (probs_w if len(probs_w) >= TPC else probs_t)[:TPC]
            ctx.instantiate_many(n, first.pairs, np.stack([p.U for p in grp]), prm,
                                 np.stack([p.samples() for p in grp]), np.stack([p.init_gates() for p in grp]))
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        if args.restart_doubling:
            e2e_res = []
            for i, (U_h, Ps_h, G_h) in enumerate(hin):
                prm.seed = probs_t[i].seed
                e2e_res.append(ctx.instantiate(n, first.pairs, U_h[0], prm))
        elif TPC == 1:
            e2e_res = [ctx.instantiate(n, first.pairs, U_h[0], prm, Ps_h[0], G_h[0]) for (U_h, Ps_h, G_h) in hin]
        else:
            e2e_res = [r for (U_h, Ps_h, G_h) in hin
                       for r in ctx.instantiate_many(n, first.pairs, U_h, prm, Ps_h, G_h)]
        torch.cuda.synchronize(dev)
        t_e2e = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        conv_e2e = sum(r.converged for r in e2e_res)
        (t_e2e,), (conv_e2e,) = combine([t_e2e], [conv_e2e], dev)
        N = 1 << n
        e2e = {"value": conv_e2e / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": TPC * 16 * (N * N + N * M + S * L * 16),
               "d2h_bytes_per_step": TPC * (16 * L * 16 + 8 * S), "steps": len(hin),
               "targets": "the timed targets"}

    # Roofline of the dominant kernel from a separate pass over the same
    # targets with every launch bracketed by CUDA events on its stream.
    ctx.profile_reset()
    ctx.profile(True)
    for i in range(args.steps):
        step(probs_t, dev_t, i)
    torch.cuda.synchronize(dev)
    ctx.profile(False)
    prof = {name: ctx.profile_read(k) for k, name in enumerate(qfs.PROF_NAMES)}
    peak, peak_src = peaks()
    # The dominant kernel: the dataflow sweep (one launch per sweep of all
    # starts) or, with per-step launches, the fused backward step.
    if prof["dataflow"]["timed"]:
        dom, kname = prof["dataflow"], "k_sweep_df"
        kdesc = "k_sweep_df (one launch per sweep of all starts: forward, backward + update, residual)"
    else:
        dom, kname = prof["backward"], "k_backward_q4"
        kdesc = "k_backward_q4 (fused Phi update + environment + update)"
    avg_ms = dom["ms"] / max(dom["timed"], 1)
    bytes_per = dom["bytes"] / max(dom["timed"], 1)
    achieved = bytes_per / (avg_ms / 1e3) / 1e9 if dom["timed"] else None
    tr = traffic_record(kname, kind)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64" if prec == 1 else "f64",
        "data": "synthetic (seeded Haar-random targets of the stated structure)",
        "config": {"workload": WORKLOADS[kind][2] + (", double-and-restart of M (overtrain ratio 0.1)"
                                                     if args.restart_doubling else ""),
                   "n": n, "gates": L, "M": M, "multistarts": S,
                   "tol": first.tol, "max_sweeps": first.max_sweeps, "parallelism": f"{world} independent ranks",
                   "targets_per_call": TPC,
                   "timed_target_seeds": f"rank r: r*100000 + (0..{args.steps * TPC - 1}); warm-up targets separate",
                   "l2": "inputs larger than L2 (B list 512 MiB per target), no flush"},
        "converged": int(conv_all), "instantiations": args.steps * world * TPC,
        "sweeps_per_instantiation": float(np.mean(sweeps)),
        "training_states": [int(r.training_states) for r in results],
        "roofline": {"bound": "hbm", "kernel": kdesc,
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s",
                     "traffic": tr, "avg_launch_us": avg_ms * 1e3, "algorithmic_bytes_per_launch": bytes_per,
                     "launches_timed": dom["timed"],
                     "measured": "separate pass over the timed targets, every launch bracketed by CUDA events"},
        "kernel_time_share": {k: round(v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-9), 4)
                              for k, v in prof.items()},
        "clocks": clk, "e2e": e2e, "gpu_launches": int(launches_all),
    }
    if rank == 0 and args.cpu_baseline:
        g = golden_runs(kind)
        if g is not None:
            ctx_mp = mp.get_context("spawn")
            cores = os.cpu_count()
            with ctx_mp.Pool(cores) as pool:
                smp = [oracle_sample(kind, target_seeds(0, 1)[0], pool=pool, cores=cores)]
            v, _ = oracle_rate(smp, g)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": oracle_note(g, 1, cores)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def profile_case(args):
    """One sweep of the workload (all starts) through qfs_sweep_once: a small,
    fixed launch sequence for ncu captures of single kernels."""
    import torch  # noqa: F401
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import qfs
    qbuild.build()
    if args.workload == "uneven_blocks":
        # One batched launch over the 4096 uneven problems (8 starts each).
        from paper_2405_12866_gb300 import workloads as w
        import torch
        probs = w.uneven_blocks(P=args.batch_problems, seed=4, S=8)
        ns, Ls, pairs, tg, sm, ig = _pack_batch(probs, 8)
        dev = torch.device("cuda", 0)
        prm = qfs.default_params(M=0, multistarts=8, max_sweeps=500, dist_tol=1e-8, refine_sweeps_max=20)
        with qfs.Context(0) as ctx:
            # the shape the tuner keeps for this batch (16 lanes per start, two
            # starts per warp), without its trial launches
            ctx.set_option(qfs.QFS_OPT_BATCH_LANES_PER_START, 16)
            out = torch.zeros(int(Ls.sum()) * 16, dtype=torch.complex128, device=dev)
            info = ctx.instantiate_batch_dev(ns, Ls, pairs, torch.from_numpy(tg).to(dev), torch.from_numpy(sm).to(dev),
                                             torch.from_numpy(ig).to(dev), prm, out)
        print(json.dumps({"profile_case": "uneven_blocks", "converged": int(sum(r["converged"] for r in info))}))
        return 0
    if args.workload == "learned":
        # One loss-and-gradient pass of the warm-start network on a batch of
        # 4096 targets: the training GEMMs of one step.
        from paper_2405_12866_gb300 import learned
        T = learned.make_targets(11, 4096)
        lab = np.zeros((4096, 192))
        with qfs.Context(0) as ctx:
            ws = qfs.WarmStart(ctx, seed=3, batch_cap=4096)
            loss, _ = ws.loss_grad(T, lab)
            ws.close()
        print(json.dumps({"profile_case": "learned_loss_grad_4096", "loss": loss}))
        return 0
    p = _problem(args.workload, 0)
    prec = WORKLOADS[args.workload][1]
    with qfs.Context(0) as ctx:
        g, _, c = ctx.sweep_once(p.n, p.pairs, p.U, p.samples(), p.init_gates(), prec, want_envs=False)
    print(json.dumps({"profile_case": p.name, "min_cost": float(np.min(c))}))
    return 0


def _pack_batch(probs, S):
    ns = np.array([p.n for p in probs], dtype=np.int32)
    Ls = np.array([p.L for p in probs], dtype=np.int32)
    pairs = np.concatenate([np.asarray(p.pairs, dtype=np.int32).reshape(-1) for p in probs])
    tg = np.concatenate([p.U.reshape(-1) for p in probs])
    sm = np.concatenate([p.samples().reshape(-1) for p in probs])
    ig = np.concatenate([p.init_gates()[:S].reshape(-1) for p in probs])
    return ns, Ls, pairs, tg, sm, ig


def unit_trace_summary(tr, probs, info):
    """Critical path of one traced batched run: how long the GPU stays full,
    the tail after it, and the unit that ends the run (its problem's size,
    sweeps, start and duration).  tr: Context.batch_trace_read()."""
    if len(tr["t0"]) == 0:
        return None
    t0 = (tr["t0"] - tr["t0"].min()).astype(np.float64) / 1e6
    t1 = (tr["t1"] - tr["t0"].min()).astype(np.float64) / 1e6
    span = float(t1.max())
    grid = np.linspace(0.0, span, 401)
    active = np.array([int(((t0 <= t) & (t1 > t)).sum()) for t in grid])
    peak = int(active.max())
    full = grid[active >= 0.9 * peak]
    full_until = float(full.max()) if len(full) else 0.0
    last = int(np.argmax(t1))
    p = int(tr["problem"][last])
    sw = info[p]["sweeps"]
    return {"units": int(len(t0)), "span_ms": span, "peak_concurrent_units": peak,
            "full_until_ms": full_until, "tail_ms": span - full_until,
            "last_unit": {"n": int(probs[p].n), "L": int(probs[p].L), "converged": bool(info[p]["converged"]),
                          "sweeps": int(sw), "lanes_per_start": int(tr["G"][last]),
                          "start_ms": float(t0[last]), "duration_ms": float(t1[last] - t0[last]),
                          "us_per_sweep": float(1e3 * (t1[last] - t0[last]) / max(1, sw))}}


def run_ours_batch(args):
    """The batched form: one step = one whole batch of problems."""
    import torch
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    qbuild.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = qfs.Context(0, stream.cuda_stream)
    S, P = 8, args.batch_problems
    batches = []
    for seed in (4, 5):
        probs = w.uneven_blocks(P=P, seed=seed, S=S)
        ns, Ls, pairs, tg, sm, ig = _pack_batch(probs, S)
        batches.append((ns, Ls, pairs, torch.from_numpy(tg).to(dev), torch.from_numpy(sm).to(dev),
                        torch.from_numpy(ig).to(dev), probs, (tg, sm, ig)))
    prm = qfs.default_params(M=0, multistarts=S, max_sweeps=500, dist_tol=1e-8, refine_sweeps_max=20)
    if args.plateau:
        # the paper's suggested plateau detection (App. A): window 5, diff_tol_r 1e-5, min_iter 6
        prm.plateau_window, prm.diff_tol_r, prm.min_sweeps = 5, 1e-5, 6
    outs = [torch.zeros(int(b[1].sum()) * 16, dtype=torch.complex128, device=dev) for b in batches]

    def step(i):
        b = batches[i % 2]
        return ctx.instantiate_batch_dev(b[0], b[1], b[2], b[3], b[4], b[5], prm, outs[i % 2])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    ctx.profile_reset()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [step(args.warmup + i) for i in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = ctx.profile_read(-1)["launches"]
    conv = sum(r["converged"] for inf in infos for r in inf)
    value = conv / (ms / 1e3)
    # Algorithmic FP32 sweep arithmetic, 96 L N M flops per start-sweep,
    # counting every start at its problem's reported sweep count.
    flops = 0.0
    for i, inf in enumerate(infos):
        probs = batches[(args.warmup + i) % 2][6]
        for pr, r in zip(probs, inf):
            flops += S * r["sweeps"] * 96.0 * pr.L * (pr.M << pr.n)
    achieved = flops / (ms / 1e3) / 1e12
    fp32_peak = 72.9
    # End to end through the C-ABI's host entry (qfs_instantiate_batch): each
    # step's packed inputs in pinned host memory, its gates back into a pinned
    # host array, the copies inside the timed region; the same two batches
    # alternate as in the device-timed steps, after one untimed host call.
    hin = [[torch.from_numpy(x).pin_memory().numpy() for x in bb[7]] for bb in batches]
    hout = [torch.zeros(int(bb[1].sum()) * 16, dtype=torch.complex128).pin_memory().numpy() for bb in batches]

    def e2e_step(i):
        bb, h = batches[i % 2], hin[i % 2]
        return ctx.instantiate_batch_packed(bb[0], bb[1], bb[2], h[0], h[1], h[2], prm, hout[i % 2])[1]

    e2e_step(0)
    t0 = time.perf_counter()
    e2e_infos = [e2e_step(args.warmup + i) for i in range(args.steps)]
    t_e2e = time.perf_counter() - t0
    conv_e2e = sum(r["converged"] for inf in e2e_infos for r in inf)
    h2d = sum(sum(x.nbytes for x in hin[(args.warmup + i) % 2]) for i in range(args.steps)) / args.steps
    d2h = sum(hout[(args.warmup + i) % 2].nbytes for i in range(args.steps)) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic (seeded Haar-random targets of the stated structures)",
        "config": {"workload": WORKLOADS["uneven_blocks"][2] + (", plateau detection (window 5, diff_tol_r 1e-5)"
                                                                if args.plateau else ""),
                   "problems_per_step": P, "multistarts": S,
                   "tol": 1e-8, "max_sweeps": 500, "l2": "working set on chip; no flush"},
        "converged": int(conv), "instantiations": P * args.steps,
        "roofline": {"bound": "alu", "kernel": "k_batch_sweep (persistent)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "peak_source": "FP32 FMA peak measured on GB300 by an FMA-chain throughput kernel: 72.9 TFLOP/s",
                     "traffic": None if args.plateau else traffic_record("k_batch_sweep", "uneven_blocks"),
                     "algorithmic_flops_per_step": flops / args.steps},
        "clocks": clk,
        "e2e": {"value": conv_e2e / t_e2e, "unit": UNIT,
                "note": "C-ABI host entry on packed pinned host arrays, host-device copies and result records included",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
    }
    # One more step, untimed, with the unit trace on: where the makespan goes.
    ctx.batch_trace(1 << 20)
    tr_info = step(0)
    torch.cuda.synchronize(dev)
    line["unit_trace"] = unit_trace_summary(ctx.batch_trace_read(), batches[0][6], tr_info)
    ctx.batch_trace(0)
    tuned, trials = ctx.batch_schedules()
    line["config"]["schedules"] = {f"n{t['n']}_L{t['L']}": f"G{t['G']}w{t['warps']}" for t in tuned}
    line["config"]["batch_plans"] = ctx.batch_plans
    print(json.dumps({"batch_trials": trials}), file=sys.stderr, flush=True)
    if args.cpu_baseline:
        t0 = time.perf_counter()
        n_sample = 0
        conv_o = 0
        for pr in batches[0][6]:
            Psi, G0 = pr.samples(), pr.init_gates()[:S]
            r = __import__("oracle.qfs_oracle", fromlist=["x"]).instantiate(pr.U, Psi, G0, pr.pairs, pr.n, 1e-8, 500)
            conv_o += r.converged
            n_sample += 1
            if time.perf_counter() - t0 > 15.0:
                break
        t_o = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": conv_o / t_o, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the first {n_sample} problems of the batch, run to completion by the oracle on one core ({t_o:.1f} s)"}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_ours_learned(args):
    """The learned form: labels from the method, training on the GPU, then
    one step = the whole evaluation set through the warm-start policy
    (predicted start, random multistarts as the fallback), host arrays in
    and out (so value and e2e are the same end-to-end measurement)."""
    import torch
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import learned, qfs
    qbuild.build()
    dev = torch.device("cuda", 0)
    ctx = qfs.Context(0)
    workers = max(1, min(16, os.cpu_count() or 1))
    ntrain, neval, epochs = args.learned_train, args.learned_eval, args.learned_epochs
    t0 = time.perf_counter()
    Ttr = learned.make_targets(11, ntrain, workers=workers)
    Tev = learned.make_targets(12, neval, workers=workers)
    # Pinned host memory for the targets the timed steps upload (the
    # end-to-end contract: host inputs from pinned memory).
    Tev = torch.from_numpy(np.ascontiguousarray(Tev)).pin_memory().numpy()
    t_targets = time.perf_counter() - t0
    ls = learned.method_labels(ctx, Ttr, workers=workers)
    # The training GEMMs' rate: per-launch CUDA events (harvested after each
    # replayed training step) over two epochs of a separate network of the
    # same shapes, so that the timed training below runs unprofiled.
    probe = qfs.WarmStart(ctx, seed=99, batch_cap=4096)
    nprobe = min(len(ls.targets), 1 << 16)
    ctx.profile(True)
    ctx.profile_reset()
    probe.train(ls.targets[:nprobe], ls.labels[:nprobe], epochs=2, batch=4096, lr=2e-3, lr_final=4e-5, seed=1)
    mlp = ctx.profile_read(qfs.PROF_NAMES.index("mlp"))
    ctx.profile(False)
    probe.close()
    gemm_tflops = mlp["bytes"] / (mlp["ms"] / 1e3) / 1e12 if mlp["ms"] > 0 else None
    ws = qfs.WarmStart(ctx, seed=3, batch_cap=4096)
    t0 = time.perf_counter()
    losses = ws.train(ls.targets, ls.labels, epochs=epochs, batch=4096, lr=2e-3, lr_final=4e-5, seed=1)
    t_train = time.perf_counter() - t0
    first_rand = learned.random_starts(5000, neval, 1)[:, 0]

    def step(i):
        return learned.two_stage(ctx, Tev, None, ws=ws, seed=7000 + i, name="learned")

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    ctx.profile(True)
    ctx.profile_reset()
    stats = [step(args.warmup + i) for i in range(args.steps)]
    clk = clocks.stop()
    launches = ctx.profile_read(-1)["launches"]
    ctx.profile(False)
    secs = sum(s.seconds for s in stats)
    conv = sum(s.converged for s in stats)
    value = conv / secs
    rand = learned.two_stage(ctx, Tev, first_rand, ws=ws, seed=7000, name="random first start")
    base = learned.multistart(ctx, Tev, S=8, seed=7000, name="8 random starts")
    # The plain FP64 GPU path (one problem per call, 8 starts) on a sample.
    nfp = min(64, neval)
    p64 = qfs.default_params(M=learned.M_SAMPLES, multistarts=8, max_sweeps=300, dist_tol=1e-8,
                             precision=qfs.QFS_FP64, seed=0)
    t0 = time.perf_counter()
    c64 = sum(ctx.instantiate(learned.N_QUBITS, learned.PAIRS, Tev[i], p64).converged for i in range(nfp))
    t64 = time.perf_counter() - t0
    tc_peak, tc_src = bf16_peak(sustained=True)

    def pol(s):
        return {"converged": s.converged, "of": s.P, "seconds": s.seconds, "converged_per_s": s.converged_per_s,
                "first_start_converged": s.first_stage_converged, "start_sweeps": s.start_sweeps}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64 sweeps, bf16 MLP",
        "data": "synthetic (seeded Haar-random circuits of the learned structure)",
        "config": {"workload": WORKLOADS["learned"][2], "train_pairs_generated": ntrain,
                   "train_pairs_converged": int(len(ls.labels)), "eval_targets": neval, "epochs": epochs,
                   "first_sweeps": 100, "fallback_starts": 8, "max_sweeps": 300, "tol": 1e-8,
                   "l2": "eval targets 256 MiB > L2; no flush"},
        "learned": {"policy": pol(stats[-1]), "random_first_start_policy": pol(rand),
                    "eight_random_starts": pol(base),
                    "plain_fp64_gpu_path": {"converged": int(c64), "of": nfp, "converged_per_s": c64 / t64},
                    "train_seconds": t_train, "train_samples_per_s": len(ls.labels) * epochs / t_train,
                    "epoch_loss_first_last": [float(losses[0]), float(losses[-1])],
                    "label_generation_seconds": ls.seconds, "target_generation_seconds": t_targets},
        "roofline": {"bound": "tensor", "kernel": "k_gemm_bf16_tma (training GEMMs, all shapes)",
                     "achieved": gemm_tflops, "peak": tc_peak, "unit": "TFLOP/s",
                     "frac": gemm_tflops / tc_peak if gemm_tflops else None, "peak_source": tc_src,
                     "traffic": None,
                     "measured": "per-launch CUDA events inside replayed training-step graphs, two epochs of a "
                                 "same-shape network on %d pairs" % nprobe},
        "clocks": clk,
        "e2e": {"value": value, "unit": UNIT, "note": "host targets in, host gates out: value is end to end",
                "h2d_bytes_per_step": int(Tev.nbytes), "d2h_bytes_per_step": int(neval * 6 * 256)},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    ws.close()
    ctx.close()
    return 0


def run_qf_vs_qfs(args):
    """Full-unitary QFactor (M = 2^n) against QFactor-Sample with the paper's
    double-and-restart (M from 2, overtrain ratio 0.1), on the same kernels,
    the same targets and the same initial gates: time per instantiation for
    n = 3..args.qf_max_n, brick walls of 4 half-layers (FP64, 8 starts).
    The paper's ratios (QF-J over QFS-J on A100) are context only."""
    import torch
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    qbuild.build()
    ctx = qfs.Context(0)
    rows = []
    S, sweeps, tol = 8, 500, 1e-8
    for n in range(3, args.qf_max_n + 1):
        pairs = w.brick_pairs(n, 4)
        times = {"qf": [], "qfs": []}
        conv = {"qf": 0, "qfs": 0}
        ms = []
        for t in range(args.steps + args.warmup):
            p = w.make_problem(f"qf_{n}", n, pairs, 1 << n, S, 7000 + 100 * n + t, 9000 + 100 * n + t, tol, sweeps)
            for kind in ("qf", "qfs"):
                if kind == "qf":
                    prm = qfs.default_params(M=1 << n, multistarts=S, max_sweeps=sweeps, dist_tol=tol, seed=p.seed)
                else:
                    prm = qfs.default_params(M=2, multistarts=S, max_sweeps=sweeps, dist_tol=tol, seed=p.seed,
                                             restart_doubling=1, overtrain_ratio=0.1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = ctx.instantiate(n, pairs, p.U, prm)
                dt = time.perf_counter() - t0
                if t >= args.warmup:
                    times[kind].append(dt)
                    conv[kind] += int(r.converged)
                    if kind == "qfs":
                        ms.append(int(r.training_states))
        tq, ts = float(np.mean(times["qf"])), float(np.mean(times["qfs"]))
        rows.append({"n": n, "gates": len(pairs), "qf_s": tq, "qfs_s": ts, "ratio": tq / ts,
                     "qf_converged": conv["qf"], "qfs_converged": conv["qfs"], "of": args.steps,
                     "qfs_final_M": ms})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    big = [r["ratio"] for r in rows if r["n"] > 8]
    line = {"metric": "QF/QFS instantiation-time ratio (same kernels)", "value": float(np.exp(np.mean(np.log(
        [r["ratio"] for r in rows])))), "unit": "x (geometric mean over n)", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Haar-random brick-wall targets)",
        "config": {"workload": "QF (M = 2^n) vs QFS (double-and-restart from M = 2), brick walls of 4 half-layers, "
                               "n = 3..%d, 8 starts, tol 1e-8" % args.qf_max_n},
        "ratio_above_8_qubits": float(np.exp(np.mean(np.log(big)))) if big else None,
        "rows": rows, "paper_context": "QF-J / QFS-J on A100: 17.7x average, 69x above 8 qubits (Sec. 4)"}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_states_ablation(args):
    """Training-state distribution (Appendix D): Haar states against
    distinct computational-basis states as training data, on the same
    kernels, targets and initial gates.  For brick walls of 4 half-layers
    (n = 6, 8, 10; FP64, 8 starts, tol 1e-8) and args.steps targets each:
    (a) fixed M = 2, 4, ..., 2^n: how many results generalise, i.e. converge
    and have a full-unitary cost ||U - C||_F^2 / N (Eq. 1 per state,
    evaluated on the host from the returned gates) within tol (1 + otr);
    M_gen of a target = the smallest M whose result generalises; (b) double-and-restart
    from M = 2 with validation states of the same distribution: the final M,
    whether the returned gates generalise, time per instantiation."""
    import torch
    from paper_2405_12866_gb300 import build as qbuild
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    qbuild.build()
    ctx = qfs.Context(0)
    S, sweeps, tol, otr, T = 8, 500, 1e-8, 0.1, max(1, args.steps)
    names = {qfs.QFS_STATES_HAAR: "haar", qfs.QFS_STATES_BASIS: "basis"}
    rows = []
    for n in args.ablation_n:
        pairs = w.brick_pairs(n, 4)
        N = 1 << n
        probs = [w.make_problem(f"abl_{n}", n, pairs, 2, S, 5000 + 100 * n + t, 6000 + 100 * n + t, tol, sweeps)
                 for t in range(T)]

        def generalises(p, gates):
            C = w.target_unitary(gates, pairs, n)
            return float(np.sum(np.abs(p.U - C) ** 2) / N)

        row = {"n": n, "gates": len(pairs), "targets": T}
        for dist, name in names.items():
            fixed, m_gen = {}, [None] * T
            M = 2
            while M <= N and any(m is None for m in m_gen):
                ok = conv = 0
                for t, p in enumerate(probs):
                    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=sweeps, dist_tol=tol, seed=p.seed,
                                             training_distribution=dist)
                    r = ctx.instantiate(n, pairs, p.U, prm)
                    conv += int(r.converged)
                    good = r.converged and generalises(p, r.gates) <= tol * (1 + otr)
                    ok += int(good)
                    if good and m_gen[t] is None:
                        m_gen[t] = M
                fixed[M] = {"converged": conv, "generalised": ok}
                M *= 2
            final_m, gen, times = [], 0, []
            for t, p in enumerate(probs):
                prm = qfs.default_params(M=2, multistarts=S, max_sweeps=sweeps, dist_tol=tol, seed=p.seed,
                                         restart_doubling=1, overtrain_ratio=otr, training_distribution=dist)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = ctx.instantiate(n, pairs, p.U, prm)
                times.append(time.perf_counter() - t0)
                final_m.append(int(r.training_states))
                gen += int(r.converged and generalises(p, r.gates) <= tol * (1 + otr))
            row[name] = {"M_gen": m_gen, "fixed_M": fixed, "restart_final_M": final_m,
                         "restart_generalised": gen, "restart_s": float(np.mean(times))}
        print(json.dumps(row), file=sys.stderr, flush=True)
        rows.append(row)
    ratios = [b / h for r in rows for b, h in zip(r["basis"]["M_gen"], r["haar"]["M_gen"]) if b and h]
    line = {"metric": "training data needed to generalise, computational-basis / Haar states (per-target M_gen ratio)",
            "value": float(np.exp(np.mean(np.log(ratios)))) if ratios else None,
            "unit": "x (geometric mean over targets)", "n_gpus": 1, "steps": T, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Haar-random brick-wall targets)",
            "config": {"workload": "Haar vs computational-basis training states, brick walls of 4 half-layers, "
                                   "n = %s, 8 starts, tol 1e-8, overtrain ratio 0.1, %d targets per n"
                                   % (",".join(map(str, args.ablation_n)), T)},
            "rows": rows,
            "paper_context": "Appendix D: computational-basis training needs much more data than Haar states"}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="brick_n12")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false",
                    help="skip the end-to-end pass through the host-pointer API")
    ap.add_argument("--targets-per-call", type=int, default=1,
                    help="instantiate this many targets per call, their starts sweeping together")
    ap.add_argument("--slots", type=int, default=0,
                    help="targets sweeping concurrently within a call (0: the library's choice)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--batch-problems", type=int, default=4096)
    ap.add_argument("--plateau", action="store_true",
                    help="batched form: the paper's plateau detection (window 5, diff_tol_r 1e-5, min_iter 6)")
    ap.add_argument("--restart-doubling", action="store_true",
                    help="the paper's double-and-restart of the training states (host targets)")
    ap.add_argument("--qf-max-n", type=int, default=10)
    ap.add_argument("--ablation-n", type=int, nargs="+", default=[6, 8, 10])
    ap.add_argument("--learned-train", type=int, default=1 << 20)
    ap.add_argument("--learned-eval", type=int, default=65536)
    ap.add_argument("--learned-epochs", type=int, default=40)
    ap.add_argument("--start-groups", type=int, default=0,
                    help="concurrent groups of multistarts (0 = the library's choice)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one sweep of the workload and exit (for ncu captures)")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven_blocks":
        return run_ours_batch(args)
    if args.workload == "learned":
        return run_ours_learned(args)
    if args.workload == "qf_vs_qfs":
        return run_qf_vs_qfs(args)
    if args.workload == "states_ablation":
        return run_states_ablation(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
