"""Write oracle reference runs of full-size workloads to tests/golden/.

TEST INFRASTRUCTURE: calls only the oracle and the seeded input generator.
For each target it runs the oracle's multistart instantiation (Appendix A
stopping rule, lock step) with the starts spread over host processes in
chunks of sweeps, which gives the same result as the sequential lock-step
loop because the starts never interact before the stop.  Records, per
target: converged, the stopping sweep, the selected start and its cost.

    python -m oracle.make_golden brick_n12 0 1 2 3
    python -m oracle.make_golden brick_n8_restart 0 1 2
    python -m oracle.make_golden uneven_blocks 512

The second form runs the oracle's double-and-restart outer loop on the
brick_n8 workload (one target per process) and records converged, the
total sweeps, the selected start, the final M and the costs.  The third
runs the oracle's multistart instantiation on the first P problems of the
batched workload (one problem per process).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import qfs_oracle as o  # noqa: E402


def _chunk(args):
    UPsi, Psi, G, pairs, n, sweeps = args
    costs = []
    for _ in range(sweeps):
        r = o.sweep(UPsi, Psi, G, pairs, n)
        G = r.gates
        costs.append(r.cost)
    return G, costs


def lockstep_parallel(UPsi, Psi, G0, pairs, n, tol, max_sweeps, pool, chunk=10):
    """The oracle's instantiate() with the starts on a process pool."""
    S = G0.shape[0]
    G = [G0[s] for s in range(S)]
    trace = []
    done = 0
    while done < max_sweeps:
        step = min(chunk, max_sweeps - done)
        res = pool.map(_chunk, [(UPsi, Psi, G[s], pairs, n, step) for s in range(S)])
        G = [r[0] for r in res]
        block = np.array([r[1] for r in res]).T   # (step, S)
        for i in range(step):
            trace.append(block[i])
            if np.any(block[i] <= tol):
                # the sequential loop stops here; rerun the starts to this sweep
                stop = done + i + 1
                res = pool.map(_chunk, [(UPsi, Psi, G0[s], pairs, n, stop) for s in range(S)])
                final = np.array([r[1][-1] for r in res])
                best = int(np.argmin(final))
                return dict(converged=True, sweeps=stop, best_start=best, cost=float(final[best]),
                            start_costs=final.tolist())
        done += step
    final = np.array(trace[-1])
    best = int(np.argmin(final))
    return dict(converged=bool(final[best] <= tol), sweeps=done, best_start=best,
                cost=float(final[best]), start_costs=final.tolist())


def _restart_run(sd):
    """Double-and-restart (Sec. 3, App. A) of brick_n8 target sd from its
    literal M = 16, with the library's draws of seed p.seed: training
    states of attempt a from attempt_seed(seed, a) (stream 1), validation
    states from stream 5, initial gates from stream 2."""
    from paper_2405_12866_gb300 import workloads as w
    p = w.brick_n8(target_seed=sd)
    t = time.time()
    tr = lambda M, a: w.training_states(0, w.attempt_seed(p.seed, a), p.n, M)
    va = lambda M, a: w.training_states(0, w.attempt_seed(p.seed, a), p.n, M, stream=w.STREAM_VALIDATION)
    r = o.instantiate_restarting(p.U, tr, va, w.initial_gates(p.seed, p.S, p.L), p.pairs, p.n, p.tol,
                                 p.max_sweeps, p.M, RESTART_OTR, min_sweeps=RESTART_MIN_SWEEPS)
    return dict(converged=r.converged, sweeps=r.sweeps, best_start=r.best_start, cost=r.cost,
                validation_cost=r.validation_cost, training_states=r.training_states, attempts=r.attempts,
                name=p.name + "_restart", target_seed=sd, run_seed=p.seed, M0=p.M, tol=p.tol,
                max_sweeps=p.max_sweeps, overtrain_ratio=RESTART_OTR, min_sweeps=RESTART_MIN_SWEEPS,
                seconds=round(time.time() - t, 1))


def _uneven_run(args):
    """The oracle's multistart run of problem i of the uneven-blocks batch."""
    i, seed, S, max_sweeps, tol = args
    from paper_2405_12866_gb300 import workloads as w
    p = w.uneven_blocks(P=i + 1, seed=seed, S=S)[i]
    r = o.instantiate(p.U, p.samples(), p.init_gates()[:S], p.pairs, p.n, tol, max_sweeps)
    return dict(n=p.n, L=p.L, converged=r.converged, sweeps=r.sweeps, best_start=r.best_start, cost=r.cost)


UNEVEN_SEED, UNEVEN_S, UNEVEN_MAX_SWEEPS, UNEVEN_TOL = 4, 8, 300, 1e-8


RESTART_OTR = 0.1
RESTART_MIN_SWEEPS = 6


def main(argv):
    from paper_2405_12866_gb300 import workloads as w
    kind = argv[0]
    seeds = [int(x) for x in argv[1:]] or [0]
    if kind == "uneven_blocks":
        # problems 0 .. P-1 of the batched workload (seed 4, 8 starts, 300 sweeps)
        P = seeds[0]
        out_path = os.path.join(ROOT, "tests", "golden", "uneven_blocks_oracle_runs.json")
        jobs = [(i, UNEVEN_SEED, UNEVEN_S, UNEVEN_MAX_SWEEPS, UNEVEN_TOL) for i in range(P)]
        t = time.time()
        with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
            runs = pool.map(_uneven_run, jobs, chunksize=4)
        json.dump(dict(seed=UNEVEN_SEED, starts=UNEVEN_S, max_sweeps=UNEVEN_MAX_SWEEPS, tol=UNEVEN_TOL,
                       seconds=round(time.time() - t, 1), runs=runs), open(out_path, "w"), indent=0)
        print(kind, P, sum(r["converged"] for r in runs), "converged", flush=True)
        return
    if kind == "brick_n8_restart":
        out_path = os.path.join(ROOT, "tests", "golden", "brick_n8_restart_oracle_runs.json")
        runs = json.load(open(out_path)) if os.path.exists(out_path) else {}
        with mp.get_context("spawn").Pool(min(len(seeds), os.cpu_count())) as pool:
            for sd, r in zip(seeds, pool.map(_restart_run, seeds)):
                runs[str(sd)] = r
                print(kind, sd, {k: r[k] for k in ("converged", "sweeps", "best_start", "training_states")},
                      flush=True)
        json.dump(runs, open(out_path, "w"), indent=1)
        return
    factory = {"brick_n12": w.brick_n12, "brick_n8": w.brick_n8}[kind]
    out_path = os.path.join(ROOT, "tests", "golden", f"{kind}_oracle_runs.json")
    runs = json.load(open(out_path)) if os.path.exists(out_path) else {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool:
        for sd in seeds:
            p = factory(target_seed=sd)
            Psi, G0 = p.samples(), p.init_gates()
            t = time.time()
            r = lockstep_parallel(p.U @ Psi, Psi, G0, p.pairs, p.n, p.tol, p.max_sweeps, pool)
            r.update(name=p.name, target_seed=sd, run_seed=p.seed, tol=p.tol,
                     max_sweeps=p.max_sweeps, seconds=round(time.time() - t, 1),
                     host_cores=os.cpu_count())
            runs[str(sd)] = r
            print(kind, sd, {k: r[k] for k in ("converged", "sweeps", "best_start", "cost")}, flush=True)
            json.dump(runs, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
