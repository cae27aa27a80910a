"""Full instantiations of the benchmark workloads against stored oracle runs.

The oracle's runs (tests/golden/*_oracle_runs.json, written by
oracle/make_golden.py, which calls only the oracle and the seeded input
generator) fix, per target, whether the multistart run converges, the sweep
at which it stops (Appendix A: the first sweep at which some start's sample
cost is <= dist_tol), the selected start and its cost.

- brick_n12 (n = 12, 17 gates, M = 32, 32 starts, tol 1e-8), the mixed
  path: complex64 sweeps, FP64 updates, FP64 cost check.  The stopping sweep
  may differ by up to K_MIXED sweeps: a complex64 trajectory differs from the
  FP64 one by about 1e-7 relative per sweep, which can move the sweep at
  which the converging start's cost crosses the tolerance.  The returned
  gates' FP64 sample cost is recomputed by the oracle.
- The same targets with refine_switch_tol = 1e-5: every start is handed to
  FP64 refinement sweeps as soon as its complex64 cost is below 1e-5, so the
  refinement branch must run and still end at an oracle-confirmed cost
  <= tol, on the start the oracle selects.
- brick_n8 (n = 8, 28 gates, M0 = 16, 16 starts) with double-and-restart on,
  FP64: the same final M, convergence, selected start and (up to one sweep
  per attempt) sweep count as the oracle's outer loop.
"""
import json
import os

import numpy as np
import pytest

from oracle import qfs_oracle as o
from paper_2405_12866_gb300 import workloads as w

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
K_MIXED = 3


def _golden(name):
    return json.load(open(os.path.join(GOLDEN, name)))


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import build, qfs
    build.build()
    c = qfs.Context(0)
    yield c
    c.close()


def _check_against_oracle_cost(p, Psi, got):
    c = o.sample_cost(p.U @ Psi, Psi, got.gates, p.pairs, p.n)
    assert c <= p.tol, c
    assert abs(c - got.cost) < 1e-11, (c, got.cost)


@pytest.mark.parametrize("sd", [str(i) for i in range(12)])
def test_brick_n12_mixed_instantiation_matches_oracle_run(ctx, sd):
    from paper_2405_12866_gb300 import qfs
    runs = _golden("brick_n12_oracle_runs.json")
    if sd not in runs:
        pytest.skip(f"no oracle run of target {sd} recorded")
    g = runs[sd]
    p = w.brick_n12(target_seed=int(sd))
    assert g["run_seed"] == p.seed and g["tol"] == p.tol
    Psi, G0 = p.samples(), p.init_gates()
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=p.max_sweeps, dist_tol=p.tol,
                             precision=qfs.QFS_MIXED)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm, Psi, G0)
    print(f"\ntarget {sd}: sweeps {got.sweeps} (oracle {g['sweeps']}), start {got.best_start} "
          f"(oracle {g['best_start']}), FP64 sweeps {got.fp64_sweeps}, cost {got.cost:.3e}")
    assert got.converged == g["converged"]
    assert got.best_start == g["best_start"]
    assert abs(got.sweeps - g["sweeps"]) <= K_MIXED, (got.sweeps, g["sweeps"])
    _check_against_oracle_cost(p, Psi, got)


@pytest.mark.parametrize("sd", ["0", "1"])
def test_brick_n12_forced_fp64_refinement_matches_oracle_run(ctx, sd):
    from paper_2405_12866_gb300 import qfs
    g = _golden("brick_n12_oracle_runs.json")[sd]
    p = w.brick_n12(target_seed=int(sd))
    Psi, G0 = p.samples(), p.init_gates()
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=p.max_sweeps, dist_tol=p.tol,
                             precision=qfs.QFS_MIXED, refine_switch_tol=1e-5, refine_sweeps_max=50)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm, Psi, G0)
    print(f"\ntarget {sd}: complex64 sweeps {got.sweeps} + FP64 sweeps {got.fp64_sweeps} (oracle {g['sweeps']})")
    assert got.fp64_sweeps > 0
    assert got.converged == g["converged"]
    assert got.best_start == g["best_start"]
    # complex64 sweeps to the switch, then FP64 sweeps of the selected start
    assert got.sweeps < g["sweeps"]
    assert abs(got.sweeps + got.fp64_sweeps - g["sweeps"]) <= K_MIXED, (got.sweeps, got.fp64_sweeps, g["sweeps"])
    _check_against_oracle_cost(p, Psi, got)


@pytest.mark.parametrize("sd", ["0", "1", "2"])
def test_brick_n8_restart_matches_oracle_outer_loop(ctx, sd):
    from paper_2405_12866_gb300 import qfs
    g = _golden("brick_n8_restart_oracle_runs.json")[sd]
    p = w.brick_n8(target_seed=int(sd))
    assert g["run_seed"] == p.seed and g["M0"] == p.M
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=p.max_sweeps, dist_tol=p.tol, seed=p.seed,
                             restart_doubling=1, overtrain_ratio=g["overtrain_ratio"],
                             min_sweeps=g["min_sweeps"], precision=qfs.QFS_FP64)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm)
    assert got.training_states == g["training_states"]
    assert got.converged == g["converged"]
    assert got.best_start == g["best_start"]
    assert abs(got.sweeps - g["sweeps"]) <= g["attempts"], (got.sweeps, g["sweeps"])
    if g["converged"]:
        assert got.cost <= p.tol
        assert abs(got.cost - g["cost"]) < 1e-11
        Psi = w.training_states(0, w.attempt_seed(p.seed, g["attempts"] - 1), p.n, g["training_states"])
        c = o.sample_cost(p.U @ Psi, Psi, got.gates, p.pairs, p.n)
        assert abs(c - got.cost) < 1e-11
