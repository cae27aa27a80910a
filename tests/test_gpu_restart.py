"""Double-and-restart of the training states (Sec. 3, App. A) on the GPU
against the oracle's outer loop on the same draws."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("M0,min_sweeps", [(2, 0), (2, 6), (4, 0)])
def test_chain_n3_restart_matches_oracle(ctx, M0, min_sweeps):
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    p = w.chain_n3(target_seed=1)
    seed, S, otr = 77, 2, 0.1
    tr = lambda M, a: w.sample_states(w.attempt_seed(seed, a), p.n, M)
    va = lambda M, a: w.sample_states(w.attempt_seed(seed, a), p.n, M, stream=w.STREAM_VALIDATION)
    want = o.instantiate_restarting(p.U, tr, va, w.initial_gates(seed, S, p.L), p.pairs, p.n, 1e-10, 200, M0, otr,
                                    min_sweeps=min_sweeps)
    prm = qfs.default_params(M=M0, multistarts=S, max_sweeps=200, dist_tol=1e-10, seed=seed, min_sweeps=min_sweeps,
                             restart_doubling=1, overtrain_ratio=otr, precision=qfs.QFS_FP64)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm)
    assert got.training_states == want.training_states
    assert got.converged == want.converged
    assert abs(got.sweeps - want.sweeps) <= 1
    if want.converged:
        assert got.cost <= 1e-10 and abs(got.cost - want.cost) < 1e-11
        assert got.best_start == want.best_start
        assert np.max(np.abs(got.gates - want.gates)) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_brick_n8_restart_reaches_a_generalising_solution(ctx, prec):
    """At its literal M = 16 this target stalls near cost 1.3 on every start;
    the outer loop doubles M until the validation cost agrees with the
    training cost and returns gates whose full-unitary cost (Eq. 1) is
    within the paper's bound dist_tol (1 + overtrain_ratio), up to a margin."""
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    p = w.brick_n8(target_seed=1)
    otr = 0.1
    prm = qfs.default_params(M=16, multistarts=16, max_sweeps=500, dist_tol=p.tol, seed=5, restart_doubling=1,
                             overtrain_ratio=otr, precision=qfs.QFS_MIXED if prec == "mixed" else qfs.QFS_FP64)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm)
    assert got.converged and got.cost <= p.tol
    assert got.training_states >= 32
    per_state = o.full_cost(p.U, got.gates, p.pairs, p.n) / (1 << p.n)
    assert per_state <= 10 * p.tol * (1 + otr)
