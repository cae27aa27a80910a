"""Several targets per call (qfs_instantiate_many): each target's result is
the one it gets alone, bit for bit, while the targets share the dataflow
launches."""
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


def _same(a, b):
    assert a.converged == b.converged and a.sweeps == b.sweeps and a.best_start == b.best_start
    assert a.fp64_sweeps == b.fp64_sweeps
    assert a.cost == b.cost
    assert np.array_equal(np.asarray(a.gates), np.asarray(b.gates))
    assert np.array_equal(a.start_costs, b.start_costs)


@pytest.mark.parametrize("kind,prec,T,plateau,slots", [
    ("brick_n8", "mixed", 3, 0, 0), ("brick_n8", "fp64", 2, 0, 0), ("chain_n4", "fp64", 3, 0, 0),
    ("brick_n8", "mixed", 2, 5, 0), ("brick_n12", "mixed", 2, 0, 0),
    ("brick_n8", "mixed", 5, 0, 2), ("chain_n4", "fp64", 6, 0, 4), ("brick_n8", "mixed", 4, 5, 3)])
def test_many_targets_match_single_calls(ctx, kind, prec, T, plateau, slots):
    """slots < T: a slot whose target finishes takes the next target."""
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    if kind == "brick_n12":
        probs = [w.brick_n12(target_seed=40 + t) for t in range(T)]
        S, M, sweeps = 32, 32, 500
    elif kind == "brick_n8":
        probs = [w.make_problem("b8", 8, w.brick_pairs(8, 4), 16, 8, 50 + t, 60 + t, 1e-8, 300) for t in range(T)]
        S, M, sweeps = 8, 16, 300
    else:
        probs = [w.make_problem("c4", 4, w.chain_pairs(4, 5), 8, 4, 70 + t, 80 + t, 1e-10, 200) for t in range(T)]
        S, M, sweeps = 4, 8, 200
    p0 = probs[0]
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=sweeps, dist_tol=p0.tol, plateau_window=plateau,
                             precision=qfs.QFS_MIXED if prec == "mixed" else qfs.QFS_FP64, concurrent_targets=slots)
    alone = [ctx.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates()) for p in probs]
    many = ctx.instantiate_many(p0.n, p0.pairs, np.stack([p.U for p in probs]), prm,
                                np.stack([p.samples() for p in probs]), np.stack([p.init_gates() for p in probs]))
    assert len(many) == T
    for a, b in zip(alone, many):
        _same(a, b)
    # the targets need different sweep counts, so some finish while others sweep on
    if kind != "brick_n12":
        assert len({r.sweeps for r in alone}) > 1 or T == 1


def test_many_targets_device_entry_and_drawn_inputs(ctx):
    import torch
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    T, S, M = 2, 8, 16
    probs = [w.make_problem("b8", 8, w.brick_pairs(8, 4), M, S, 90 + t, 95 + t, 1e-8, 300) for t in range(T)]
    p0 = probs[0]
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=300, dist_tol=1e-8, precision=qfs.QFS_MIXED, seed=123)
    dev = torch.device("cuda", 0)
    Ud = torch.from_numpy(np.stack([p.U for p in probs])).to(dev)
    Pd = torch.from_numpy(np.stack([p.samples() for p in probs])).to(dev)
    Gd = torch.from_numpy(np.ascontiguousarray(np.stack([p.init_gates() for p in probs]))).to(dev)
    out = torch.zeros((T, p0.L, 4, 4), dtype=torch.complex128, device=dev)
    many = ctx.instantiate_many_dev(p0.n, p0.pairs, Ud, Pd, Gd, prm, out)
    host = ctx.instantiate_many(p0.n, p0.pairs, np.stack([p.U for p in probs]), prm,
                                np.stack([p.samples() for p in probs]), np.stack([p.init_gates() for p in probs]))
    for a, b in zip(many, host):
        assert a.sweeps == b.sweeps and a.cost == b.cost
        assert np.array_equal(np.asarray(a.gates.cpu()), np.asarray(b.gates))
    # drawn inputs: target t uses seed + t, as a single call with that seed
    drawn = ctx.instantiate_many(p0.n, p0.pairs, np.stack([p.U for p in probs]), prm)
    for t, p in enumerate(probs):
        prm1 = qfs.default_params(M=M, multistarts=S, max_sweeps=300, dist_tol=1e-8, precision=qfs.QFS_MIXED,
                                  seed=123 + t)
        _same(ctx.instantiate(p.n, p.pairs, p.U, prm1), drawn[t])


def test_many_targets_rejects_restart(ctx):
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    p = w.chain_n3()
    prm = qfs.default_params(M=2, multistarts=2, max_sweeps=10, restart_doubling=1)
    with pytest.raises(qfs.QfsError):
        ctx.instantiate_many(p.n, p.pairs, np.stack([p.U, p.U]), prm)
