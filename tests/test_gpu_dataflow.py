"""The dataflow sweep (one cooperative persistent launch per sweep) against
the per-step launches and against the CPU oracle, on structures that reach
every kind of step: forward steps, backward steps whose two gates touch
four, three (all four placements) or two qubits (both orders), the first
backward step without a gate, and the complex64 residual pass."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(dataflow: bool):
    from paper_2405_12866_gb300 import qfs
    c = qfs.Context(0)
    c.set_option(qfs.QFS_OPT_DATAFLOW, 1 if dataflow else 0)
    return c


@pytest.fixture(scope="module")
def ctxs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import build
    build.build()
    a, b = _ctx(True), _ctx(False)
    yield a, b
    a.close()
    b.close()


# (n, pairs, M, S): structures whose consecutive gates cover every case.
CASES = {
    "brick_n8": (8, None, 16, 6),
    "chain_shared_qubit": (5, [(0, 1), (1, 2), (2, 3), (3, 4), (2, 3), (1, 2), (0, 1)], 8, 5),
    "shared_qubit_other_side": (5, [(1, 2), (0, 1), (2, 3), (1, 2), (3, 4), (2, 3)], 6, 3),
    "same_pair_both_orders": (4, [(0, 1), (0, 1), (1, 0), (2, 3), (3, 2), (1, 2)], 4, 4),
    "single_gate": (3, [(0, 2)], 2, 3),
    "shared_first_qubit": (4, [(1, 0), (1, 2), (2, 3), (2, 1)], 4, 3),
}


def _inputs(name):
    from paper_2405_12866_gb300 import workloads as w
    n, pairs, M, S = CASES[name]
    if pairs is None:
        pairs = w.brick_pairs(n, 8)
    L = len(pairs)
    gt = w.haar_gates(17, w.STREAM_TARGET_GATES, L)
    U = w.target_unitary(gt, pairs, n)
    Psi = w.sample_states(5, n, M)
    G0 = w.initial_gates(23, S, L)
    return n, pairs, U, Psi, G0


@pytest.mark.parametrize("name", sorted(CASES))
def test_dataflow_fp64_sweep_matches_oracle_and_step_launches(ctxs, name):
    from oracle import qfs_oracle as O
    from paper_2405_12866_gb300 import qfs
    df, steps = ctxs
    n, pairs, U, Psi, G0 = _inputs(name)
    g1, e1, c1 = df.sweep_once(n, pairs, U, Psi, G0, qfs.QFS_FP64)
    g2, e2, c2 = steps.sweep_once(n, pairs, U, Psi, G0, qfs.QFS_FP64)
    assert np.max(np.abs(g1 - g2)) < 1e-11
    assert np.max(np.abs(c1 - c2)) < 1e-12
    assert np.max(np.abs(e1 - e2)) < 1e-11 * max(1.0, np.max(np.abs(e2)))
    UPsi = U @ Psi
    for s in range(G0.shape[0]):
        r = O.sweep(UPsi, Psi, G0[s], pairs, n)
        assert abs(c1[s] - r.cost) < 1e-12
        assert np.max(np.abs(e1[s] - r.envs)) < 1e-11 * max(1.0, np.max(np.abs(r.envs)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_dataflow_mixed_sweep_matches_step_launches(ctxs, name):
    from paper_2405_12866_gb300 import qfs
    df, steps = ctxs
    n, pairs, U, Psi, G0 = _inputs(name)
    if Psi.shape[1] % 2:
        pytest.skip("complex64 dataflow sweeps need an even M")
    g1, e1, c1 = df.sweep_once(n, pairs, U, Psi, G0, qfs.QFS_MIXED)
    g2, e2, c2 = steps.sweep_once(n, pairs, U, Psi, G0, qfs.QFS_MIXED)
    L = len(pairs)
    dg = np.array([[np.max(np.abs(g1[s, k] - g2[s, k])) for k in range(L)] for s in range(G0.shape[0])])
    de = np.array([[np.max(np.abs(e1[s, k] - e2[s, k])) for k in range(L)] for s in range(G0.shape[0])])
    assert np.max(dg) < 1e-4, f"gate differences per (start, gate):\n{dg}\nenv differences:\n{de}\ncosts {c1} {c2}"
    assert np.max(de) < 1e-4 * max(1.0, np.max(np.abs(e2)))
    assert np.max(np.abs(c1 - c2)) < 1e-4, f"costs {c1} vs {c2}"


def test_dataflow_instantiation_matches_step_launches(ctxs):
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    df, steps = ctxs
    p = w.chain_n3()
    for prec in (qfs.QFS_FP64, qfs.QFS_MIXED):
        prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=p.max_sweeps, dist_tol=p.tol, precision=prec)
        a = df.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
        b = steps.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
        assert a.converged == b.converged
        assert a.best_start == b.best_start
        assert abs(a.sweeps - b.sweeps) <= 2
    p = w.brick_n8()
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=40, dist_tol=p.tol, precision=qfs.QFS_FP64)
    a = df.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
    b = steps.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
    assert a.sweeps == b.sweeps == 40
    assert abs(a.cost - b.cost) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dataflow_full_size_sweeps_repeat_exactly(ctxs, prec):
    """Starts run at different steps at the same time; steps differ in chunk
    count.  Repeated full-size sweeps must agree with the per-step launches
    every time (a slot shared by two starts would show up as a wrong start)."""
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    df, steps = ctxs
    p = w.brick_n12(target_seed=3) if prec == "mixed" else w.brick_n8(target_seed=3)
    pr = qfs.QFS_MIXED if prec == "mixed" else qfs.QFS_FP64
    Psi, G = p.samples(), p.init_gates()
    g2, _, c2 = steps.sweep_once(p.n, p.pairs, p.U, Psi, G, pr, want_envs=False)
    tol_g = 1e-4 if prec == "mixed" else 1e-11
    tol_c = 1e-5 if prec == "mixed" else 1e-12
    first = None
    for rep in range(4):
        g1, _, c1 = df.sweep_once(p.n, p.pairs, p.U, Psi, G, pr, want_envs=False)
        assert np.max(np.abs(g1 - g2)) < tol_g, f"repeat {rep}"
        assert np.max(np.abs(c1 - c2)) < tol_c, f"repeat {rep}"
        if first is None:
            first = (g1, c1)
        else:
            # the reduction order is fixed: repeats are bitwise identical
            assert np.array_equal(first[0], g1) and np.array_equal(first[1], c1), f"repeat {rep}"
