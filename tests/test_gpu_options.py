"""Context options through the C-ABI: the alternative sweep paths against
the default ones and the oracle, and the two failure paths that can be
provoked safely.

- QFS_OPT_FUSED_UPDATE = 0 runs each gate update as its own launch after the
  backward step; QFS_OPT_TWO_GATE_FORWARD = 0 applies one forward gate per
  dataflow step; QFS_OPT_FP64_TARGET_PRODUCT = 1 forms U Psi in FP64 in
  mixed runs.  Each must give the oracle's sweep (FP64: 1e-10 on gates,
  1e-12 on the cost; complex64: 1e-4 on gates).
- QFS_OPT_WAIT_LIMIT = 1: the dataflow sweep's dependency waits give up
  after one poll, which happens as soon as an item's previous step is still
  running.  The kernel sets its error word and every CTA returns; the call
  must return QFS_ETIMEOUT and the context must still give the right answer
  once the limit is restored.  Nothing faults, traps or waits without bound.
- QFS_OPT_WORKSPACE_CAP: a call that needs more device workspace than the
  cap returns QFS_ENOMEM before it allocates.
"""
import numpy as np
import pytest

from oracle import qfs_oracle as o
from paper_2405_12866_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qfs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import build, qfs as q
    build.build()
    return q


def _ctx(qfs, **opts):
    c = qfs.Context(0)
    for k, v in opts.items():
        c.set_option(getattr(qfs, "QFS_OPT_" + k), v)
    return c


def _problem(n, pairs, M, S, seed):
    gt = w.haar_gates(seed, w.STREAM_TARGET_GATES, len(pairs))
    U = w.target_unitary(gt, pairs, n)
    return U, w.sample_states(seed + 1, n, M), w.initial_gates(seed + 2, S, len(pairs))


def _oracle(U, Psi, G, pairs, n):
    UPsi = U @ Psi
    rs = [o.sweep(UPsi, Psi, G[s], pairs, n) for s in range(G.shape[0])]
    return np.stack([r.gates for r in rs]), np.array([r.cost for r in rs])


def test_options_round_trip_and_reject_bad_values(qfs):
    with _ctx(qfs) as c:
        assert c.get_option(qfs.QFS_OPT_WAIT_LIMIT) == 1 << 25
        assert c.get_option(qfs.QFS_OPT_WORKSPACE_CAP) == 0
        for opt, default in ((qfs.QFS_OPT_FUSED_UPDATE, 1), (qfs.QFS_OPT_DATAFLOW, 1),
                             (qfs.QFS_OPT_TWO_GATE_FORWARD, 1), (qfs.QFS_OPT_FP64_TARGET_PRODUCT, 0)):
            assert c.get_option(opt) == default
            c.set_option(opt, 1 - default)
            assert c.get_option(opt) == 1 - default
        with pytest.raises(qfs.QfsError) as e:
            c.set_option(qfs.QFS_OPT_WAIT_LIMIT, 0)
        assert e.value.code == qfs.QFS_EINVAL
        with pytest.raises(qfs.QfsError) as e:
            c.set_option(99, 1)
        assert e.value.code == qfs.QFS_EINVAL


@pytest.mark.parametrize("n,pairs,M,S", [
    (6, [(0, 1), (2, 3), (4, 5), (1, 2), (3, 4), (0, 1), (2, 3)], 8, 4),
    (5, [(0, 1), (1, 2), (2, 3), (3, 4), (2, 3), (1, 2), (0, 1)], 8, 3),
    (4, [(0, 1), (0, 1), (1, 0), (2, 3), (3, 2), (1, 2)], 4, 4),
])
def test_separate_update_launch_matches_oracle(qfs, n, pairs, M, S):
    U, Psi, G = _problem(n, pairs, M, S, 611)
    g_o, c_o = _oracle(U, Psi, G, pairs, n)
    with _ctx(qfs, DATAFLOW=0, FUSED_UPDATE=0) as c:
        g, _, cost = c.sweep_once(n, pairs, U, Psi, G, qfs.QFS_FP64)
        assert np.max(np.abs(g - g_o)) < 1e-10
        assert np.max(np.abs(cost - c_o)) < 1e-12
        g32, _, _ = c.sweep_once(n, pairs, U, Psi, G, qfs.QFS_MIXED)
        assert np.max(np.abs(g32 - g_o)) < 1e-4


@pytest.mark.parametrize("n,layers,M,S", [(8, 6, 8, 4), (12, 3, 32, 4)])
def test_one_gate_forward_steps_match_two_gate_steps_and_oracle(qfs, n, layers, M, S):
    pairs = w.brick_pairs(n, layers)
    U, Psi, G = _problem(n, pairs, M, S, 612)
    with _ctx(qfs) as a, _ctx(qfs, TWO_GATE_FORWARD=0) as b:
        for prec, tg in ((qfs.QFS_FP64, 1e-10), (qfs.QFS_MIXED, 1e-4)):
            g1, _, c1 = a.sweep_once(n, pairs, U, Psi, G, prec, want_envs=False)
            g2, _, c2 = b.sweep_once(n, pairs, U, Psi, G, prec, want_envs=False)
            assert np.max(np.abs(g1 - g2)) < tg
            assert np.max(np.abs(c1 - c2)) < (1e-12 if prec == qfs.QFS_FP64 else 1e-5)
    if n <= 8:
        g_o, c_o = _oracle(U, Psi, G, pairs, n)
        assert np.max(np.abs(g2 - g_o)) < 1e-4


def test_fp64_target_product_in_mixed_runs_gives_the_same_result(qfs):
    p = w.brick_n8(target_seed=5)
    prm = qfs.default_params(M=p.M, multistarts=4, max_sweeps=30, dist_tol=p.tol, precision=qfs.QFS_MIXED)
    Psi, G = p.samples(), p.init_gates()[:4]
    with _ctx(qfs) as a, _ctx(qfs, FP64_TARGET_PRODUCT=1) as b:
        ra = a.instantiate(p.n, p.pairs, p.U, prm, Psi, G)
        rb = b.instantiate(p.n, p.pairs, p.U, prm, Psi, G)
    assert ra.sweeps == rb.sweeps
    assert np.max(np.abs(ra.start_costs - rb.start_costs)) < 1e-6
    assert abs(ra.cost - rb.cost) < 1e-6


def test_exhausted_dependency_wait_returns_timeout_and_context_recovers(qfs):
    p = w.brick_n12(target_seed=7)
    prm = qfs.default_params(M=p.M, multistarts=8, max_sweeps=3, dist_tol=p.tol, precision=qfs.QFS_MIXED)
    Psi, G = p.samples(), p.init_gates()[:8]
    with _ctx(qfs) as ref:
        want = ref.instantiate(p.n, p.pairs, p.U, prm, Psi, G)
    with _ctx(qfs, WAIT_LIMIT=1) as c:
        with pytest.raises(qfs.QfsError) as e:
            c.instantiate(p.n, p.pairs, p.U, prm, Psi, G)
        assert e.value.code == qfs.QFS_ETIMEOUT
        c.set_option(qfs.QFS_OPT_WAIT_LIMIT, 1 << 25)
        got = c.instantiate(p.n, p.pairs, p.U, prm, Psi, G)
    assert got.sweeps == want.sweeps == 3
    assert np.array_equal(got.start_costs, want.start_costs)
    assert np.array_equal(got.gates, want.gates)


def test_workspace_cap_gives_enomem_before_allocating(qfs):
    p = w.brick_n8(target_seed=2)
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=2, dist_tol=p.tol)
    with _ctx(qfs, WORKSPACE_CAP=1 << 20) as c:
        with pytest.raises(qfs.QfsError) as e:
            c.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
        assert e.value.code == qfs.QFS_ENOMEM
        assert "cap" in str(e.value)
        c.set_option(qfs.QFS_OPT_WORKSPACE_CAP, 0)
        r = c.instantiate(p.n, p.pairs, p.U, prm, p.samples(), p.init_gates())
        assert r.sweeps == 2


@pytest.mark.parametrize("win", [1, 3, 5])
def test_plateau_window_length_on_the_gpu(qfs, win):
    """One gate on three qubits with a target it cannot reach: the first
    update is already optimal and the cost stays constant, so plateau
    detection with a window of w sweeps ends every run at sweep w + 1 (the
    oracle's pin of the same rule), in FP64, in the mixed path and in the
    batched form."""
    n, pairs = 3, [(0, 1)]
    U = w.target_unitary(w.haar_gates(141, w.STREAM_TARGET_GATES, 2), [(0, 1), (1, 2)], n)
    Psi, G0 = w.sample_states(142, n, 8), w.initial_gates(143, 2, 1)
    want = o.instantiate(U, Psi, G0, pairs, n, 0.0, 100, plateau_window=win, diff_tol_r=1e-3, min_sweeps=0)
    assert want.sweeps == win + 1
    with _ctx(qfs) as c:
        for prec in (qfs.QFS_FP64, qfs.QFS_MIXED):
            prm = qfs.default_params(M=8, multistarts=2, max_sweeps=100, dist_tol=0.0, precision=prec,
                                     plateau_window=win, diff_tol_r=1e-3, min_sweeps=0)
            r = c.instantiate(n, pairs, U, prm, Psi, G0)
            assert r.sweeps == win + 1, (prec, r.sweeps)
        prm = qfs.default_params(M=8, multistarts=2, max_sweeps=100, dist_tol=0.0, plateau_window=win,
                                 diff_tol_r=1e-3, min_sweeps=0, refine_sweeps_max=0)
        _, info = c.instantiate_batch([(n, pairs, U)], prm, [Psi], [G0])
        assert info[0]["sweeps"] == win + 1, info[0]
