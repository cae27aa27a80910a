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


@pytest.mark.parametrize("target,M0,min_sweeps,dist",
                         [(1, 2, 0, 0), (0, 2, 0, 0), (0, 2, 6, 0), (4, 4, 0, 0), (7, 2, 0, 0), (3, 4, 0, 0)])
def test_chain_n3_restart_matches_oracle(ctx, target, M0, min_sweeps, dist):
    """Haar training and validation states drawn by the library against the
    oracle's outer loop on the generator's draws: target 1 stalls (cost
    0.0555 on both starts, no M converges), the others converge.  Both sides
    run the same FP64 updates and differ only in the order of rounded sums,
    so the returned gates agree to ~3e-14 (measured); 1e-11 bounds that with
    room for the amplification by ~200 sweeps.  (Computational-basis states
    make the first gate's environment rank-deficient at small M, where the
    update is not unique; they are checked for validity below.)"""
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    p = w.chain_n3(target_seed=target)
    seed, S, otr = 77, 2, 0.1
    tr = lambda M, a: w.training_states(dist, w.attempt_seed(seed, a), p.n, M)
    va = lambda M, a: w.training_states(dist, w.attempt_seed(seed, a), p.n, M, stream=w.STREAM_VALIDATION)
    want = o.instantiate_restarting(p.U, tr, va, w.initial_gates(seed, S, p.L), p.pairs, p.n, 1e-10, 200, M0, otr,
                                    min_sweeps=min_sweeps)
    prm = qfs.default_params(M=M0, multistarts=S, max_sweeps=200, dist_tol=1e-10, seed=seed, min_sweeps=min_sweeps,
                             restart_doubling=1, overtrain_ratio=otr, precision=qfs.QFS_FP64,
                             training_distribution=dist)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm)
    assert got.training_states == want.training_states
    assert got.converged == want.converged
    assert abs(got.sweeps - want.sweeps) <= 1
    assert abs(got.cost - want.cost) < 1e-11
    if want.converged:
        assert got.cost <= 1e-10
        assert got.best_start == want.best_start
        assert np.max(np.abs(got.gates - want.gates)) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_brick_n8_restart_reaches_a_generalising_solution(ctx, prec):
    """At its literal M = 16 this target stalls near cost 1.3 on every start;
    the outer loop doubles M until the validation cost agrees with the
    training cost and returns gates whose full-unitary cost (Eq. 1) per
    state is within the paper's bound dist_tol (1 + overtrain_ratio)
    (measured: 7.8e-9 in FP64, 9.1e-9 in the mixed path, against 1.1e-8)."""
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
    assert per_state <= p.tol * (1 + otr)


@pytest.mark.parametrize("dist", [0, 1])
def test_fixed_m_instantiation_with_library_drawn_states(ctx, dist):
    """Seed-driven instantiation with either training distribution equals
    the oracle's run on the generator's draw of the same states."""
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    n, seed, S, M = 6, 31, 4, 16
    pairs = w.brick_pairs(n, 4)
    U = w.target_unitary(w.haar_gates(1001, w.STREAM_TARGET_GATES, len(pairs)), pairs, n)
    want = o.instantiate(U, w.training_states(dist, seed, n, M), w.initial_gates(seed, S, len(pairs)), pairs, n,
                         1e-8, 300)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=300, dist_tol=1e-8, seed=seed,
                             precision=qfs.QFS_FP64, training_distribution=dist)
    got = ctx.instantiate(n, pairs, U, prm)
    assert got.converged == want.converged
    assert abs(got.sweeps - want.sweeps) <= 1
    if want.converged:
        assert got.best_start == want.best_start
        assert np.max(np.abs(got.gates - want.gates)) < 1e-6


def test_rank_deficient_environments_get_optimal_updates(ctx):
    """M = 2 computational-basis states: the first gate's environment has
    rank <= 2, so its polar factor is not unique.  What is unique is checked
    against the oracle: every environment as used (rebuilt by the oracle
    from the kernel's own updated gates), the objective Re Tr(u E) = the
    nuclear norm of E (the maximum over unitaries), and the cost."""
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    n, S, M = 6, 4, 2
    pairs = w.brick_pairs(n, 4)
    L = len(pairs)
    U = w.target_unitary(w.haar_gates(1002, w.STREAM_TARGET_GATES, L), pairs, n)
    Psi = w.basis_states(8, n, M)
    G0 = w.initial_gates(8, S, L)
    new, envs, costs = ctx.sweep_once(n, pairs, U, Psi, G0, precision=qfs.QFS_FP64)
    rank1 = 0
    for i in range(S):
        for k in range(L, 0, -1):
            B = Psi
            for j in range(k - 1):
                B = o.apply_gate(B, G0[i, j], pairs[j], n)
            Phi = U @ Psi
            for j in range(L - 1, k - 1, -1):
                Phi = o.apply_gate(Phi, new[i, j].conj().T, pairs[j], n)
            E = o.environment(B, Phi, pairs[k - 1], n)
            assert np.max(np.abs(envs[i, k - 1] - E)) < 1e-12
            u = new[i, k - 1]
            assert np.max(np.abs(u.conj().T @ u - np.eye(4))) < 1e-12
            sv = np.linalg.svd(E, compute_uv=False)
            rank1 += int(k == 1 and sv[2] < 1e-12 * sv[0])
            assert abs(np.real(np.trace(u @ E)) - np.sum(sv)) < 1e-12 * (1 + np.sum(sv))
        assert abs(costs[i] - o.sample_cost(U @ Psi, Psi, new[i], pairs, n)) < 1e-12
    assert rank1 == S  # the first gate's environment is rank-deficient for every start


@pytest.mark.parametrize("n,M0", [(3, 2), (6, 2), (6, 8)])
def test_restart_with_basis_states_returns_a_valid_result(ctx, n, M0):
    """Double-and-restart with computational-basis training and validation
    states (Appendix D).  The update is not unique at small M, so the run is
    checked for validity: M doubled from M0, the reported cost is the
    sample cost of the returned gates on the last attempt's training states
    (regenerated by the seeded generator), and a converged result meets the
    success relation c_train <= dist_tol, c_val <= (1 + otr) c_train."""
    from oracle import qfs_oracle as o
    from paper_2405_12866_gb300 import qfs
    from paper_2405_12866_gb300 import workloads as w
    pairs = w.chain_pairs(3, 4) if n == 3 else w.brick_pairs(n, 4)
    U = w.target_unitary(w.haar_gates(1003 + n, w.STREAM_TARGET_GATES, len(pairs)), pairs, n)
    seed, S, otr, tol, N = 41, 4, 0.1, 1e-10, 1 << n
    prm = qfs.default_params(M=M0, multistarts=S, max_sweeps=400, dist_tol=tol, seed=seed, restart_doubling=1,
                             overtrain_ratio=otr, precision=qfs.QFS_FP64, training_distribution=1)
    got = ctx.instantiate(n, pairs, U, prm)
    M = got.training_states
    a = int(np.log2(M // M0))
    assert M0 <= M <= N and M == M0 << a
    sa = w.attempt_seed(seed, a)
    Psi = w.basis_states(sa, n, M)
    assert abs(got.cost - o.sample_cost(U @ Psi, Psi, got.gates, pairs, n)) < 1e-12
    if got.converged:
        assert got.cost <= tol
        if M < N:
            Pv = w.basis_states(sa, n, M, stream=w.STREAM_VALIDATION)
            assert o.sample_cost(U @ Pv, Pv, got.gates, pairs, n) <= (1 + otr) * got.cost + 1e-14
