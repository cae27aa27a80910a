"""GPU parity: the CUDA path through the C-ABI against the CPU oracle on the
same seeded inputs.

Tolerances: FP64 path, per sweep, 1e-10 max-abs on gates and 1e-12 on the
cost; complex64 sweeps, 1e-4 max-abs on gates per sweep.  Gates are compared
only where the update is unique (sigma_min(E) > 1e-8 sigma_max(E)); a
rank-deficient E admits any optimal completion, which is checked by its
properties instead.
"""
import numpy as np
import pytest

from oracle import qfs_oracle as o
from paper_2405_12866_gb300 import workloads as w

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


def _qfs():
    from paper_2405_12866_gb300 import qfs
    return qfs


def oracle_sweeps(U, Psi, G, pairs, n, beta=0.0):
    UPsi = U @ Psi
    out = [o.sweep(UPsi, Psi, G[s], pairs, n, beta) for s in range(G.shape[0])]
    return (np.stack([r.gates for r in out]), np.stack([r.envs for r in out]),
            np.array([r.cost for r in out]))


def unique_update_mask(envs):
    sv = np.linalg.svd(envs, compute_uv=False)
    return sv[..., -1] > 1e-8 * sv[..., 0]


def gate_errors_ok(got, want, envs, tol):
    """Max-abs gate error within tol where the update is unique and well
    conditioned; with condition number kappa > 1e4 the allowed error grows as
    1e-14 kappa (both sides round at the level eps * kappa)."""
    sv = np.linalg.svd(envs, compute_uv=False)
    kappa = sv[..., 0] / np.maximum(sv[..., -1], 1e-300)
    uniq = sv[..., -1] > 1e-8 * sv[..., 0]
    err = np.max(np.abs(got - want), axis=(-2, -1))
    allowed = np.maximum(tol, 1e-14 * kappa)
    return bool(np.all(err[uniq] <= allowed[uniq]))


# ------------------------------------------------------------- update step

def test_gate_update_random_and_damped(ctx):
    E = w.complex_normals(3, 9, 0, 16 * 300).reshape(300, 4, 4)
    G0 = w.haar_gates(4, 3, 300)
    got = ctx.gate_update(E)
    want = np.stack([o.gate_update(e) for e in E])
    assert np.max(np.abs(got - want)) < 1e-12
    got_b = ctx.gate_update(E, G0, 0.3)
    want_b = np.stack([o.gate_update(e, g, 0.3) for e, g in zip(E, G0)])
    assert np.max(np.abs(got_b - want_b)) < 1e-12


def test_gate_update_ill_conditioned_and_rank_deficient(ctx):
    rng_E = w.complex_normals(5, 9, 0, 16 * 64).reshape(64, 4, 4)
    Es = []
    for i, e in enumerate(rng_E):
        X, d, Yh = np.linalg.svd(e)
        # conditioning from 1 down to exactly singular
        d = np.array([1.0, 0.5, 10.0 ** -(i % 7), 0.0 if i % 4 == 0 else 10.0 ** -(i % 15)])
        Es.append(X @ np.diag(d) @ Yh)
    Es.append(np.zeros((4, 4), complex))
    Es.append(np.outer([1, 1j, 0, 0], [0, 1, 1, 1]).astype(complex))
    Es = np.array(Es)
    got = ctx.gate_update(Es)
    for e, g in zip(Es, got):
        assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-12
        nuc = np.sum(np.linalg.svd(e, compute_uv=False))
        assert abs(np.real(np.trace(g @ e)) - nuc) < 1e-12 * max(1.0, nuc)
    want = np.stack([o.gate_update(e) for e in Es])
    assert gate_errors_ok(got, want, Es, 1e-12)


# ------------------------------------------------------------ one FP64 sweep

SWEEP_CASES = [
    # name, n, pairs, M, S
    ("chain_n3_M4", 3, w.chain_pairs(3, 4), 4, 1),
    ("n2_single_gate_M4", 2, [(0, 1)], 4, 2),
    ("n2_M1", 2, [(0, 1), (1, 0)], 1, 3),
    ("n4_all_pairs_M3", 4, [(0, 1), (2, 3), (1, 3), (3, 0), (2, 1), (0, 2)], 3, 5),
    ("n5_brick_M5", 5, w.brick_pairs(5, 4), 5, 6),
    ("n6_brick_M16_S9", 6, w.brick_pairs(6, 3), 16, 9),
    ("n7_M64", 7, w.brick_pairs(7, 2) + [(6, 0)], 64, 3),
    ("n8_M256_full", 8, w.brick_pairs(8, 2), 256, 2),
    ("n10_M7", 10, w.brick_pairs(10, 2), 7, 2),
]


def _case(n, pairs, M, S, seed):
    tg = w.haar_gates(seed, w.STREAM_TARGET_GATES, len(pairs))
    U = w.target_unitary(tg, pairs, n)
    Psi = w.sample_states(seed + 1, n, M)
    G = w.initial_gates(seed + 2, S, len(pairs))
    return U, Psi, G


@pytest.mark.parametrize("name,n,pairs,M,S", SWEEP_CASES, ids=[c[0] for c in SWEEP_CASES])
def test_fp64_sweep_matches_oracle(ctx, name, n, pairs, M, S):
    qfs = _qfs()
    U, Psi, G = _case(n, pairs, M, S, 1000 + n)
    UPsi = U @ Psi
    L = len(pairs)
    for it in range(3):
        g_got, e_got, c_got = ctx.sweep_once(n, pairs, U, Psi, G, qfs.QFS_FP64)
        g_want, e_want, c_want = oracle_sweeps(U, Psi, G, pairs, n)
        for s in range(S):
            # Updates happen for k = L..1; after a rank-deficient environment
            # the update is not unique and later environments may differ.
            unique_so_far = True
            for k in range(L - 1, -1, -1):
                if not unique_so_far:
                    break
                assert np.max(np.abs(e_got[s, k] - e_want[s, k])) < 1e-10 * max(1.0, M / 4)
                assert gate_errors_ok(g_got[s, k], g_want[s, k], e_want[s, k], 1e-10)
                unique_so_far = bool(unique_update_mask(e_want[s, k]))
            if unique_so_far:
                assert abs(c_got[s] - c_want[s]) < 1e-12
            else:
                c_in = o.sample_cost(UPsi, Psi, G[s], pairs, n)
                assert -1e-12 <= c_got[s] <= c_in + 1e-12
                assert abs(c_got[s] - o.sample_cost(UPsi, Psi, g_got[s], pairs, n)) < 1e-12
        for g in g_got.reshape(-1, 4, 4):
            assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-12
        G = g_want   # next sweep starts from the oracle's gates


def test_fp64_sweep_with_beta(ctx):
    qfs = _qfs()
    n, pairs, M, S = 5, w.brick_pairs(5, 3), 8, 3
    U, Psi, G = _case(n, pairs, M, S, 77)
    g_got, _, c_got = ctx.sweep_once(n, pairs, U, Psi, G, qfs.QFS_FP64, beta=0.25)
    g_want, _, c_want = oracle_sweeps(U, Psi, G, pairs, n, beta=0.25)
    assert np.max(np.abs(g_got - g_want)) < 1e-10
    assert np.max(np.abs(c_got - c_want)) < 1e-12


# ------------------------------------------------------- one complex64 sweep

@pytest.mark.parametrize("name,n,pairs,M,S", SWEEP_CASES[3:], ids=[c[0] for c in SWEEP_CASES[3:]])
def test_mixed_sweep_within_1e4(ctx, name, n, pairs, M, S):
    qfs = _qfs()
    U, Psi, G = _case(n, pairs, M, S, 2000 + n)
    g_got, e_got, c_got = ctx.sweep_once(n, pairs, U, Psi, G, qfs.QFS_MIXED)
    g_want, e_want, _ = oracle_sweeps(U, Psi, G, pairs, n)
    assert gate_errors_ok(g_got, g_want, e_want, 1e-4)
    # the reported cost is the residual form of the swept gates
    UPsi = U @ Psi
    c_ref = np.array([o.sample_cost(UPsi, Psi, g_got[s], pairs, n) for s in range(S)])
    assert np.max(np.abs(c_got - c_ref)) < 1e-5


# ---------------------------------------------------------- full instantiation

def test_chain_n3_instantiation_matches_oracle(ctx):
    """n = 3 chain of 4 gates, M = 4, one start, 200 sweeps, tol 1e-10."""
    qfs = _qfs()
    p = w.chain_n3()
    Psi, G0 = p.samples(), p.init_gates()
    want = o.instantiate(p.U, Psi, G0, p.pairs, p.n, p.tol, p.max_sweeps)
    prm = qfs.default_params(M=p.M, multistarts=p.S, max_sweeps=p.max_sweeps, dist_tol=p.tol)
    got = ctx.instantiate(p.n, p.pairs, p.U, prm, Psi, G0)
    assert got.converged == want.converged
    assert got.sweeps == want.sweeps
    assert abs(got.cost - want.cost) < 1e-12
    assert np.max(np.abs(got.gates - want.gates)) < 1e-8


MULTI_CASES = [
    ("n4_brick2", 4, w.brick_pairs(4, 2), 8, 4, 11),
    ("n4_brick3", 4, w.brick_pairs(4, 3), 8, 6, 12),
    ("n5_chain6", 5, w.chain_pairs(5, 6), 8, 8, 13),
    ("n6_brick3", 6, w.brick_pairs(6, 3), 16, 8, 14),
]


@pytest.mark.parametrize("name,n,pairs,M,S,seed", MULTI_CASES, ids=[c[0] for c in MULTI_CASES])
def test_fp64_multistart_matches_oracle(ctx, name, n, pairs, M, S, seed):
    qfs = _qfs()
    p = w.make_problem(name, n, pairs, M, S, seed, seed + 50, 1e-10, 400)
    Psi, G0 = p.samples(), p.init_gates()
    want = o.instantiate(p.U, Psi, G0, pairs, n, p.tol, p.max_sweeps)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=p.max_sweeps, dist_tol=p.tol)
    got = ctx.instantiate(n, pairs, p.U, prm, Psi, G0)
    assert got.converged == want.converged
    assert got.sweeps == want.sweeps
    assert got.best_start == want.best_start
    assert np.max(np.abs(got.start_costs - want.start_costs)) < 1e-10
    assert np.max(np.abs(got.gates - want.gates)) < 1e-7


@pytest.mark.parametrize("name,n,pairs,M,S,seed", MULTI_CASES, ids=[c[0] for c in MULTI_CASES])
def test_mixed_converges_on_the_same_targets(ctx, name, n, pairs, M, S, seed):
    qfs = _qfs()
    p = w.make_problem(name, n, pairs, M, S, seed, seed + 50, 1e-8, 400)
    Psi, G0 = p.samples(), p.init_gates()
    want = o.instantiate(p.U, Psi, G0, pairs, n, p.tol, p.max_sweeps)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=p.max_sweeps, dist_tol=p.tol,
                             precision=qfs.QFS_MIXED)
    got = ctx.instantiate(n, pairs, p.U, prm, Psi, G0)
    assert got.converged == want.converged
    if got.converged:
        assert got.cost <= 1e-8
        # the oracle's FP64 cost of the returned gates agrees with the reported one
        c = o.sample_cost(p.U @ Psi, Psi, got.gates, pairs, n)
        assert c <= 1e-8 and abs(c - got.cost) < 1e-11
        for g in got.gates:
            assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_start_groups_do_not_change_results(ctx, precision):
    """Concurrent groups of starts give bitwise the same run as one group."""
    qfs = _qfs()
    n, pairs, M, S = 6, w.brick_pairs(6, 3), 16, 12
    p = w.make_problem("g", n, pairs, M, S, 61, 62, 1e-8, 300)
    Psi, G0 = p.samples(), p.init_gates()
    runs = []
    for groups in (1, 3, 5):
        prm = qfs.default_params(M=M, multistarts=S, max_sweeps=300, dist_tol=1e-8,
                                 precision=precision, start_groups=groups)
        runs.append(ctx.instantiate(n, pairs, p.U, prm, Psi, G0))
    for r in runs[1:]:
        assert r.sweeps == runs[0].sweeps and r.best_start == runs[0].best_start
        assert np.array_equal(r.gates, runs[0].gates)
        assert np.array_equal(r.start_costs, runs[0].start_costs)


def test_seeded_entry_point_equals_explicit_inputs(ctx):
    qfs = _qfs()
    n, pairs, M, S = 4, w.brick_pairs(4, 3), 8, 3
    p = w.make_problem("s", n, pairs, M, S, 5, 6, 1e-10, 100)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=100, dist_tol=1e-10, seed=777)
    a = ctx.instantiate(n, pairs, p.U, prm)
    b = ctx.instantiate(n, pairs, p.U, prm, w.sample_states(777, n, M), w.initial_gates(777, S, len(pairs)))
    assert a.sweeps == b.sweeps and a.best_start == b.best_start
    assert np.max(np.abs(a.gates - b.gates)) < 1e-12


def test_device_entry_point_equals_host(ctx):
    import torch
    qfs = _qfs()
    n, pairs, M, S = 5, w.brick_pairs(5, 3), 8, 4
    p = w.make_problem("d", n, pairs, M, S, 21, 22, 1e-10, 200)
    Psi, G0 = p.samples(), p.init_gates()
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=200, dist_tol=1e-10)
    host = ctx.instantiate(n, pairs, p.U, prm, Psi, G0)
    dev = torch.device("cuda:0")
    out = torch.zeros((len(pairs), 4, 4), dtype=torch.complex128, device=dev)
    got = ctx.instantiate_dev(n, pairs, torch.from_numpy(p.U).to(dev), torch.from_numpy(Psi).to(dev),
                              torch.from_numpy(np.ascontiguousarray(G0)).to(dev), prm, out)
    assert got.sweeps == host.sweeps and got.best_start == host.best_start
    assert np.max(np.abs(out.cpu().numpy() - host.gates)) < 1e-13


def test_nonfinite_target_is_rejected(ctx):
    qfs = _qfs()
    n, pairs = 3, [(0, 1), (1, 2)]
    U = np.eye(8, dtype=complex)
    U[3, 2] = np.nan
    prm = qfs.default_params(M=4, multistarts=1, max_sweeps=3)
    with pytest.raises(qfs.QfsError) as e:
        ctx.instantiate(n, pairs, U, prm)
    assert e.value.code == qfs.QFS_ENONFINITE


def test_plateau_matches_oracle(ctx):
    qfs = _qfs()
    n, pairs, M, S = 5, w.brick_pairs(5, 6), 4, 2
    p = w.make_problem("pl", n, pairs, M, S, 131, 132, 1e-14, 5000)
    Psi, G0 = p.samples(), p.init_gates()
    want = o.instantiate(p.U, Psi, G0, pairs, n, 1e-14, 5000, plateau_window=5, diff_tol_r=1e-3,
                         min_sweeps=6)
    prm = qfs.default_params(M=M, multistarts=S, max_sweeps=5000, dist_tol=1e-14, plateau_window=5,
                             diff_tol_r=1e-3, min_sweeps=6)
    got = ctx.instantiate(n, pairs, p.U, prm, Psi, G0)
    assert got.sweeps == want.sweeps
    assert got.best_start == want.best_start
    assert np.max(np.abs(got.start_costs - want.start_costs)) < 1e-10


# ------------------------------------------------------------ full-size cases

def test_brick_n8_fp64_sweep_full_size(ctx):
    """n = 8 brick wall of 28 gates, M = 16, 16 starts: one sweep, all starts."""
    qfs = _qfs()
    p = w.brick_n8(target_seed=0)
    Psi, G = p.samples(), p.init_gates()
    g_got, e_got, c_got = ctx.sweep_once(p.n, p.pairs, p.U, Psi, G, qfs.QFS_FP64)
    g_want, e_want, c_want = oracle_sweeps(p.U, Psi, G, p.pairs, p.n)
    assert gate_errors_ok(g_got, g_want, e_want, 1e-10)
    assert np.max(np.abs(c_got - c_want)) < 1e-12


def test_brick_n12_mixed_sweep_full_size(ctx):
    """n = 12 brick wall of 17 gates, M = 32, 32 starts, complex64 sweep: every
    start's gates within 1e-4 of the oracle's FP64 sweep."""
    qfs = _qfs()
    p = w.brick_n12(target_seed=0)
    Psi, G = p.samples(), p.init_gates()
    g_got, e_got, c_got = ctx.sweep_once(p.n, p.pairs, p.U, Psi, G, qfs.QFS_MIXED)
    sample = range(0, p.S, 4)   # the oracle computes 8 of the 32 starts
    UPsi = p.U @ Psi
    for s in sample:
        r = o.sweep(UPsi, Psi, G[s], p.pairs, p.n)
        assert np.max(np.abs(g_got[s] - r.gates)) < 1e-4
        assert abs(c_got[s] - o.sample_cost(UPsi, Psi, g_got[s], p.pairs, p.n)) < 1e-5
