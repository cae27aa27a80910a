"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each check is written as a function that returns True when the pin holds, so
that the planted-mistake test at the bottom can run the same checks against
deliberately broken copies of the oracle and show that each mistake is caught.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import qfs_oracle as o
from paper_2405_12866_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------- brute-force pieces

def embed_full(g, pair, n):
    """Dense N x N matrix of gate g on `pair`, built entry by entry from the
    bit convention: nonzero only where the untouched bits agree."""
    N = 1 << n
    a, b = pair
    pa, pb = n - 1 - a, n - 1 - b
    keep = ~((1 << pa) | (1 << pb))
    G = np.zeros((N, N), dtype=np.complex128)
    for i in range(N):
        li = 2 * ((i >> pa) & 1) + ((i >> pb) & 1)
        for j in range(N):
            if (i & keep) != (j & keep):
                continue
            lj = 2 * ((j >> pa) & 1) + ((j >> pb) & 1)
            G[i, j] = g[li, lj]
    return G


def kron_embed(g, q, n):
    """Adjacent pair (q, q+1): I_{2^q} (x) g (x) I_{2^(n-q-2)} (qubit 0 leftmost)."""
    return np.kron(np.kron(np.eye(1 << q), g), np.eye(1 << (n - q - 2)))


def dense_circuit(gates, pairs, n):
    C = np.eye(1 << n, dtype=np.complex128)
    for g, p in zip(gates, pairs):
        C = embed_full(g, p, n) @ C
    return C


def rand_problem(n, pairs, M, seed):
    tg = w.haar_gates(seed, w.STREAM_TARGET_GATES, len(pairs))
    U = dense_circuit(tg, pairs, n)
    Psi = w.sample_states(seed + 11, n, M)
    G = w.initial_gates(seed + 12, 1, len(pairs))[0]
    return U, Psi, G


ALL_PAIRS_4 = [(a, b) for a in range(4) for b in range(4) if a != b]
MIXED_PAIRS = [(0, 1), (2, 3), (1, 2), (3, 0), (0, 2), (1, 3)]


# ------------------------------------------------------------ pin checks

def check_apply(orc, n=4):
    X = w.sample_states(5, n, 3)
    gs = w.haar_gates(6, w.STREAM_TARGET_GATES, len(ALL_PAIRS_4))
    return all(np.allclose(orc.apply_gate(X, g, p, n), embed_full(g, p, n) @ X, atol=1e-13)
               for g, p in zip(gs, ALL_PAIRS_4))


def check_kron(orc, n=5):
    pairs = [(0, 1), (3, 4), (1, 2), (2, 3), (0, 1)]
    gs = w.haar_gates(7, w.STREAM_TARGET_GATES, len(pairs))
    C = np.eye(1 << n)
    for g, (q, _) in zip(gs, pairs):
        C = kron_embed(g, q, n) @ C
    return np.allclose(orc.circuit_unitary(gs, pairs, n), C, atol=1e-12)


def check_env_definition(orc, n=4):
    """E[y][x] = sum_j <Phi_j| (e_xy embedded) |B_j>, for all 16 basis matrices."""
    B = w.sample_states(8, n, 5)
    Phi = w.sample_states(9, n, 5)
    for p in MIXED_PAIRS:
        E = orc.environment(B, Phi, p, n)
        for x in range(4):
            for y in range(4):
                e = np.zeros((4, 4))
                e[x, y] = 1.0
                want = np.trace(Phi.conj().T @ embed_full(e, p, n) @ B)
                if abs(E[y, x] - want) > 1e-13:
                    return False
    return True


def check_sweep_objectives(orc, n=4):
    """At step k the environment pairs with the circuit whose gates k+1..L
    are already new: Re Tr(g_k,old E_k) and Re Tr(g_k,new E_k) both equal
    Re sum_j <psi_j|U^dag C|psi_j> for the matching dense circuit."""
    pairs = MIXED_PAIRS
    U, Psi, G = rand_problem(n, pairs, 6, 21)
    r = orc.sweep(U @ Psi, Psi, G, pairs, n)
    L = len(pairs)
    for k in range(1, L + 1):
        before = list(G[:k]) + list(r.gates[k:])
        after = list(G[:k - 1]) + list(r.gates[k - 1:])
        t_before = np.real(np.trace(Psi.conj().T @ U.conj().T @ dense_circuit(before, pairs, n) @ Psi))
        t_after = np.real(np.trace(Psi.conj().T @ U.conj().T @ dense_circuit(after, pairs, n) @ Psi))
        if abs(np.real(np.trace(G[k - 1] @ r.envs[k - 1])) - t_before) > 1e-12:
            return False
        if abs(r.objective[k - 1] - t_after) > 1e-12:
            return False
    return abs(r.cost - (2 - 2 / Psi.shape[1] * r.objective[0])) < 1e-14


def check_update_optimal(orc):
    """Re Tr(u_new E) equals the nuclear norm (von Neumann trace inequality)
    and beats every other unitary; u_new is the polar factor of E^dagger."""
    rng_seed = 31
    Es = w.complex_normals(rng_seed, 9, 0, 16 * 8).reshape(8, 4, 4)
    hs = w.haar_gates(rng_seed, 10, 64)
    for E in Es:
        u = orc.gate_update(E)
        if np.max(np.abs(u.conj().T @ u - np.eye(4))) > 1e-12:
            return False
        val = np.real(np.trace(u @ E))
        if abs(val - np.sum(np.linalg.svd(E, compute_uv=False))) > 1e-12:
            return False
        if any(np.real(np.trace(h @ E)) > val + 1e-12 for h in hs):
            return False
        if not np.allclose(u, scipy.linalg.polar(E.conj().T)[0], atol=1e-12):
            return False
    return True


def check_single_gate_closed_form(orc):
    """n=2, one gate, M=4: E = Psi Psi^dag U^dag = U^dag, so u_new = U."""
    U = w.haar_gates(41, 3, 1)[0]
    Psi = w.sample_states(42, 2, 4)
    G = w.haar_gates(43, 3, 1)
    r = orc.sweep(U @ Psi, Psi, G, [(0, 1)], 2)
    return np.allclose(r.gates[0], U, atol=1e-12) and abs(r.cost) < 1e-13


def check_cost_forms(orc, n=4):
    pairs = MIXED_PAIRS
    U, Psi, G = rand_problem(n, pairs, 5, 51)
    a = orc.sample_cost(U @ Psi, Psi, G, pairs, n)
    b = orc.sample_cost_trace(U @ Psi, Psi, G, pairs, n)
    direct = np.sum(np.abs(U @ Psi - dense_circuit(G, pairs, n) @ Psi) ** 2) / Psi.shape[1]
    return abs(a - b) < 1e-12 and abs(a - direct) < 1e-12


def check_full_cost(orc, n=4):
    """Eq. (1), and with M = N the sample cost is the full cost over N."""
    pairs = MIXED_PAIRS
    U, Psi, G = rand_problem(n, pairs, 1 << n, 61)
    fro = np.linalg.norm(U - dense_circuit(G, pairs, n)) ** 2
    fc = orc.full_cost(U, G, pairs, n)
    sc = orc.sample_cost(U @ Psi, Psi, G, pairs, n)
    return abs(fro - fc) < 1e-10 and abs(sc - fc / (1 << n)) < 1e-12


def check_monotone(orc, n=5, sweeps=6):
    pairs = w.brick_pairs(n, 3)
    U, Psi, G = rand_problem(n, pairs, 8, 71)
    prev = -np.inf
    for _ in range(sweeps):
        r = orc.sweep(U @ Psi, Psi, G, pairs, n)
        for k in range(len(pairs) - 1, -1, -1):   # order in which updates happen
            if r.objective[k] < prev - 1e-12:
                return False
            prev = r.objective[k]
        G = r.gates
    return True


def check_recovery(orc):
    """A target built from random gates in the same structure is recovered."""
    cases = [(4, w.brick_pairs(4, 2), 8, 4), (6, w.brick_pairs(6, 3), 16, 8),
             (5, w.chain_pairs(5, 6), 8, 8)]
    for i, (n, pairs, M, S) in enumerate(cases):
        p = w.make_problem("r", n, pairs, M, S, 80 + i, 90 + i, 1e-10, 400)
        r = orc.instantiate(p.U, p.samples(), p.init_gates(), pairs, n, 1e-10, 400)
        if not r.converged or r.cost > 1e-10:
            return False
        if orc.sample_cost(p.U @ p.samples(), p.samples(), r.gates, pairs, n) > 1e-10:
            return False
    return True


PINS = [check_apply, check_kron, check_env_definition, check_sweep_objectives,
        check_update_optimal, check_single_gate_closed_form, check_cost_forms,
        check_full_cost, check_monotone, check_recovery]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin):
    assert pin(o)


# ------------------------------------------------------- further pins

def test_same_pair_converges_in_one_sweep():
    """Every gate on one pair: the first update already reaches cost 0."""
    n, pairs = 3, [(1, 2)] * 3
    U, Psi, G = rand_problem(n, pairs, 4, 101)
    r = o.sweep(U @ Psi, Psi, G, pairs, n)
    assert abs(r.cost) < 1e-12
    assert o.sample_cost(U @ Psi, Psi, r.gates, pairs, n) < 1e-12


def test_beta_one_keeps_gate_and_half_mixes():
    E = w.complex_normals(5, 9, 0, 16).reshape(4, 4)
    g = w.haar_gates(6, 3, 1)[0]
    assert np.allclose(o.gate_update(E, g, 1.0), g, atol=1e-12)
    mix = 0.5 * E + 0.5 * g.conj().T
    assert np.allclose(o.gate_update(E, g, 0.5), scipy.linalg.polar(mix.conj().T)[0], atol=1e-12)


def test_gates_stay_unitary_over_sweeps():
    n, pairs = 5, w.brick_pairs(5, 4)
    U, Psi, G = rand_problem(n, pairs, 8, 111)
    for _ in range(10):
        G = o.sweep(U @ Psi, Psi, G, pairs, n).gates
    for g in G:
        assert np.max(np.abs(g.conj().T @ g - np.eye(4))) < 1e-12


def test_multistart_selection_rule():
    """The run stops at the first sweep where a start reaches tol and returns
    the lowest-cost start at that sweep."""
    n, pairs = 4, w.brick_pairs(4, 3)
    p = w.make_problem("m", n, pairs, 8, 6, 121, 122, 1e-10, 400)
    r = o.instantiate(p.U, p.samples(), p.init_gates(), pairs, n, 1e-10, 400)
    assert r.converged
    tr = r.cost_trace
    assert np.all(tr[:-1].min(axis=1) > 1e-10)
    assert r.best_start == int(np.argmin(tr[-1]))
    # each start in lock step equals running it alone for the same sweeps
    solo = o.instantiate(p.U, p.samples(), p.init_gates()[r.best_start:r.best_start + 1],
                         pairs, n, 0.0, r.sweeps)
    assert np.allclose(solo.gates, r.gates, atol=1e-13)


def test_plateau_stops_run():
    n, pairs = 5, w.brick_pairs(5, 6)
    p = w.make_problem("pl", n, pairs, 4, 2, 131, 132, 1e-14, 5000)
    r = o.instantiate(p.U, p.samples(), p.init_gates(), pairs, n, 1e-14, 5000,
                      plateau_window=5, diff_tol_r=1e-3, min_sweeps=6)
    assert r.sweeps < 5000
    tr = r.cost_trace
    # the last window of sweeps of a stopped start shows no relative gain
    i = int(np.argmin(tr[-1]))
    last = tr[-6:, i]
    assert all(not (abs(last[j - 1]) - abs(last[j]) > 1e-3 * abs(last[j])) for j in range(1, 6))


def test_plateau_window_length_is_exact():
    """One gate on three qubits: the gate's environment does not depend on
    the gate itself, so the first update already is the exact minimiser and
    every later sweep returns the same gate and the same cost, bit for bit
    (Eq. 2 is the optimum of the single-gate cost).  The cost never improves
    after sweep 1, so a window of w sweeps without improvement ends the run
    at sweep w + 1, or at min_sweeps if that is later (Appendix A)."""
    n, pairs = 3, [(0, 1)]
    # a target the single gate cannot reach: two gates on (0, 1), (1, 2)
    U = w.target_unitary(w.haar_gates(141, w.STREAM_TARGET_GATES, 2), [(0, 1), (1, 2)], n)
    Psi, G0 = w.sample_states(142, n, 8), w.initial_gates(143, 2, 1)
    base = o.instantiate(U, Psi, G0, pairs, n, 0.0, 8)
    assert base.cost > 1e-3
    assert np.all(base.cost_trace[1:] == base.cost_trace[0])
    for win in range(1, 7):
        r = o.instantiate(U, Psi, G0, pairs, n, 0.0, 100, plateau_window=win, diff_tol_r=1e-12, min_sweeps=0)
        assert r.sweeps == win + 1, (win, r.sweeps)
        r = o.instantiate(U, Psi, G0, pairs, n, 0.0, 100, plateau_window=win, diff_tol_r=1e-12,
                          min_sweeps=win + 4)
        assert r.sweeps == win + 4, (win, r.sweeps)


def test_target_generator_matches_kron():
    n = 5
    pairs = [(0, 1), (3, 4), (1, 2), (2, 3)]
    gs = w.haar_gates(3, w.STREAM_TARGET_GATES, len(pairs))
    C = np.eye(1 << n)
    for g, (q, _) in zip(gs, pairs):
        C = kron_embed(g, q, n) @ C
    assert np.allclose(w.target_unitary(gs, pairs, n), C, atol=1e-12)


def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = w.philox4x32_10(np.array([v[:4]], dtype=np.uint32), v[4:6])[0]
        assert [int(x) for x in out] == v[6:]


def test_sample_states_orthonormal_and_haar_moments():
    Psi = w.sample_states(3, 6, 20)
    assert np.allclose(Psi.conj().T @ Psi, np.eye(20), atol=1e-13)
    gs = w.haar_gates(17, 3, 4000)
    # Haar U(4): E|u_ij|^2 = 1/4 and E|Tr u|^2 = 1
    m2 = np.mean(np.abs(gs) ** 2, axis=0)
    assert np.max(np.abs(m2 - 0.25)) < 0.02
    tr2 = np.mean(np.abs(np.trace(gs, axis1=1, axis2=2)) ** 2)
    assert abs(tr2 - 1.0) < 0.1
    for g in gs[:50]:
        assert np.allclose(g.conj().T @ g, np.eye(4), atol=1e-13)


def test_structures():
    assert len(w.brick_pairs(8, 8)) == 28
    assert len(w.brick_pairs(12, 3)) == 17
    assert w.chain_pairs(3, 4) == [(0, 1), (1, 2), (0, 1), (1, 2)]
    probs = w.uneven_blocks(P=64)
    assert {p.n for p in probs} <= {3, 4, 5}
    assert all(2 <= p.L <= 10 and p.M == 1 << (p.n - 1) for p in probs)
    assert all(0 <= a < p.n - 1 and b == a + 1 for p in probs for a, b in p.pairs)


# ------------------------------------------------ planted-mistake check

class _Broken:
    """A copy of the oracle with one planted mistake (on the CPU only)."""

    def __init__(self, **overrides):
        for name in dir(o):
            if not name.startswith("__"):
                setattr(self, name, getattr(o, name))
        for k, v in overrides.items():
            setattr(self, k, v)
        me = self

        def sweep(UPsi, Psi, gates, pairs, n, beta=0.0):
            return _sweep_with(me, UPsi, Psi, gates, pairs, n, beta)
        if "sweep" not in overrides:
            self.sweep = sweep


def _sweep_with(m, UPsi, Psi, gates, pairs, n, beta=0.0):
    """The oracle's sweep routed through the (possibly broken) pieces of m."""
    L = len(pairs)
    M = Psi.shape[1]
    B = [Psi]
    for k in range(1, L):
        B.append(m.apply_gate(B[k - 1], gates[k - 1], pairs[k - 1], n))
    new = np.array(gates, dtype=np.complex128, copy=True)
    envs = np.zeros((L, 4, 4), dtype=np.complex128)
    obj = np.zeros(L)
    Phi = UPsi
    for k in range(L, 0, -1):
        E = m.environment(B[k - 1], Phi, pairs[k - 1], n)
        g = m.gate_update(E, new[k - 1], beta)
        envs[k - 1], new[k - 1] = E, g
        obj[k - 1] = np.real(np.trace(g @ E))
        if k > 1:
            Phi = m.apply_gate(Phi, m._dagger(g), pairs[k - 1], n)
    return o.SweepResult(new, envs, obj, float(2.0 - 2.0 / M * obj[0]))


def _circuit_unitary_with(m):
    def cu(gates, pairs, n):
        X = np.eye(1 << n, dtype=np.complex128)
        for g, p in zip(gates, pairs):
            X = m.apply_gate(X, g, p, n)
        return X
    return cu


MISTAKES = {
    "env_without_conj": dict(environment=lambda B, P, p, n: o.pair_major(B, n, p) @ o.pair_major(P, n, p).T),
    "env_transposed": dict(environment=lambda B, P, p, n: (o.pair_major(B, n, p) @ o.pair_major(P, n, p).conj().T).T),
    "update_X_Ydag": dict(gate_update=lambda E, g=None, beta=0.0: (lambda X, D, Yh: X @ Yh)(*np.linalg.svd(E))),
    "pair_swapped": dict(apply_gate=lambda X, g, p, n: o.apply_gate(X, g, (p[1], p[0]), n)),
    "gate_transposed": dict(apply_gate=lambda X, g, p, n: o.apply_gate(X, g.T, p, n)),
    "phi_update_no_dagger": dict(_dagger=lambda g: g),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_is_caught(name):
    over = dict(_dagger=lambda g: g.conj().T)
    over.update(MISTAKES[name])
    m = _Broken(**over)
    m.circuit_unitary = _circuit_unitary_with(m)

    def circuit_apply(state, gates, pairs, n):
        X = state
        for g, p in zip(gates, pairs):
            X = m.apply_gate(X, g, p, n)
        return X
    m.circuit_apply = circuit_apply
    m.sample_cost = lambda UPsi, Psi, G, pairs, n: float(
        np.sum(np.abs(UPsi - circuit_apply(Psi, G, pairs, n)) ** 2) / Psi.shape[1])
    m.sample_cost_trace = lambda UPsi, Psi, G, pairs, n: float(
        2 - 2 / Psi.shape[1] * np.real(np.vdot(UPsi, circuit_apply(Psi, G, pairs, n))))
    fast = [check_apply, check_kron, check_env_definition, check_sweep_objectives,
            check_update_optimal, check_single_gate_closed_form, check_cost_forms,
            check_monotone]
    failed = []
    for pin in fast:
        try:
            ok = pin(m)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"planted mistake {name} passed every pin"


def test_unbroken_copy_passes():
    m = _Broken(_dagger=lambda g: g.conj().T)
    for pin in [check_env_definition, check_sweep_objectives, check_single_gate_closed_form]:
        assert pin(m)


# ------------------------------------------------------ double-and-restart

def _restart_inputs(name):
    p = w.chain_n3(target_seed=1) if name == "chain_n3" else None
    tr = lambda M, a: w.sample_states(w.attempt_seed(p.seed, a), p.n, M)
    va = lambda M, a: w.sample_states(w.attempt_seed(p.seed, a), p.n, M, stream=w.STREAM_VALIDATION)
    return p, tr, va


def test_restart_without_overtraining_is_the_plain_run():
    """With an overtrain ratio no run can exceed, the outer loop is one
    attempt identical to the fixed-M instantiation."""
    p, tr, va = _restart_inputs("chain_n3")
    G0 = w.initial_gates(p.seed, 2, p.L)
    r = o.instantiate_restarting(p.U, tr, va, G0, p.pairs, p.n, 1e-10, 60, 4, 1e300)
    plain = o.instantiate(p.U, tr(4, 0), G0, p.pairs, p.n, 1e-10, 60)
    assert r.attempts == 1 and r.training_states == 4
    assert r.sweeps == plain.sweeps and r.best_start == plain.best_start
    assert abs(r.cost - plain.cost) < 1e-15
    assert np.max(np.abs(r.gates - plain.gates)) < 1e-15


def test_restart_doubles_until_the_target_generalises():
    """chain_n3 stalls at M = 4 (sample-cost plateau ~3e-4); the outer loop
    detects the gap between validation and training cost, doubles M and
    converges, and the returned gates generalise: the full-unitary cost
    (Eq. 1, all 2^n states) is below the bound dist_tol (1 + otr)."""
    p, tr, va = _restart_inputs("chain_n3")
    G0 = w.initial_gates(p.seed, 1, p.L)
    otr = 0.1
    r = o.instantiate_restarting(p.U, tr, va, G0, p.pairs, p.n, 1e-10, 200, 2, otr)
    assert r.converged and r.cost <= 1e-10
    assert r.training_states > 2 and r.training_states <= 8
    assert r.training_states & (r.training_states - 1) == 0
    assert r.attempts == int(np.log2(r.training_states)) - 1 + 1
    if r.training_states < 8:
        assert r.validation_cost <= (1 + otr) * r.cost
    # generalisation to all states: ||U - C||_F^2 / N is the M = N sample cost
    assert o.full_cost(p.U, r.gates, p.pairs, p.n) / (1 << p.n) <= 1e-10 * (1 + otr)


# ------------------------------------ training-state distribution (Appendix D)

def test_basis_draw_is_distinct_and_uniform():
    """The computational-basis draw gives M distinct unit vectors, and every
    M-subset is equally likely (partial Fisher-Yates), checked by counting
    over seeds: N = 4, M = 2 has 6 unordered pairs, each 1/6."""
    P = w.basis_states(5, 5, 32)
    assert np.array_equal(P.conj().T @ P, np.eye(32))
    assert np.array_equal(np.sort(w.basis_indices(5, 5, 32)), np.arange(32))
    counts = {}
    T = 6000
    for seed in range(T):
        key = tuple(sorted(w.basis_indices(seed, 2, 2)))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    chi2 = sum((c - T / 6) ** 2 / (T / 6) for c in counts.values())
    assert chi2 < 20.5  # 5 degrees of freedom, p ~ 0.001


def test_all_basis_states_give_the_full_cost():
    """With all N computational-basis states (in any order) the sample cost
    (residual form) equals the full cost of Eq. (1) divided by N."""
    p = w.chain_n3(target_seed=4)
    G = w.initial_gates(9, 1, p.L)[0]
    Psi = w.basis_states(3, p.n, 1 << p.n)
    c = o.sample_cost(p.U @ Psi, Psi, G, p.pairs, p.n)
    assert abs(c - o.full_cost(p.U, G, p.pairs, p.n) / (1 << p.n)) < 1e-13


def test_basis_states_blind_to_a_phase_on_unset_qubit():
    """Appendix D's example: a phase diag(1, e^{i alpha}) on qubit 0 before
    the circuit acts trivially on every basis state whose qubit 0 is |0>, so
    a training set of such states cannot tell alpha from alpha'; one Haar
    state can."""
    n = 3
    pairs = [(0, 1), (1, 2), (0, 1)]
    rest = w.haar_gates(3, w.STREAM_TARGET_GATES, 2)

    def circuit(alpha):
        ph = np.diag([1, 1, np.exp(1j * alpha), np.exp(1j * alpha)])  # on (0, 1): local index 2*b0 + b1
        return np.stack([ph, rest[0], rest[1]])

    U = w.target_unitary(circuit(0.7), pairs, n)
    zero_q0 = np.zeros((8, 4), np.complex128)
    zero_q0[[0, 1, 2, 3], [0, 1, 2, 3]] = 1.0  # rows 0..3: bit 2 (qubit 0) is 0
    assert o.sample_cost(U @ zero_q0, zero_q0, circuit(2.1), pairs, n) < 1e-28
    haar = w.sample_states(1, n, 1)
    assert o.sample_cost(U @ haar, haar, circuit(2.1), pairs, n) > 1e-3


def test_basis_states_need_more_data_than_haar_states():
    """Appendix D, numerically (seeded): on n = 6 brick-wall circuits of 10
    gates, M = 16 Haar training states give results that generalise (full
    cost / N within dist_tol (1 + otr)) while M = 16 computational-basis
    states fit the training set as well but do not generalise; at M = 32
    both do."""
    n, tol, otr = 6, 1e-8, 0.1
    pairs = w.brick_pairs(n, 4)
    gen = {w.STATES_HAAR: {}, w.STATES_BASIS: {}}
    for dist in gen:
        for M in (16, 32):
            ok = 0
            for t in range(4):
                U = w.target_unitary(w.haar_gates(1000 + t, w.STREAM_TARGET_GATES, len(pairs)), pairs, n)
                Psi = w.training_states(dist, 77 + t, n, M)
                r = o.instantiate(U, Psi, w.initial_gates(77 + t, 4, len(pairs)), pairs, n, tol, 300)
                if dist == w.STATES_BASIS:
                    assert r.cost <= tol  # the training set is fitted
                ok += o.full_cost(U, r.gates, pairs, n) / (1 << n) <= tol * (1 + otr)
            gen[dist][M] = ok
    assert gen[w.STATES_HAAR][16] >= 3 and gen[w.STATES_BASIS][16] == 0
    assert gen[w.STATES_HAAR][32] == 4 and gen[w.STATES_BASIS][32] == 4


def test_generalisation_error_against_the_full_cost():
    """With every computational-basis state as the validation set, the
    validation cost is the full cost of Eq. (1) per state, so the normalised
    generalisation error c_val / c_train - 1 follows from Eq. (1) alone."""
    p = w.chain_n3(target_seed=6)
    G = w.initial_gates(4, 1, p.L)[0]
    Pv = w.basis_states(2, p.n, 1 << p.n)
    c_train = 0.25
    want = o.full_cost(p.U, G, p.pairs, p.n) / (1 << p.n) / c_train - 1.0
    got = o.generalisation_error(p.U @ Pv, Pv, G, p.pairs, p.n, c_train)
    assert abs(got - want) < 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("n,pair", [(2, (0, 1)), (2, (1, 0)), (3, (0, 2)), (4, (3, 1)), (5, (2, 4))])
def test_pair_major_view_round_trip_and_row_order(n, pair):
    """pair_major groups a state's rows by the two qubits' bits (row 2*bit_a +
    bit_b, qubit q = bit n-1-q of the row index) and from_pair_major undoes
    it; each entry is checked against that definition directly."""
    M = 3
    rng = np.random.default_rng(n)
    X = rng.standard_normal((1 << n, M)) + 1j * rng.standard_normal((1 << n, M))
    P = o.pair_major(X, n, pair)
    assert P.shape == (4, (1 << n) // 4 * M)
    assert np.array_equal(o.from_pair_major(P, n, pair, M), X)
    a, b = pair
    for r in range(1 << n):
        loc = 2 * ((r >> (n - 1 - a)) & 1) + ((r >> (n - 1 - b)) & 1)
        # the entries of row r land in row loc of the view, in the same sample order
        assert any(np.array_equal(P[loc, k * M:(k + 1) * M], X[r]) for k in range((1 << n) // 4))
