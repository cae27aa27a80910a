"""CPU FP64 oracle for QFactor-Sample (arXiv 2405.12866). TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may use this module.  The product path (the CUDA library and its binding)
never imports it, and this module imports nothing from the product.

It restates the method step by step, in float64 numpy, in the paper's order
and notation:

  * Instantiation problem and full cost, Section 2.1, Eq. (1).
  * Training set {(psi_j, U psi_j)} and the sample cost, Section 2.3 and
    Section 3, Eq. (qfactor_sample_cost_function).
  * The sweep: right to left, at each gate the environment E, its SVD
    E = X D Y^dagger and the update u = Y X^dagger, Section 2.1 Eq. (2) and
    Section 3; the objective Re Tr(E u_i) of the gate being updated, Section 3.
  * The A tensor (<psi_j| U^dagger, kept here as Phi_L = U Psi) and the list B
    of intermediate states C_{<=k} Psi, Section 3 and Fig. (pre-comp).
  * The damped update on (1 - beta) E + beta u^dagger, Appendix A.
  * Plateau detection |c_{i-1}| - |c_i| > diff_tol_r |c_i|, Appendix A.
  * Validation cost and normalised generalisation error c_val / c_train - 1
    with double-and-restart of M up to 2^n, Section 3 and Appendix A.

Readings where the paper is silent (each one is a choice, not the paper's):
  * Qubit q is bit (n-1-q) of a row index; a gate on (a, b) uses the local
    index 2*bit_a + bit_b; the gate listed first acts first on the state.
  * E[x][y] = sum over the untouched index r and samples j of
    B[(x, r), j] * conj(Phi[(y, r), j]), so that Re Tr(u E) is the objective.
  * One sweep = rebuild B_1..B_{L-1} with the current gates, then update
    gates L, L-1, ..., 1; the cost is evaluated once per sweep after gate 1
    from its environment: c = 2 - (2/M) Re Tr(u_1 E_1).
  * Multistarts run in lock step; the run stops at the first sweep s* at
    which some start has c <= tol and returns the start with the smallest
    cost at s* (lowest index on ties); if none converges, the start with the
    smallest final cost.
  * An ill-conditioned SVD has no unique update; numpy's SVD picks one.

Library routines used as steps: numpy matmul, numpy.linalg.svd.
"""
from __future__ import annotations

import dataclasses
import numpy as np


# ------------------------------------------------------------ state algebra

def pair_major(state: np.ndarray, n: int, pair) -> np.ndarray:
    """View an N x M state as 4 x (N/4 * M): row = local index 2*bit_a+bit_b."""
    a, b = pair
    M = state.shape[1]
    T = state.reshape((2,) * n + (M,))
    T = np.moveaxis(T, (a, b), (0, 1))
    return T.reshape(4, -1)


def from_pair_major(P: np.ndarray, n: int, pair, M: int) -> np.ndarray:
    a, b = pair
    T = P.reshape((2, 2) + (2,) * (n - 2) + (M,))
    T = np.moveaxis(T, (0, 1), (a, b))
    return np.ascontiguousarray(T).reshape(1 << n, M)


def apply_gate(state: np.ndarray, gate: np.ndarray, pair, n: int) -> np.ndarray:
    """(gate tensor identity) applied to every sample of the state."""
    M = state.shape[1]
    return from_pair_major(gate @ pair_major(state, n, pair), n, pair, M)


def circuit_apply(state: np.ndarray, gates, pairs, n: int) -> np.ndarray:
    """C Psi with C = g_L ... g_1 (the first listed gate acts first)."""
    X = state
    for g, p in zip(gates, pairs):
        X = apply_gate(X, g, p, n)
    return X


def circuit_unitary(gates, pairs, n: int) -> np.ndarray:
    return circuit_apply(np.eye(1 << n, dtype=np.complex128), gates, pairs, n)


# --------------------------------------------------------------- cost forms

def full_cost(U: np.ndarray, gates, pairs, n: int) -> float:
    """Eq. (1): ||U - C||_F^2 = 2^(n+1) (1 - Re Tr(U^dagger C) / 2^n)."""
    C = circuit_unitary(gates, pairs, n)
    N = 1 << n
    return float(2 * N * (1.0 - np.real(np.trace(U.conj().T @ C)) / N))


def sample_cost(UPsi: np.ndarray, Psi: np.ndarray, gates, pairs, n: int) -> float:
    """Sample cost, residual form: (1/M) sum_j ||U psi_j - C psi_j||^2."""
    M = Psi.shape[1]
    R = UPsi - circuit_apply(Psi, gates, pairs, n)
    return float(np.sum(np.abs(R) ** 2) / M)


def sample_cost_trace(UPsi: np.ndarray, Psi: np.ndarray, gates, pairs, n: int) -> float:
    """Sample cost, trace form: 2 - (2/M) Re sum_j <psi_j| U^dagger C |psi_j>."""
    M = Psi.shape[1]
    CPsi = circuit_apply(Psi, gates, pairs, n)
    return float(2.0 - 2.0 / M * np.real(np.vdot(UPsi, CPsi)))


# ----------------------------------------------------------- the local step

def environment(B_prev: np.ndarray, Phi: np.ndarray, pair, n: int) -> np.ndarray:
    """E[x][y] = sum_{r,j} B_{k-1}[(x,r),j] conj(Phi^(k)[(y,r),j]) (4x4).

    With Phi^(k) = g_{k+1}^dagger ... g_L^dagger U Psi this gives
    Re Tr(g_k E) = Re sum_j <psi_j| U^dagger C |psi_j>, the quantity the
    gate update maximises (Section 3)."""
    return pair_major(B_prev, n, pair) @ pair_major(Phi, n, pair).conj().T


def gate_update(E: np.ndarray, g_old: np.ndarray | None = None, beta: float = 0.0) -> np.ndarray:
    """Eq. (2): SVD E = X D Y^dagger, u_new = Y X^dagger.  With beta > 0 the
    SVD is taken of (1 - beta) E + beta g_old^dagger (Appendix A)."""
    if beta != 0.0:
        E = (1.0 - beta) * E + beta * g_old.conj().T
    X, D, Yh = np.linalg.svd(E)
    return Yh.conj().T @ X.conj().T


# ------------------------------------------------------------------- sweeps

@dataclasses.dataclass
class SweepResult:
    gates: np.ndarray          # (L, 4, 4) gates after the sweep
    envs: np.ndarray           # (L, 4, 4) environment of each gate as used
    objective: np.ndarray      # (L,) Re Tr(g_k,new E_k) after each update
    cost: float                # 2 - (2/M) Re Tr(g_1 E_1)


def sweep(UPsi: np.ndarray, Psi: np.ndarray, gates: np.ndarray, pairs, n: int,
          beta: float = 0.0) -> SweepResult:
    """One right-to-left sweep (Section 3, Fig. pre-comp and env_calc_tensor).

    B_0 = Psi and B_k = g_k B_{k-1} for k < L are built with the gates of the
    previous sweep; then for k = L..1 the environment of gate k is formed from
    B_{k-1} and Phi^(k), gate k is replaced, and Phi^(k-1) = g_k^dagger Phi^(k)
    carries the updated gate towards the input side."""
    L = len(pairs)
    M = Psi.shape[1]
    B = [Psi]
    for k in range(1, L):
        B.append(apply_gate(B[k - 1], gates[k - 1], pairs[k - 1], n))
    new = np.array(gates, dtype=np.complex128, copy=True)
    envs = np.zeros((L, 4, 4), dtype=np.complex128)
    obj = np.zeros(L)
    Phi = UPsi
    for k in range(L, 0, -1):
        E = environment(B[k - 1], Phi, pairs[k - 1], n)
        g = gate_update(E, new[k - 1], beta)
        envs[k - 1] = E
        new[k - 1] = g
        obj[k - 1] = np.real(np.trace(g @ E))
        if k > 1:
            Phi = apply_gate(Phi, g.conj().T, pairs[k - 1], n)
    cost = float(2.0 - 2.0 / M * obj[0])
    return SweepResult(new, envs, obj, cost)


@dataclasses.dataclass
class InstantiateResult:
    gates: np.ndarray          # (L, 4, 4) of the selected start
    cost: float
    sweeps: int
    converged: bool
    best_start: int
    start_costs: np.ndarray    # (S,) cost of every start after the last sweep
    all_gates: np.ndarray      # (S, L, 4, 4) every start's gates at the end
    cost_trace: np.ndarray     # (sweeps, S)


def instantiate(U: np.ndarray | None, Psi: np.ndarray, init_gates: np.ndarray, pairs,
                n: int, tol: float, max_sweeps: int, beta: float = 0.0,
                UPsi: np.ndarray | None = None, min_sweeps: int = 0,
                plateau_window: int = 0, diff_tol_r: float = 0.0) -> InstantiateResult:
    """Multistart QFactor-Sample with fixed M.

    Stops at the first sweep at which some start has cost <= tol (Appendix A,
    dist_tol) or after max_sweeps (max_iter).  With plateau_window > 0 a start
    stops once, over plateau_window consecutive sweeps, the cost never
    improved by diff_tol_r relative to the newer cost (Appendix A) and at
    least min_sweeps sweeps ran; the run ends when every start stopped."""
    if UPsi is None:
        UPsi = U @ Psi
    G = np.array(init_gates, dtype=np.complex128, copy=True)
    S = G.shape[0]
    costs = np.full(S, np.inf)
    active = np.ones(S, dtype=bool)
    stall = np.zeros(S, dtype=int)
    trace = []
    s = 0
    while s < max_sweeps:
        s += 1
        for i in range(S):
            if not active[i]:
                continue
            r = sweep(UPsi, Psi, G[i], pairs, n, beta)
            prev = costs[i]
            G[i] = r.gates
            costs[i] = r.cost
            if plateau_window > 0 and np.isfinite(prev):
                improved = abs(prev) - abs(r.cost) > diff_tol_r * abs(r.cost)
                stall[i] = 0 if improved else stall[i] + 1
                if stall[i] >= plateau_window and s >= min_sweeps:
                    active[i] = False
        trace.append(costs.copy())
        if np.any(costs <= tol) or not np.any(active):
            break
    best = int(np.argmin(costs))      # argmin returns the lowest index on ties
    return InstantiateResult(G[best].copy(), float(costs[best]), s,
                             bool(costs[best] <= tol), best, costs.copy(), G,
                             np.array(trace))


# ------------------------------------------- generalisation check (Sec. 3)

def generalisation_error(UPsi_val: np.ndarray, Psi_val: np.ndarray, gates, pairs,
                         n: int, c_train: float) -> float:
    """Normalised generalisation error c_val / c_train - 1 (Section 3)."""
    c_val = sample_cost(UPsi_val, Psi_val, gates, pairs, n)
    return c_val / c_train - 1.0


# ------------------------------------------- double-and-restart (Sec. 3, App. A)

@dataclasses.dataclass
class RestartResult:
    gates: np.ndarray          # (L, 4, 4) of the returned start
    cost: float                # its training cost
    validation_cost: float     # its validation cost (NaN when M reached 2^n)
    converged: bool
    best_start: int
    training_states: int       # M of the last attempt
    attempts: int
    sweeps: int                # over all attempts


def instantiate_restarting(U: np.ndarray, training_states, validation_states, init_gates: np.ndarray,
                           pairs, n: int, tol: float, max_sweeps: int, M0: int,
                           overtrain_ratio: float, min_sweeps: int = 0) -> RestartResult:
    """QFactor-Sample with the on-the-fly generalisation check (Sec. 3 and
    Appendix A): multistart sweeps on M training states; after every sweep
    (from min_sweeps on) the start with the lowest training cost c_train is
    evaluated on M validation states (c_val).  When c_val / c_train - 1 >
    overtrain_ratio the attempt halts, M doubles (up to 2^n), new training and
    validation states are drawn, every start keeps its gates, and the run
    restarts.  Success needs c_train <= tol and c_val <= (1 + overtrain_ratio)
    c_train; at M = 2^n the check is skipped.  max_sweeps bounds each attempt.

    training_states(M, attempt) and validation_states(M, attempt) return
    the N x M states of an attempt."""
    N = 1 << n
    G = np.array(init_gates, dtype=np.complex128, copy=True)
    S = G.shape[0]
    M, attempt, total = M0, 0, 0
    while True:
        Psi = training_states(M, attempt)
        UPsi = U @ Psi
        check = M < N
        if check:
            Psi_v = validation_states(M, attempt)
            UPsi_v = U @ Psi_v
        costs = np.full(S, np.inf)
        overtrained, done, cv = False, False, float("nan")
        s = 0
        while s < max_sweeps and not done:
            s += 1
            for i in range(S):
                r = sweep(UPsi, Psi, G[i], pairs, n)
                G[i] = r.gates
                costs[i] = r.cost
            b = int(np.argmin(costs))
            converged_now = costs[b] <= tol
            if check and s >= min_sweeps:
                cv = sample_cost(UPsi_v, Psi_v, G[b], pairs, n)
                if cv / costs[b] - 1.0 > overtrain_ratio:
                    overtrained, done = True, True
            if converged_now:
                done = True
        total += s
        b = int(np.argmin(costs))
        if check and not overtrained:
            cv = sample_cost(UPsi_v, Psi_v, G[b], pairs, n)
        if overtrained and 2 * M <= N:
            M, attempt = 2 * M, attempt + 1
            continue
        conv = bool(costs[b] <= tol and not overtrained)
        return RestartResult(G[b].copy(), float(costs[b]), float(cv) if check else float("nan"), conv, b, M,
                             attempt + 1, total)
