"""Learned warm start for the fixed 6-gate, 4-qubit structure.

The network (WarmStart, kernels in csrc/mlp.cu and csrc/mlp_gemm.cu) maps a
target to six gates.  This module holds the host-side steps around it:

  * training labels come from the method itself: the batched engine runs
    QFactor-Sample on each training target, and the converged gates
    (cost <= tol) become the label after a gauge fix.  The method's
    solutions are only defined up to local unitaries passed along each
    qubit wire between consecutive gates (and phases passed between
    gates); raw converged gates scatter over that orbit and no network
    can regress them.  canonical_gauge picks one point of the orbit, a
    smooth function of the circuit away from a measure-zero set, so the
    labels become a function of the target;
  * a prediction becomes start 0 of a multistart run; the other starts stay
    random (the fallback), and the sweep judges every start as usual, so a
    bad prediction costs one start, never correctness.

The paper has no learned part; this follows the warm-start form named for
the accelerated implementation (target applied to 8 fixed states as input,
three hidden layers of 1024 with GELU, six U(4) gates as output).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import qfs, workloads

N_QUBITS = 4
M_SAMPLES = 8
PAIRS = workloads.LEARNED_PAIRS
L = len(PAIRS)


def gates_to_labels(gates: np.ndarray) -> np.ndarray:
    """(P, 6, 4, 4) complex -> (P, 192) float64 (gate g, entry 4r+c, re/im)."""
    g = np.ascontiguousarray(gates, dtype=np.complex128)
    return g.view(np.float64).reshape(g.shape[0], 2 * 16 * L)


def _polar_unitary(A: np.ndarray) -> np.ndarray:
    u, _s, vh = np.linalg.svd(A)
    return u @ vh


def _dagger(A: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(A, -1, -2))


def _kron2(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Batched A (x) B for (P, 2, 2) operands: A on the first qubit of the pair."""
    return np.einsum("pij,pkl->pikjl", A, B).reshape(A.shape[0], 4, 4)


def canonical_gauge(gates: np.ndarray, pairs=PAIRS) -> np.ndarray:
    """Gauge-fixed copy of circuits gates (P, L, 4, 4) with the same product.

    Gates are visited in circuit order.  Gate k first absorbs the local
    unitaries that earlier gates pushed onto its input wires.  If an output
    wire of gate k feeds a later gate, the local unitary K on that wire is
    chosen so that the leading term A (x) B of the operator-Schmidt
    decomposition of gate k (the SVD of the 4x4 realignment
    R[(i_a j_a), (i_b j_b)] = g[2 i_a + i_b, 2 j_a + j_b]) becomes positive
    semidefinite on that factor: K = polar(A)^dagger; then the gate's phase
    is set so that its trace is real positive.  The inverse of both moves
    travels along the wires to the next gates, and the last gate absorbs
    what remains.  Any gauge transform of the input gives the same output
    (left factors X on a wire change A to X A, and polar(X A) = X polar(A);
    phases are absorbed downstream)."""
    G = np.array(gates, dtype=np.complex128, copy=True)
    P, Lg = G.shape[:2]
    n = 1 + max(max(p) for p in pairs)
    eye = np.broadcast_to(np.eye(2, dtype=np.complex128), (P, 2, 2))
    pending = [eye.copy() for _ in range(n)]
    for k, (a, b) in enumerate(pairs):
        g = G[:, k] @ _kron2(pending[a], pending[b])
        cont_a = any(a in pairs[j] for j in range(k + 1, Lg))
        cont_b = any(b in pairs[j] for j in range(k + 1, Lg))
        if cont_a or cont_b:
            R = g.reshape(P, 2, 2, 2, 2).transpose(0, 1, 3, 2, 4).reshape(P, 4, 4)
            u, _s, vh = np.linalg.svd(R)
            Ka = _dagger(_polar_unitary(u[:, :, 0].reshape(P, 2, 2))) if cont_a else eye
            Kb = _dagger(_polar_unitary(vh[:, 0, :].reshape(P, 2, 2))) if cont_b else eye
            g = _kron2(Ka, Kb) @ g
            ph = np.trace(g, axis1=1, axis2=2)
            ph = ph / np.maximum(np.abs(ph), 1e-300)
            g = g / ph[:, None, None]
            if cont_a:
                pending[a] = _dagger(Ka)
            if cont_b:
                pending[b] = _dagger(Kb)
            w = a if cont_a else b
            pending[w] = pending[w] * ph[:, None, None]
        G[:, k] = g
    return G


def _targets_chunk(args):
    seed, first, count = args
    return workloads.learned_targets(seed, first, count)


def make_targets(seed: int, count: int, chunk: int = 1 << 15, workers: int = 0) -> np.ndarray:
    """Targets (count, 16, 16) of the learned structure, drawn in chunks, in
    a spawn pool of `workers` processes when workers > 1 (the values do not
    depend on the chunking or the pool)."""
    jobs = [(seed, f, min(chunk, count - f)) for f in range(0, count, chunk)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.map(_targets_chunk, jobs)
    else:
        parts = [_targets_chunk(j) for j in jobs]
    return np.concatenate(parts)


def random_starts(seed: int, P: int, S: int) -> np.ndarray:
    """The library's own random starts (P, S, 6, 4, 4): problem i uses seed + i,
    as the batched entry point draws them when it is given no initial gates."""
    out = np.empty((P, S, L, 4, 4), dtype=np.complex128)
    for i in range(P):
        _, out[i] = qfs.generate_inputs(seed + i, N_QUBITS, M_SAMPLES, S, L)
    return out


def instantiate_params(S: int, tol: float = 1e-8, max_sweeps: int = 300, seed: int = 0) -> qfs.Params:
    return qfs.default_params(M=M_SAMPLES, multistarts=S, max_sweeps=max_sweeps, dist_tol=tol,
                              precision=qfs.QFS_MIXED, seed=seed)


@dataclasses.dataclass
class LabelSet:
    targets: np.ndarray      # (P, 16, 16) complex128, converged problems only
    labels: np.ndarray       # (P, 192) float64
    generated: int           # problems run
    sweeps: np.ndarray       # sweeps the method took on the kept problems
    seconds: float           # time in the batched engine


def _canonical_chunk(gates):
    return gates_to_labels(canonical_gauge(gates))


def method_labels(ctx: qfs.Context, targets: np.ndarray, S: int = 4, tol: float = 1e-8,
                  max_sweeps: int = 300, chunk: int = 1 << 16, seed: int = 0, workers: int = 0) -> LabelSet:
    """Run the method (S random starts, drawn by the library from seed +
    index) on every target; keep the converged ones, their gates in the
    canonical gauge as labels.  The gauge fix runs in a spawn pool of
    `workers` processes when workers > 1."""
    params = instantiate_params(S, tol, max_sweeps, seed)
    keep_t, keep_g, keep_s = [], [], []
    secs = 0.0
    for c0 in range(0, len(targets), chunk):
        T = targets[c0:c0 + chunk]
        params.seed = seed + c0
        t0 = time.perf_counter()
        gates, _cost, sweeps, conv, _best = ctx.instantiate_batch_uniform(N_QUBITS, PAIRS, T, params)
        secs += time.perf_counter() - t0
        keep_t.append(T[conv])
        keep_g.append(gates[conv])
        keep_s.append(sweeps[conv])
    if workers > 1 and len(keep_g) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(keep_g))) as pool:
            labels = pool.map(_canonical_chunk, keep_g)
    else:
        labels = [_canonical_chunk(g) for g in keep_g]
    return LabelSet(np.concatenate(keep_t), np.concatenate(labels), len(targets), np.concatenate(keep_s), secs)


@dataclasses.dataclass
class RunStats:
    P: int
    converged: int
    seconds: float             # predict (warm only) + batched instantiation
    predict_seconds: float
    mean_sweeps: float         # over converged problems
    start0_wins: int           # problems whose answer came from start 0

    @property
    def converged_per_s(self) -> float:
        return self.converged / self.seconds


def run_multistart(ctx: qfs.Context, targets: np.ndarray, starts: np.ndarray, params: qfs.Params,
                   ws: "qfs.WarmStart | None" = None) -> RunStats:
    """Instantiate every target with the given starts (P, S, 6, 4, 4); with a
    model, start 0 is replaced by its prediction (inside the timed region)."""
    P = len(targets)
    starts = np.array(starts, dtype=np.complex128, copy=True)
    t0 = time.perf_counter()
    tp = 0.0
    if ws is not None:
        starts[:, 0] = ws.predict(targets)
        tp = time.perf_counter() - t0
    _g, _c, sweeps, conv, best = ctx.instantiate_batch_uniform(N_QUBITS, PAIRS, targets, params, starts)
    secs = time.perf_counter() - t0
    return RunStats(P, int(conv.sum()), secs, tp, float(sweeps[conv].mean()) if conv.any() else float("nan"),
                    int(((best == 0) & conv).sum()))


@dataclasses.dataclass
class PolicyStats:
    name: str
    P: int
    converged: int
    seconds: float
    start_sweeps: int            # sum over problems of starts x sweeps (the sweep work done)
    first_stage_converged: int
    predict_seconds: float = 0.0

    @property
    def converged_per_s(self) -> float:
        return self.converged / self.seconds


def two_stage(ctx: qfs.Context, targets: np.ndarray, first: np.ndarray | None, S_fallback: int = 8,
              first_sweeps: int = 100, max_sweeps: int = 300, tol: float = 1e-8, seed: int = 0,
              ws: "qfs.WarmStart | None" = None, name: str = "") -> PolicyStats:
    """The library's two-stage policy (qfs_ws_instantiate): one start per
    target first (the model's prediction when `first` is None, else the given
    starts (P, 6, 4, 4)), at most first_sweeps sweeps; the targets it leaves
    unconverged fall back to S_fallback random starts drawn by the library.
    Prediction, both stages and all host<->device copies are inside the
    timed region and inside the one call."""
    if ws is None:
        raise ValueError("the policy runs through a WarmStart model's entry point")
    params = instantiate_params(S_fallback, tol, max_sweeps, seed)
    t0 = time.perf_counter()
    _g, r, st = ws.instantiate(targets, params, first_sweeps=first_sweeps, first_gates=first)
    secs = time.perf_counter() - t0
    work = st["first_start_sweeps"] + st["fallback_start_sweeps"]
    return PolicyStats(name, len(targets), int(r["converged"].sum()), secs, work, st["first_converged"], 0.0)


def multistart(ctx: qfs.Context, targets: np.ndarray, S: int = 8, max_sweeps: int = 300, tol: float = 1e-8,
               seed: int = 0, name: str = "") -> PolicyStats:
    """The method without the model: S random starts (drawn by the library)."""
    t0 = time.perf_counter()
    _g, _c, sw, conv, _b = ctx.instantiate_batch_uniform(N_QUBITS, PAIRS, targets,
                                                          instantiate_params(S, tol, max_sweeps, seed))
    secs = time.perf_counter() - t0
    return PolicyStats(name, len(targets), int(conv.sum()), secs, int(sw.sum()) * S, int(conv.sum()))
