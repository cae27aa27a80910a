"""Host-side pieces of the learned warm start: the gauge fix that turns the
method's converged gates into regression labels, the label layout and the
target generator of the learned structure."""
import numpy as np
import pytest

from paper_2405_12866_gb300 import learned
from paper_2405_12866_gb300 import workloads as w


def _haar2(rng, P):
    z = rng.normal(size=(P, 2, 2)) + 1j * rng.normal(size=(P, 2, 2))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    return q * (d / np.abs(d))[:, None, :] * np.exp(1j * rng.uniform(0, 2 * np.pi, size=(P, 1, 1)))


def _on_wire(X, wire, pair):
    """X (P, 2, 2) acting on `wire` of the 2-qubit pair, as (P, 4, 4)."""
    I = np.broadcast_to(np.eye(2), X.shape)
    if wire == pair[0]:
        return np.einsum("pij,pkl->pikjl", X, I).reshape(-1, 4, 4)
    return np.einsum("pij,pkl->pikjl", I, X).reshape(-1, 4, 4)


def _random_gauge(g, seed):
    """Insert X X^dagger on every wire segment between two gates."""
    rng = np.random.default_rng(seed)
    g = g.copy()
    pairs = learned.PAIRS
    for k, pk in enumerate(pairs):
        for wire in pk:
            nk = next((j for j in range(k + 1, len(pairs)) if wire in pairs[j]), None)
            if nk is None:
                continue
            X = _haar2(rng, g.shape[0])
            g[:, k] = _on_wire(X, wire, pk) @ g[:, k]
            g[:, nk] = g[:, nk] @ _on_wire(np.conj(np.swapaxes(X, 1, 2)), wire, pairs[nk])
    return g


def test_learned_targets_match_the_gate_by_gate_product():
    U = learned.make_targets(3, 5)
    gs = w.haar_gates(3, w.STREAM_TARGET_GATES, 30).reshape(5, 6, 4, 4)
    for i in range(5):
        assert np.max(np.abs(U[i] - w.target_unitary(gs[i], learned.PAIRS, 4))) < 1e-14
    # chunking and the first-problem offset do not change the draws
    assert np.max(np.abs(learned.make_targets(3, 5, chunk=2) - U)) == 0.0
    assert np.max(np.abs(w.learned_targets(3, 2, 3) - U[2:])) == 0.0


def test_canonical_gauge_keeps_the_circuit():
    g = w.haar_gates(5, w.STREAM_TARGET_GATES, 6 * 40).reshape(40, 6, 4, 4)
    c = learned.canonical_gauge(g)
    U = w.target_unitaries(g, learned.PAIRS, 4)
    assert np.max(np.abs(w.target_unitaries(c, learned.PAIRS, 4) - U)) < 1e-13
    eye = np.eye(4)
    assert np.max(np.abs(np.einsum("pkij,pkil->pkjl", c.conj(), c) - eye)) < 1e-13
    # gates with a wire that feeds a later gate have a real positive trace
    tr = np.trace(c[:, :5], axis1=2, axis2=3)
    assert np.all(np.abs(tr.imag) < 1e-12) and np.all(tr.real > 0)


def test_canonical_gauge_is_gauge_invariant_and_idempotent():
    g = w.haar_gates(6, w.STREAM_TARGET_GATES, 6 * 40).reshape(40, 6, 4, 4)
    c = learned.canonical_gauge(g)
    moved = _random_gauge(g, 1)
    assert np.max(np.abs(moved - g)) > 0.5
    assert np.max(np.abs(learned.canonical_gauge(moved) - c)) < 1e-10
    assert np.max(np.abs(learned.canonical_gauge(c) - c)) < 1e-10


def test_converged_solutions_from_different_starts_share_the_label():
    """The labels are a function of the target: two runs of the method from
    different random starts converge to gates with one canonical form."""
    from oracle import qfs_oracle as O
    g = w.haar_gates(8, w.STREAM_TARGET_GATES, 6 * 4).reshape(4, 6, 4, 4)
    U = w.target_unitaries(g, learned.PAIRS, 4)
    want = learned.canonical_gauge(g)
    Psi = w.sample_states(2, 4, 8)
    checked = 0
    for i in range(4):
        for s in range(3):
            init = w.initial_gates(500 + 7 * i + s, 1, 6)
            r = O.instantiate(U[i], Psi, init, learned.PAIRS, 4, 1e-13, 600)
            if not r.converged:
                continue
            got = learned.canonical_gauge(r.gates[None])[0]
            assert np.max(np.abs(got - want[i])) < 1e-4
            checked += 1
    assert checked >= 6


def test_label_layout():
    g = w.haar_gates(9, w.STREAM_TARGET_GATES, 12).reshape(2, 6, 4, 4)
    lab = learned.gates_to_labels(g)
    assert lab.shape == (2, 192)
    for t in range(2):
        for k in range(6):
            for r in range(4):
                for c in range(4):
                    assert lab[t, 32 * k + 2 * (4 * r + c)] == g[t, k, r, c].real
                    assert lab[t, 32 * k + 2 * (4 * r + c) + 1] == g[t, k, r, c].imag
