"""Seeded synthetic inputs for QFactor-Sample instantiation problems.

This module draws random numbers and shapes them into problem inputs; it
holds none of the sweep's arithmetic (no environments, no gate updates, no
cost).  Both the CPU oracle's tests and the CUDA path's tests and benchmark
take their inputs from here, so neither side generates inputs for the other.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), a counter-based generator, so a
value depends only on (seed, stream, index).  The C library carries its own
implementation of the same published generator for its seed-driven entry
point; a CPU test checks that both produce the same sample states.

Conventions (shared by every part of this project):
  * n qubits, N = 2**n; qubit q is bit (n-1-q) of a row index (qubit 0 is the
    most significant bit).
  * A 2-qubit gate on the ordered pair (a, b) is a 4x4 unitary indexed by
    the local index 2*bit_a + bit_b.
  * A circuit is a list of pairs applied in list order: the first listed
    gate acts first on the state, so C = g_L ... g_2 g_1.
  * States are N x M complex matrices, row-major, sample index fastest.

The training states are the columns of a Haar-random unitary, as the paper's
appendix on implementation details describes; here they are the Q factor of
a complex Gaussian N x M matrix with a positive real R diagonal, which has
the same distribution (Mezzadri, "How to generate random matrices from the
classical compact groups", Notices AMS 2007).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Philox4x32-10 constants (Salmon et al. 2011, Section 5).
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# Stream identifiers (third counter word).  The C library uses the same
# numbers for the two draws the method itself makes (samples, initial gates).
STREAM_SAMPLES = 1
STREAM_INIT_GATES = 2
STREAM_TARGET_GATES = 3
STREAM_STRUCTURE = 4
STREAM_VALIDATION = 5


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 block function on a (K, 4) uint32 counter array."""
    ctr = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
    c0, c1, c2, c3 = (ctr[:, i].astype(np.uint64) for i in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _PHILOX_W0) & _MASK32
        k1 = (k1 + _PHILOX_W1) & _MASK32
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def _blocks(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    key = (seed & 0xFFFFFFFF, seed >> 32)
    out = np.empty((count, 4), dtype=np.uint32)
    step = 1 << 15   # cache-sized pieces; the values do not depend on it
    for c0 in range(0, count, step):
        c1 = min(count, c0 + step)
        idx = np.arange(first + c0, first + c1, dtype=np.uint64)
        ctr = np.zeros((c1 - c0, 4), dtype=np.uint32)
        ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
        ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
        ctr[:, 2] = np.uint32(stream)
        out[c0:c1] = philox4x32_10(ctr, key)
    return out


def _u53(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """Uniform double in (0, 1) from two 32-bit words (53 random bits)."""
    a = (hi >> np.uint32(5)).astype(np.float64)
    b = (lo >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def complex_normals(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    """Standard complex normals (E|z|^2 = 1); element i uses counter first+i.

    One Philox block -> two uniforms -> one Box-Muller pair -> (re, im).
    """
    x = _blocks(seed, stream, first, count)
    u1 = _u53(x[:, 0], x[:, 1])
    u2 = _u53(x[:, 2], x[:, 3])
    r = np.sqrt(-2.0 * np.log(u1)) * np.sqrt(0.5)
    t = 2.0 * np.pi * u2
    return r * np.cos(t) + 1j * (r * np.sin(t))


def uniform_ints(seed: int, stream: int, first: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) from word 0 of each block."""
    x = _blocks(seed, stream, first, count)[:, 0].astype(np.uint64)
    span = np.uint64(hi - lo + 1)
    return (lo + (x * span >> np.uint64(32))).astype(np.int64)


def positive_qr_q(g: np.ndarray) -> np.ndarray:
    """Q factor of g = QR with R's diagonal made real positive (unique)."""
    q, r = np.linalg.qr(g)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def sample_states(seed: int, n: int, M: int, stream: int = STREAM_SAMPLES) -> np.ndarray:
    """M orthonormal sample states as an N x M complex128 matrix."""
    N = 1 << n
    if not (1 <= M <= N):
        raise ValueError(f"need 1 <= M <= 2^n, got M={M}, n={n}")
    g = complex_normals(seed, stream, 0, N * M).reshape(N, M)
    return positive_qr_q(g)


def basis_indices(seed: int, n: int, M: int, stream: int = STREAM_SAMPLES) -> np.ndarray:
    """M distinct computational-basis indices, uniform without replacement:
    a partial Fisher-Yates shuffle of 0..N-1 in which step j swaps position
    j with position j + floor(w_j (N - j) / 2^32), w_j = word 0 of Philox
    block j of (seed, stream)."""
    N = 1 << n
    if not (1 <= M <= N):
        raise ValueError(f"need 1 <= M <= 2^n, got M={M}, n={n}")
    w = _blocks(seed, stream, 0, M)[:, 0].astype(np.uint64)
    perm = np.arange(N, dtype=np.int64)
    for j in range(M):
        r = j + int((w[j] * np.uint64(N - j)) >> np.uint64(32))
        perm[j], perm[r] = perm[r], perm[j]
    return perm[:M].copy()


def basis_states(seed: int, n: int, M: int, stream: int = STREAM_SAMPLES) -> np.ndarray:
    """M distinct computational-basis states (columns e_i, i from
    basis_indices) as an N x M complex128 matrix: the alternative training
    distribution of the paper's Appendix D."""
    idx = basis_indices(seed, n, M, stream)
    out = np.zeros((1 << n, M), dtype=np.complex128)
    out[idx, np.arange(M)] = 1.0
    return out


STATES_HAAR = 0
STATES_BASIS = 1


def training_states(kind: int, seed: int, n: int, M: int, stream: int = STREAM_SAMPLES) -> np.ndarray:
    """States of either distribution (STATES_HAAR or STATES_BASIS)."""
    if kind == STATES_HAAR:
        return sample_states(seed, n, M, stream)
    if kind == STATES_BASIS:
        return basis_states(seed, n, M, stream)
    raise ValueError(f"unknown state distribution {kind}")


def attempt_seed(seed: int, attempt: int) -> int:
    """Seed of the training and validation states of a double-and-restart
    attempt (attempt 0 uses the run seed itself)."""
    if attempt == 0:
        return int(seed) & 0xFFFFFFFFFFFFFFFF
    return (int(seed) ^ (attempt * 0x9E3779B97F4A7C15)) & 0xFFFFFFFFFFFFFFFF


def haar_gates(seed: int, stream: int, count: int, first_gate: int = 0) -> np.ndarray:
    """`count` Haar-random U(4) matrices, gate i drawn from counters 16*i..16*i+15."""
    z = complex_normals(seed, stream, 16 * first_gate, 16 * count).reshape(count, 4, 4)
    return np.stack([positive_qr_q(z[i]) for i in range(count)])


def initial_gates(seed: int, S: int, L: int) -> np.ndarray:
    """Haar-random initial gates for S multistarts, shape (S, L, 4, 4)."""
    return haar_gates(seed, STREAM_INIT_GATES, S * L).reshape(S, L, 4, 4)


# ---------------------------------------------------------------- structures

def chain_pairs(n: int, L: int) -> list[tuple[int, int]]:
    """Linear chain: (0,1), (1,2), ..., wrapping back to (0,1)."""
    return [(k % (n - 1), k % (n - 1) + 1) for k in range(L)]


def brick_pairs(n: int, half_layers: int) -> list[tuple[int, int]]:
    """Brick wall of nearest-neighbour pairs: even half-layers (0,1),(2,3),...
    alternate with odd half-layers (1,2),(3,4),...; n=8 with 8 half-layers is
    28 gates and n=12 with 3 half-layers is 17 gates."""
    pairs = []
    for h in range(half_layers):
        start = h % 2
        pairs += [(q, q + 1) for q in range(start, n - 1, 2)]
    return pairs


LEARNED_PAIRS = [(0, 1), (2, 3), (1, 2), (0, 1), (2, 3), (1, 2)]


# ------------------------------------------------------------ target unitary

def embed_apply(gate: np.ndarray, pair, n: int, X: np.ndarray) -> np.ndarray:
    """(gate on `pair`, identity elsewhere) times X, X of shape (N, K).

    This forms the target as the stated product of embedded gates; it is the
    definition of the synthetic input, written here so that the benchmark and
    tests never ask the CUDA path or the oracle for their own inputs.
    """
    a, b = pair
    K = X.shape[1]
    T = X.reshape((2,) * n + (K,))
    T = np.moveaxis(T, (a, b), (0, 1))
    shp = T.shape
    T = (gate @ T.reshape(4, -1)).reshape(shp)
    return np.ascontiguousarray(np.moveaxis(T, (0, 1), (a, b))).reshape(1 << n, K)


def target_unitaries(gates: np.ndarray, pairs, n: int) -> np.ndarray:
    """Stack of targets for gates of shape (B, L, 4, 4): (B, N, N), each the
    product of its embedded gates (the vectorised form of target_unitary)."""
    B = gates.shape[0]
    N = 1 << n
    U = np.broadcast_to(np.eye(N, dtype=np.complex128), (B, N, N)).copy()
    for k, (a, b) in enumerate(pairs):
        T = U.reshape((B,) + (2,) * n + (N,))
        T = np.moveaxis(T, (1 + a, 1 + b), (1, 2))
        shp = T.shape
        T = np.matmul(gates[:, k], T.reshape(B, 4, -1)).reshape(shp)
        U = np.ascontiguousarray(np.moveaxis(T, (1, 2), (1 + a, 1 + b))).reshape(B, N, N)
    return U


def haar_gates_batched(seed: int, stream: int, count: int, first_gate: int = 0) -> np.ndarray:
    """Same draws as haar_gates (gate i from counters 16 i .. 16 i + 15), QR batched."""
    z = complex_normals(seed, stream, 16 * first_gate, 16 * count).reshape(count, 4, 4)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    return q * (d / np.abs(d))[:, None, :]


def target_unitary(gates: np.ndarray, pairs, n: int) -> np.ndarray:
    """U = g_L ... g_1 as a dense N x N complex128 matrix."""
    U = np.eye(1 << n, dtype=np.complex128)
    for g, p in zip(gates, pairs):
        U = embed_apply(g, p, n, U)
    return U


# ------------------------------------------------------------------ problems

@dataclasses.dataclass
class Problem:
    """One instantiation problem: structure, target and the run's draws."""
    name: str
    n: int
    pairs: list
    target_gates: np.ndarray      # (L, 4, 4) gates the target was built from
    U: np.ndarray                 # (N, N) complex128 target unitary
    M: int
    S: int
    seed: int                     # seed for samples and initial gates
    tol: float
    max_sweeps: int

    @property
    def N(self) -> int:
        return 1 << self.n

    @property
    def L(self) -> int:
        return len(self.pairs)

    def samples(self) -> np.ndarray:
        return sample_states(self.seed, self.n, self.M)

    def init_gates(self) -> np.ndarray:
        return initial_gates(self.seed, self.S, self.L)


def make_problem(name, n, pairs, M, S, target_seed, run_seed, tol, max_sweeps,
                 build_target=True) -> Problem:
    tg = haar_gates(target_seed, STREAM_TARGET_GATES, len(pairs))
    U = target_unitary(tg, pairs, n) if build_target else None
    return Problem(name, n, list(pairs), tg, U, M, S, run_seed, tol, max_sweeps)


def chain_n3(target_seed: int = 1, run_seed: int = 2) -> Problem:
    """n=3 chain of 4 gates (0,1),(1,2),(0,1),(1,2); M=4; 1 start; tol 1e-10."""
    return make_problem("chain_n3_L4_M4_S1", 3, chain_pairs(3, 4), 4, 1,
                        target_seed, run_seed, 1e-10, 200)


def brick_n8(target_seed: int = 0, run_seed: int = 100, S: int = 16) -> Problem:
    """n=8 brick wall of 28 gates; M=16; 16 starts; tol 1e-8; 500 sweeps."""
    return make_problem("brick_n8_L28_M16_S16", 8, brick_pairs(8, 8), 16, S,
                        target_seed, run_seed, 1e-8, 500)


def brick_n12(target_seed: int = 0, run_seed: int = 200, S: int = 32,
              build_target: bool = True) -> Problem:
    """n=12 brick wall of 17 gates; M=32; 32 starts; tol 1e-8."""
    return make_problem("brick_n12_L17_M32_S32", 12, brick_pairs(12, 3), 32, S,
                        target_seed, run_seed, 1e-8, 500, build_target)


def uneven_blocks(P: int = 4096, seed: int = 4, S: int = 8, max_sweeps: int = 500):
    """P problems with n uniform in {3,4,5}, L uniform in {2..10} gates on
    nearest-neighbour pairs (i, i+1), i uniform in {0..n-2}; M = 2^(n-1)."""
    probs = []
    for p in range(P):
        draws = uniform_ints(seed, STREAM_STRUCTURE, 64 * p, 1, 3, 5)
        n = int(draws[0])
        L = int(uniform_ints(seed, STREAM_STRUCTURE, 64 * p + 1, 1, 2, 10)[0])
        qs = uniform_ints(seed, STREAM_STRUCTURE, 64 * p + 2, L, 0, n - 2)
        pairs = [(int(q), int(q) + 1) for q in qs]
        tseed = (seed << 20) + p
        probs.append(make_problem(f"uneven_{p}", n, pairs, 1 << (n - 1), S,
                                  tseed, tseed + (1 << 40), 1e-8, max_sweeps))
    return probs


# ------------------------------------------------------------ learned form

def learned_targets(seed: int, first: int, count: int) -> np.ndarray:
    """Targets (count, 16, 16) of problems first .. first+count-1: each the
    product of 6 Haar U(4) gates on LEARNED_PAIRS (4 qubits)."""
    L = len(LEARNED_PAIRS)
    g = haar_gates_batched(seed, STREAM_TARGET_GATES, count * L, first * L).reshape(count, L, 4, 4)
    return target_unitaries(g, LEARNED_PAIRS, 4)
