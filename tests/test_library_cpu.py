"""CPU checks of the C-ABI library: it builds, loads, exports what include/qfs.h
declares, validates arguments on the host, and draws the same inputs as the
seeded generator.  No kernel runs here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2405_12866_gb300 import build as qbuild
from paper_2405_12866_gb300 import qfs
from paper_2405_12866_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qfs.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qfs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qfs_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    assert sorted(qfs.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_default_params(lib):
    p = qfs.default_params()
    assert (p.M, p.multistarts, p.max_sweeps, p.min_sweeps) == (2, 16, 10000, 6)
    assert p.dist_tol == 1e-8 and p.beta == 0.0 and p.precision == qfs.QFS_FP64
    assert p.restart_doubling == 0 and p.overtrain_ratio == 0.1
    assert p.training_distribution == qfs.QFS_STATES_HAAR and p.concurrent_targets == 0


def _call_instantiate(n, pairs, params, target=None):
    cir = qfs._CircuitArg(n, pairs)
    N = 1 << n
    tgt = np.zeros((N, N), np.complex128) if target is None else target
    out = np.zeros((max(cir.c.L, 1), 4, 4), np.complex128)
    res = qfs.Result()
    code = qfs.lib().qfs_instantiate(None, C.byref(cir.c), tgt.ctypes.data, C.byref(params),
                                     out.ctypes.data, C.byref(res), None)
    return code, qfs.lib().qfs_last_error().decode()


@pytest.mark.parametrize("n,pairs,frag", [
    (1, [(0, 1)], "at least 2 qubits"),
    (15, [(0, 1)], "> 14"),
    (3, [(0, 3)], "out of range"),
    (3, [(1, 1)], "both qubits"),
    (3, [(0, -1)], "out of range"),
])
def test_circuit_validation(lib, n, pairs, frag):
    code, msg = _call_instantiate(n, pairs, qfs.default_params(M=2))
    assert code in (qfs.QFS_EINVAL, qfs.QFS_EUNSUPPORTED)
    assert frag in msg


@pytest.mark.parametrize("kw,frag", [
    (dict(M=0), "M = 0"), (dict(M=9), "M = 9"), (dict(multistarts=0), "multistarts"),
    (dict(max_sweeps=0), "max_sweeps"), (dict(precision=7), "precision"),
    (dict(beta=1.0), "beta"), (dict(beta=-0.1), "beta"), (dict(dist_tol=-1.0), "dist_tol"),
    (dict(training_distribution=2), "training_distribution"),
])
def test_param_validation(lib, kw, frag):
    code, msg = _call_instantiate(3, [(0, 1), (1, 2)], qfs.default_params(**{"M": 4, **kw}))
    assert code == qfs.QFS_EINVAL
    assert frag in msg


def test_null_context_is_rejected(lib):
    code, msg = _call_instantiate(3, [(0, 1)], qfs.default_params(M=4))
    assert code == qfs.QFS_EINVAL and "context" in msg


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    code = lib.qfs_create(C.byref(h), 0, None)
    assert code == qfs.QFS_ECUDA
    assert "device" in lib.qfs_last_error().decode()


@pytest.mark.parametrize("n,M,S,L,seed", [(3, 4, 2, 4, 2), (6, 5, 3, 7, 12345), (8, 16, 1, 28, 2**40 + 3)])
def test_library_draws_match_generator(lib, n, M, S, L, seed):
    samples, gates = qfs.generate_inputs(seed, n, M, S, L)
    assert np.allclose(samples, w.sample_states(seed, n, M), atol=1e-12)
    assert np.allclose(gates, w.initial_gates(seed, S, L), atol=1e-12)
    assert np.allclose(samples.conj().T @ samples, np.eye(M), atol=1e-13)


@pytest.mark.parametrize("n,M,seed,stream", [(2, 4, 0, 1), (3, 5, 9, 5), (6, 17, 2**40 + 3, 1), (10, 64, 31, 5)])
def test_library_state_draws_match_generator(lib, n, M, seed, stream):
    """Both training distributions (Appendix D): the library's draw equals
    the seeded generator's, bit for bit."""
    haar = qfs.generate_states(seed, qfs.QFS_STATES_HAAR, stream, n, M)
    assert np.allclose(haar, w.sample_states(seed, n, M, stream), atol=1e-12)
    basis = qfs.generate_states(seed, qfs.QFS_STATES_BASIS, stream, n, M)
    assert np.array_equal(basis, w.basis_states(seed, n, M, stream))


def test_state_draw_validation(lib):
    out = np.zeros((8, 2), np.complex128)
    for args, frag in [((0, 2, 1, 3, 2), "distribution"), ((0, 1, 1, 3, 9), "M = 9"), ((0, 1, 1, 1, 1), "n = 1")]:
        assert lib.qfs_generate_states(*args, out.ctypes.data) == qfs.QFS_EINVAL
        assert frag in lib.qfs_last_error().decode()


@pytest.mark.parametrize("T,kw,code,frag", [
    (0, {}, "EINVAL", "T = 0"),
    (2, dict(concurrent_targets=-1), "EINVAL", "concurrent_targets"),
    (2, dict(restart_doubling=1), "EUNSUPPORTED", "one target per call"),
])
def test_many_targets_validation(lib, T, kw, code, frag):
    """qfs_instantiate_many checks its arguments on the host, before any
    device work (no context is needed to reach these errors)."""
    n, pairs = 3, [(0, 1), (1, 2)]
    cir = qfs._CircuitArg(n, pairs)
    prm = qfs.default_params(M=4, multistarts=2, **kw)
    tg = np.zeros((max(T, 1), 8, 8), np.complex128)
    out = np.zeros((max(T, 1), 2, 4, 4), np.complex128)
    res = (qfs.Result * max(T, 1))()
    rc = lib.qfs_instantiate_many(None, C.byref(cir.c), T, tg.ctypes.data, None, None, C.byref(prm),
                                  out.ctypes.data, res, None)
    assert rc == getattr(qfs, "QFS_" + code)
    assert frag in lib.qfs_last_error().decode()
