"""The allocation-free sweep entry point against the regular one.

qfs_sweep_once_noalloc serves callers that cannot call cudaMalloc (a host
framework that owns all device memory, or code that must not trigger the
device-wide synchronisation an allocation can cause).  Its scratch is a
static device array shared by every call, so this test calls it twice in a
row with different problems and checks each result against
qfs_sweep_once, to the FP64 sweep tolerances used elsewhere (1e-10 on gates
and environments, 1e-12 on the cost).  A third call runs a problem large
enough that its launches need more partial-sum slots per start than a
shape for all starts would give.  The file name makes pytest collect
it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2405_12866_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _problem(n, pairs, M, S, seed):
    tg = w.haar_gates(seed, w.STREAM_TARGET_GATES, len(pairs))
    U = w.target_unitary(tg, pairs, n)
    return U, w.sample_states(seed + 1, n, M), w.initial_gates(seed + 2, S, len(pairs))


def test_noalloc_sweep_matches_regular_sweep_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import build, qfs
    build.build()
    lib = qfs.lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    # The third case (8.5 MiB of scratch) is one where the backward launches,
    # shaped for a quarter of the starts, use more blocks per start than a
    # shape for all S starts would: its partial sums must still fit.
    cases = [(6, w.brick_pairs(6, 3), 16, 3, 501), (5, [(0, 1), (3, 4), (2, 1), (4, 0)], 5, 4, 502),
             (10, [(0, 1), (2, 3)], 32, 8, 503)]
    with qfs.Context(0) as ctx:
        for n, pairs, M, S, seed in cases:
            U, Psi, G = _problem(n, pairs, M, S, seed)
            L = len(pairs)
            g_ref, e_ref, c_ref = ctx.sweep_once(n, pairs, U, Psi, G, qfs.QFS_FP64)

            tU = torch.from_numpy(U).to(dev)
            tPsi = torch.from_numpy(Psi).to(dev)
            tG = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
            tOut = torch.full((S, L, 4, 4), np.nan, dtype=torch.complex128, device=dev)
            tCost = torch.full((S,), np.nan, dtype=torch.float64, device=dev)
            tEnv = torch.full((S, L, 4, 4), np.nan, dtype=torch.complex128, device=dev)
            cir = qfs._CircuitArg(n, pairs)
            code = lib.qfs_sweep_once_noalloc(stream.cuda_stream, C.byref(cir.c), tU.data_ptr(),
                                              tPsi.data_ptr(), M, S, 0.0, tG.data_ptr(),
                                              tOut.data_ptr(), tCost.data_ptr(), tEnv.data_ptr())
            assert code == qfs.QFS_OK, lib.qfs_last_error().decode()
            torch.cuda.synchronize(dev)
            assert np.max(np.abs(tOut.cpu().numpy() - g_ref)) < 1e-10
            assert np.max(np.abs(tEnv.cpu().numpy() - e_ref)) < 1e-10
            assert np.max(np.abs(tCost.cpu().numpy() - c_ref)) < 1e-12


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2405_12866_gb300 import qfs
    lib = qfs.lib()
    n, pairs, M, S = 10, w.brick_pairs(10, 4), 64, 8   # needs far more than 16 MiB
    cir = qfs._CircuitArg(n, pairs)
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    code = lib.qfs_sweep_once_noalloc(None, C.byref(cir.c), dummy.data_ptr(), dummy.data_ptr(), M, S,
                                      0.0, dummy.data_ptr(), dummy.data_ptr(), None, None)
    assert code == qfs.QFS_EUNSUPPORTED
    assert "scratch" in lib.qfs_last_error().decode()
