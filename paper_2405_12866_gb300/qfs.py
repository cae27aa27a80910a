"""ctypes binding of libqfs (include/qfs.h).  Argument marshalling only.

Every computation runs in the library's CUDA kernels.  The library must be
built (``paper_2405_12866_gb300.build.build()``); if it is missing or cannot
load, `lib()` raises instead of falling back to anything else.

Host arrays are numpy complex128; device arrays are torch complex128 CUDA
tensors (their data pointers are handed to the library as they are).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqfs.so")

QFS_OK = 0
QFS_EINVAL = -1
QFS_ENOMEM = -2
QFS_ECUDA = -3
QFS_ETIMEOUT = -4
QFS_EUNSUPPORTED = -5
QFS_ENONFINITE = -6
QFS_EINTERNAL = -7
QFS_OPT_WAIT_LIMIT = 0
QFS_OPT_WORKSPACE_CAP = 1
QFS_OPT_FUSED_UPDATE = 2
QFS_OPT_DATAFLOW = 3
QFS_OPT_TWO_GATE_FORWARD = 4
QFS_OPT_FP64_TARGET_PRODUCT = 5
QFS_OPT_BATCH_LANES_PER_START = 6
QFS_FP64 = 0
QFS_MIXED = 1
QFS_STATES_HAAR = 0
QFS_STATES_BASIS = 1

# Every function the header declares; the CPU tests check the library exports them.
EXPORTS = [
    "qfs_default_params", "qfs_create", "qfs_destroy", "qfs_last_error", "qfs_device_sms",
    "qfs_generate_inputs", "qfs_generate_states", "qfs_instantiate", "qfs_instantiate_many",
    "qfs_instantiate_many_dev", "qfs_instantiate_ex", "qfs_instantiate_dev",
    "qfs_sweep_once", "qfs_gate_update", "qfs_profile_enable", "qfs_profile_reset",
    "qfs_profile_read", "qfs_sweep_once_noalloc", "qfs_instantiate_batch",
    "qfs_instantiate_batch_dev", "qfs_gemm_bf16_dev", "qfs_ws_create", "qfs_ws_destroy", "qfs_ws_params",
    "qfs_ws_loss_grad", "qfs_ws_train", "qfs_ws_predict",
    "qfs_dataflow_trace_enable", "qfs_dataflow_trace_read", "qfs_target_product_dev",
    "qfs_set_option", "qfs_get_option", "qfs_batch_sweep_once", "qfs_ws_instantiate",
    "qfs_batch_schedules", "qfs_batch_trace_enable", "qfs_batch_trace_read",
]
(PROF_BACKWARD, PROF_FORWARD, PROF_UPDATE, PROF_GEMM, PROF_RESIDUAL, PROF_CHECK, PROF_OTHER, PROF_BATCH,
 PROF_MLP, PROF_DATAFLOW) = range(10)
PROF_NAMES = ["backward", "forward", "update", "gemm", "residual", "check", "other", "batch", "mlp", "dataflow"]


class QfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qfs error {code}: {msg}")
        self.code = code


class Circuit(C.Structure):
    _fields_ = [("n", C.c_int32), ("L", C.c_int32), ("pairs", C.POINTER(C.c_int32))]


class Params(C.Structure):
    _fields_ = [("M", C.c_int32), ("multistarts", C.c_int32), ("max_sweeps", C.c_int32),
                ("min_sweeps", C.c_int32), ("plateau_window", C.c_int32),
                ("precision", C.c_int32), ("refine_sweeps_max", C.c_int32),
                ("start_groups", C.c_int32), ("seed", C.c_uint64), ("dist_tol", C.c_double),
                ("diff_tol_r", C.c_double), ("beta", C.c_double), ("restart_doubling", C.c_int32),
                ("overtrain_ratio", C.c_double), ("training_distribution", C.c_int32),
                ("concurrent_targets", C.c_int32), ("refine_switch_tol", C.c_double)]


class Result(C.Structure):
    _fields_ = [("cost", C.c_double), ("sweeps", C.c_int32), ("converged", C.c_int32),
                ("best_start", C.c_int32), ("fp64_sweeps", C.c_int32), ("training_states", C.c_int32)]


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    """Load libqfs.so (once).  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run paper_2405_12866_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    L.qfs_default_params.argtypes = [C.POINTER(Params)]
    L.qfs_default_params.restype = None
    L.qfs_create.argtypes = [C.POINTER(_P), C.c_int, _P]
    L.qfs_destroy.argtypes = [_P]
    L.qfs_destroy.restype = None
    L.qfs_last_error.argtypes = []
    L.qfs_last_error.restype = C.c_char_p
    L.qfs_device_sms.argtypes = [_P]
    L.qfs_generate_inputs.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P]
    L.qfs_generate_states.argtypes = [C.c_uint64, C.c_int32, C.c_uint32, C.c_int32, C.c_int32, _P]
    L.qfs_instantiate.argtypes = [_P, C.POINTER(Circuit), _P, C.POINTER(Params), _P,
                                  C.POINTER(Result), _P]
    L.qfs_instantiate_ex.argtypes = [_P, C.POINTER(Circuit), _P, _P, _P, C.POINTER(Params), _P,
                                     C.POINTER(Result), _P]
    L.qfs_instantiate_dev.argtypes = [_P, C.POINTER(Circuit), _P, _P, _P, C.POINTER(Params), _P,
                                      C.POINTER(Result), _P]
    L.qfs_instantiate_many.argtypes = [_P, C.POINTER(Circuit), C.c_int32, _P, _P, _P, C.POINTER(Params), _P,
                                       C.POINTER(Result), _P]
    L.qfs_instantiate_many_dev.argtypes = [_P, C.POINTER(Circuit), C.c_int32, _P, _P, _P, C.POINTER(Params), _P,
                                           C.POINTER(Result), _P]
    L.qfs_sweep_once.argtypes = [_P, C.POINTER(Circuit), _P, _P, C.c_int32, C.c_int32, _P,
                                 C.c_int32, C.c_double, _P, _P, _P]
    L.qfs_gate_update.argtypes = [_P, C.c_int32, _P, _P, C.c_double, _P]
    L.qfs_target_product_dev.argtypes = [_P, C.c_int32, C.c_int32, _P, _P, C.c_int32, _P]
    L.qfs_instantiate_batch.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P, _P, C.POINTER(Params), _P, _P]
    L.qfs_instantiate_batch_dev.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P, _P, C.POINTER(Params), _P, _P]
    L.qfs_gemm_bf16_dev.argtypes = [_P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, _P,
                                    C.c_int32, _P, C.c_int32, C.c_int32]
    L.qfs_ws_create.argtypes = [_P, C.c_uint64, C.c_int32, C.POINTER(_P)]
    L.qfs_ws_destroy.argtypes = [_P]
    L.qfs_ws_destroy.restype = None
    L.qfs_ws_params.argtypes = [_P, _P, _P, C.POINTER(C.c_int64)]
    L.qfs_ws_loss_grad.argtypes = [_P, C.c_int32, _P, _P, C.POINTER(C.c_double), _P]
    L.qfs_ws_train.argtypes = [_P, C.c_int32, _P, _P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64, _P]
    L.qfs_ws_predict.argtypes = [_P, C.c_int32, _P, _P]
    L.qfs_dataflow_trace_enable.argtypes = [_P, C.c_int64]
    L.qfs_dataflow_trace_read.argtypes = [_P, _P, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int64)]
    L.qfs_batch_trace_enable.argtypes = [_P, C.c_int64]
    L.qfs_batch_trace_read.argtypes = [_P, _P, C.c_int64, C.POINTER(C.c_int64)]
    L.qfs_sweep_once_noalloc.argtypes = [_P, C.POINTER(Circuit), _P, _P, C.c_int32, C.c_int32,
                                         C.c_double, _P, _P, _P, _P]
    L.qfs_profile_enable.argtypes = [_P, C.c_int]
    L.qfs_set_option.argtypes = [_P, C.c_int32, C.c_int64]
    L.qfs_batch_schedules.argtypes = [_P, C.c_int32, _P, C.POINTER(C.c_int32), _P, _P, C.POINTER(C.c_int32),
                                      _P, _P, C.POINTER(C.c_int32)]
    L.qfs_ws_instantiate.argtypes = [_P, C.c_int32, _P, _P, C.POINTER(Params), C.c_int32, _P, _P,
                                     C.POINTER(C.c_int64)]
    L.qfs_batch_sweep_once.argtypes = [_P, C.c_int32, _P, _P, _P, _P, _P, C.c_int32, C.c_int32, _P, C.c_int32,
                                       _P, _P]
    L.qfs_get_option.argtypes = [_P, C.c_int32, C.POINTER(C.c_int64)]
    L.qfs_profile_reset.argtypes = [_P]
    L.qfs_profile_read.argtypes = [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    _lib = L
    return L


def _check(code: int):
    if code != QFS_OK:
        raise QfsError(code, lib().qfs_last_error().decode())


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _host_c128(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} complex values, got {a.size}")
    return a


def _wait_torch(*tensors):
    """The library runs on its own stream: finish the work torch queued on
    its current stream (which may still be writing these tensors, or reading
    memory the caching allocator hands out next) before the call."""
    import torch
    seen = set()
    for t in tensors:
        if t is not None and t.is_cuda and t.device not in seen:
            seen.add(t.device)
            torch.cuda.current_stream(t.device).synchronize()


class _CircuitArg:
    def __init__(self, n: int, pairs):
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
        self.c = Circuit(n, len(self.pairs) // 2, self.pairs.ctypes.data_as(C.POINTER(C.c_int32)))


def default_params(**kw) -> Params:
    p = Params()
    lib().qfs_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


@dataclasses.dataclass
class InstantiateOutput:
    gates: object          # (L, 4, 4) numpy, or the device tensor given as out
    cost: float
    sweeps: int
    converged: bool
    best_start: int
    fp64_sweeps: int
    start_costs: np.ndarray
    training_states: int = 0


def generate_inputs(seed: int, n: int, M: int, S: int, L: int):
    """The library's own draws of samples (N x M) and initial gates (S, L, 4, 4)."""
    samples = np.zeros((1 << n, M), dtype=np.complex128)
    gates = np.zeros((S, L, 4, 4), dtype=np.complex128)
    _check(lib().qfs_generate_inputs(seed, n, M, S, L, samples.ctypes.data, gates.ctypes.data))
    return samples, gates


def generate_states(seed: int, distribution: int, stream: int, n: int, M: int) -> np.ndarray:
    """The library's own draw of M states (N x M) of either training
    distribution (QFS_STATES_HAAR or QFS_STATES_BASIS) on a stream
    (1 = training, 5 = validation)."""
    out = np.zeros((1 << n, M), dtype=np.complex128)
    _check(lib().qfs_generate_states(seed, distribution, stream, n, M, out.ctypes.data))
    return out


class Context:
    """A libqfs context on one CUDA device (optionally on a given stream)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self._h = _P()
        _check(lib().qfs_create(C.byref(self._h), device, stream))

    def close(self):
        if self._h:
            lib().qfs_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_sms(self) -> int:
        return lib().qfs_device_sms(self._h)

    def set_option(self, option: int, value: int):
        """qfs_set_option: one of the QFS_OPT_* settings of this context."""
        _check(lib().qfs_set_option(self._h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = C.c_int64()
        _check(lib().qfs_get_option(self._h, option, C.byref(v)))
        return v.value

    def instantiate(self, n, pairs, target, params: Params, samples=None, init_gates=None):
        """Host arrays in, numpy gates out.  samples/init_gates None -> drawn from params.seed."""
        cir = _CircuitArg(n, pairs)
        N = 1 << n
        target = _host_c128(target, (N, N))
        out = np.zeros((cir.c.L, 4, 4), dtype=np.complex128)
        res = Result()
        costs = np.zeros(params.multistarts, dtype=np.float64)
        if samples is None and init_gates is None:
            _check(lib().qfs_instantiate(self._h, C.byref(cir.c), target.ctypes.data, C.byref(params),
                                         out.ctypes.data, C.byref(res), costs.ctypes.data))
        else:
            samples = _host_c128(samples, (N, params.M))
            init_gates = _host_c128(init_gates, (params.multistarts, cir.c.L, 4, 4))
            _check(lib().qfs_instantiate_ex(self._h, C.byref(cir.c), target.ctypes.data,
                                            samples.ctypes.data, init_gates.ctypes.data,
                                            C.byref(params), out.ctypes.data, C.byref(res),
                                            costs.ctypes.data))
        return InstantiateOutput(out, res.cost, res.sweeps, bool(res.converged), res.best_start,
                                 res.fp64_sweeps, costs, res.training_states)

    def instantiate_many(self, n, pairs, targets, params: Params, samples=None, init_gates=None):
        """T targets (T, N, N) host arrays in one call; samples (T, N, M) and
        init_gates (T, S, L, 4, 4) or None (target t draws from seed + t).
        Returns a list of InstantiateOutput."""
        cir = _CircuitArg(n, pairs)
        N = 1 << n
        targets = np.ascontiguousarray(np.asarray(targets, dtype=np.complex128))
        T = targets.shape[0]
        targets = _host_c128(targets, (T, N, N))
        S, L = params.multistarts, cir.c.L
        sm = None if samples is None else _host_c128(samples, (T, N, params.M))
        ig = None if init_gates is None else _host_c128(init_gates, (T, S, L, 4, 4))
        out = np.zeros((T, L, 4, 4), dtype=np.complex128)
        res = (Result * T)()
        costs = np.zeros((T, S), dtype=np.float64)
        _check(lib().qfs_instantiate_many(self._h, C.byref(cir.c), T, targets.ctypes.data,
                                          None if sm is None else sm.ctypes.data,
                                          None if ig is None else ig.ctypes.data, C.byref(params),
                                          out.ctypes.data, res, costs.ctypes.data))
        return [InstantiateOutput(out[t], res[t].cost, res[t].sweeps, bool(res[t].converged), res[t].best_start,
                                  res[t].fp64_sweeps, costs[t], res[t].training_states) for t in range(T)]

    def instantiate_many_dev(self, n, pairs, targets, samples, init_gates, params: Params, out):
        """Device (torch complex128 CUDA) tensors: targets (T, N, N), samples
        (T, N, M), init_gates (T, S, L, 4, 4), out (T, L, 4, 4)."""
        cir = _CircuitArg(n, pairs)
        for name, t in (("targets", targets), ("samples", samples), ("init_gates", init_gates), ("out", out)):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
        T = targets.shape[0]
        res = (Result * T)()
        costs = np.zeros((T, params.multistarts), dtype=np.float64)
        _wait_torch(targets, samples, init_gates, out)
        _check(lib().qfs_instantiate_many_dev(self._h, C.byref(cir.c), T, targets.data_ptr(), samples.data_ptr(),
                                              init_gates.data_ptr(), C.byref(params), out.data_ptr(), res,
                                              costs.ctypes.data))
        return [InstantiateOutput(out[t], res[t].cost, res[t].sweeps, bool(res[t].converged), res[t].best_start,
                                  res[t].fp64_sweeps, costs[t], res[t].training_states) for t in range(T)]

    def instantiate_dev(self, n, pairs, target, samples, init_gates, params: Params, out):
        """Device (torch complex128 CUDA) tensors in and out."""
        cir = _CircuitArg(n, pairs)
        for name, t in (("target", target), ("samples", samples), ("init_gates", init_gates), ("out", out)):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
        res = Result()
        costs = np.zeros(params.multistarts, dtype=np.float64)
        _wait_torch(target, samples, init_gates, out)
        _check(lib().qfs_instantiate_dev(self._h, C.byref(cir.c), target.data_ptr(), samples.data_ptr(),
                                         init_gates.data_ptr(), C.byref(params), out.data_ptr(),
                                         C.byref(res), costs.ctypes.data))
        return InstantiateOutput(out, res.cost, res.sweeps, bool(res.converged), res.best_start,
                                 res.fp64_sweeps, costs, res.training_states)

    def target_product(self, n, target, samples, precision=QFS_FP64, out=None):
        """Phi_L = U Psi on device (torch complex128 CUDA) tensors."""
        M = samples.shape[1]
        for name, t in (("target", target), ("samples", samples)):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.complex128"):
                raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
        if out is None:
            import torch
            out = torch.empty((1 << n, M), dtype=torch.complex128, device=samples.device)
        _wait_torch(target, samples, out)
        _check(lib().qfs_target_product_dev(self._h, n, M, target.data_ptr(), samples.data_ptr(), precision,
                                            out.data_ptr()))
        return out

    def sweep_once(self, n, pairs, target, samples, gates, precision=QFS_FP64, beta=0.0,
                   want_envs=True):
        """One sweep for S starts; returns (gates (S,L,4,4), envs or None, costs (S,))."""
        cir = _CircuitArg(n, pairs)
        N = 1 << n
        gates = _host_c128(gates)
        S = gates.shape[0] if gates.ndim == 4 else 1
        gates = gates.reshape(S, cir.c.L, 4, 4)
        samples = _host_c128(samples)
        M = samples.shape[1]
        target = _host_c128(target, (N, N))
        out = np.zeros_like(gates)
        envs = np.zeros_like(gates) if want_envs else None
        costs = np.zeros(S)
        _check(lib().qfs_sweep_once(self._h, C.byref(cir.c), target.ctypes.data, samples.ctypes.data,
                                    M, S, gates.ctypes.data, precision, beta, out.ctypes.data,
                                    envs.ctypes.data if envs is not None else None, costs.ctypes.data))
        return out, envs, costs

    def instantiate_batch(self, problems, params: Params, samples=None, init_gates=None):
        """problems: list of (n, pairs, U).  samples/init_gates: lists per problem or None
        (drawn from params.seed + index).  Returns (list of (L,4,4) gates, list of dicts)."""
        ns = np.array([pr[0] for pr in problems], dtype=np.int32)
        Ls = np.array([len(pr[1]) for pr in problems], dtype=np.int32)
        pairs = np.concatenate([np.asarray(pr[1], dtype=np.int32).reshape(-1) for pr in problems])
        targets = np.concatenate([_host_c128(pr[2]).reshape(-1) for pr in problems])
        sm = None if samples is None else np.concatenate([_host_c128(x).reshape(-1) for x in samples])
        ig = None if init_gates is None else np.concatenate([_host_c128(x).reshape(-1) for x in init_gates])
        out, info = self.instantiate_batch_packed(ns, Ls, pairs, targets, sm, ig, params)
        offs = np.concatenate([[0], np.cumsum(Ls * 16)])
        return [out[offs[i]:offs[i + 1]].reshape(Ls[i], 4, 4) for i in range(len(problems))], info

    def instantiate_batch_packed(self, ns, Ls, pairs, targets, samples, init_gates, params: Params, out=None):
        """qfs_instantiate_batch on packed host arrays, laid out as
        instantiate_batch_dev takes them: ns, Ls, pairs int32; targets, samples,
        init_gates complex128, problem after problem (samples and init_gates may
        be None: drawn from params.seed + index).  The library copies straight
        from these arrays (by DMA when they are pinned).  out: optional host
        complex128 array of Ls.sum() * 16 for the gates.  Returns (out, list of
        per-problem dicts)."""
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        targets = np.ascontiguousarray(targets, dtype=np.complex128)
        sm = None if samples is None else np.ascontiguousarray(samples, dtype=np.complex128)
        ig = None if init_gates is None else np.ascontiguousarray(init_gates, dtype=np.complex128)
        P = len(ns)
        if out is None:
            out = np.zeros(int(Ls.sum()) * 16, dtype=np.complex128)
        elif out.dtype != np.complex128 or not out.flags.c_contiguous or out.size != int(Ls.sum()) * 16:
            raise ValueError("out must be a contiguous complex128 array of Ls.sum() * 16 entries")
        res = (Result * P)()
        _check(lib().qfs_instantiate_batch(self._h, P, ns.ctypes.data, Ls.ctypes.data, pairs.ctypes.data,
                                           targets.ctypes.data, sm.ctypes.data if sm is not None else None,
                                           ig.ctypes.data if ig is not None else None, C.byref(params),
                                           out.ctypes.data, res))
        info = [dict(cost=r.cost, sweeps=r.sweeps, converged=bool(r.converged), best_start=r.best_start,
                     fp64_sweeps=r.fp64_sweeps, training_states=r.training_states) for r in res]
        return out, info

    def batch_schedules(self):
        """The batched form's tuned shapes: (list of dicts per class, list of
        dicts per timed trial)."""
        nt, nr, npl = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().qfs_batch_schedules(self._h, 0, None, C.byref(nt), None, None, C.byref(nr), None, None,
                                         C.byref(npl)))
        cap = max(nt.value, nr.value, npl.value, 1)
        tuned = np.zeros((cap, 6), dtype=np.int32)
        trials = np.zeros((cap, 6), dtype=np.int32)
        tns = np.zeros(cap)
        pc = np.zeros(cap, dtype=np.int32)
        pms = np.zeros((cap, 3))
        _check(lib().qfs_batch_schedules(self._h, cap, tuned.ctypes.data, C.byref(nt), trials.ctypes.data,
                                         tns.ctypes.data, C.byref(nr), pc.ctypes.data, pms.ctypes.data,
                                         C.byref(npl)))
        keys = ("n", "L", "M", "S", "G", "warps")
        self.batch_plans = [dict(choice=int(c), ms_per_class=float(m[0]), ms_warp_per_start=float(m[1]),
                                 ms_16_lanes=float(m[2]))
                            for c, m in zip(pc[:npl.value], pms[:npl.value])]
        return ([dict(zip(keys, map(int, r))) for r in tuned[:nt.value]],
                [dict(zip(keys, map(int, r)), ns_per_start_sweep=float(t)) for r, t in zip(trials[:nr.value],
                                                                                             tns[:nr.value])])

    def batch_sweep_once(self, problems, samples, init_gates, M: int = 0, lanes_per_start: int = 0):
        """qfs_batch_sweep_once: one complex64 batched sweep of every start.
        problems: list of (n, pairs, U); samples and init_gates (S, L, 4, 4)
        lists per problem.  Returns (list of (S, L, 4, 4) swept gates, (P, S) costs)."""
        P = len(problems)
        ns = np.array([pr[0] for pr in problems], dtype=np.int32)
        Ls = np.array([len(pr[1]) for pr in problems], dtype=np.int32)
        S = int(np.asarray(init_gates[0]).shape[0])
        pairs = np.ascontiguousarray(np.concatenate([np.asarray(pr[1], dtype=np.int32).reshape(-1)
                                                     for pr in problems]))
        targets = np.ascontiguousarray(np.concatenate([_host_c128(pr[2]).reshape(-1) for pr in problems]))
        sm = np.ascontiguousarray(np.concatenate([_host_c128(x).reshape(-1) for x in samples]))
        ig = np.ascontiguousarray(np.concatenate([_host_c128(x).reshape(-1) for x in init_gates]))
        out = np.zeros_like(ig)
        costs = np.zeros((P, S), dtype=np.float64)
        _check(lib().qfs_batch_sweep_once(self._h, P, ns.ctypes.data, Ls.ctypes.data, pairs.ctypes.data,
                                          targets.ctypes.data, sm.ctypes.data, M, S, ig.ctypes.data,
                                          lanes_per_start, out.ctypes.data, costs.ctypes.data))
        gates, offs = [], np.concatenate([[0], np.cumsum(S * Ls * 16)])
        for i in range(P):
            gates.append(out[offs[i]:offs[i + 1]].reshape(S, Ls[i], 4, 4))
        return gates, costs

    def instantiate_batch_uniform(self, n, pairs, targets, params: Params, init_gates=None):
        """P problems of one structure: targets (P, N, N), init_gates (P, S, L, 4, 4)
        or None (drawn from params.seed + index), samples drawn from params.seed +
        index.  Returns (gates (P, L, 4, 4), cost, sweeps, converged, best_start)."""
        t = _host_c128(targets)
        P = t.shape[0]
        L = len(pairs)
        ns = np.full(P, n, dtype=np.int32)
        Ls = np.full(P, L, dtype=np.int32)
        pr = np.ascontiguousarray(np.tile(np.asarray(pairs, dtype=np.int32).reshape(-1), P))
        ig = None if init_gates is None else _host_c128(init_gates)
        if ig is not None and ig.size != P * params.multistarts * L * 16:
            raise ValueError("init_gates must hold P x multistarts x L gates")
        out = np.zeros((P, L, 4, 4), dtype=np.complex128)
        res = (Result * P)()
        _check(lib().qfs_instantiate_batch(self._h, P, ns.ctypes.data, Ls.ctypes.data, pr.ctypes.data,
                                           t.ctypes.data, None, ig.ctypes.data if ig is not None else None,
                                           C.byref(params), out.ctypes.data, res))
        r = np.frombuffer(res, dtype=np.dtype([("cost", "f8"), ("sweeps", "i4"), ("converged", "i4"),
                                                ("best_start", "i4"), ("fp64_sweeps", "i4"),
                                                ("training_states", "i4")], align=True), count=P)
        return out, r["cost"].copy(), r["sweeps"].copy(), r["converged"].astype(bool), r["best_start"].copy()

    def instantiate_batch_dev(self, ns, Ls, pairs, targets, samples, init_gates, params: Params, out):
        """Packed device tensors (torch complex128): targets, samples, init_gates, out;
        ns, Ls, pairs host int32 arrays.  Returns the list of per-problem result dicts."""
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        P = len(ns)
        res = (Result * P)()
        _wait_torch(targets, samples, init_gates, out)
        _check(lib().qfs_instantiate_batch_dev(self._h, P, ns.ctypes.data, Ls.ctypes.data, pairs.ctypes.data,
                                               targets.data_ptr(), samples.data_ptr(), init_gates.data_ptr(),
                                               C.byref(params), out.data_ptr(), res))
        return [dict(cost=r.cost, sweeps=r.sweeps, converged=bool(r.converged), best_start=r.best_start,
                     fp64_sweeps=r.fp64_sweeps) for r in res]

    def gemm_bf16(self, A, B, bias=None, gelu=False, want_f32=True, want_bf16=False, M_valid=0):
        """C = A B^T (+ bias, GELU) for bf16 CUDA tensors A (M x K), B (N x K)."""
        import torch
        M, K = A.shape
        N = B.shape[0]
        C32 = torch.empty((M, N), dtype=torch.float32, device=A.device) if want_f32 else None
        C16 = torch.empty((M, N), dtype=torch.bfloat16, device=A.device) if want_bf16 else None
        _wait_torch(A, B, C32, C16, bias)
        _check(lib().qfs_gemm_bf16_dev(self._h, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                       C32.data_ptr() if C32 is not None else None,
                                       C16.data_ptr() if C16 is not None else None, N,
                                       bias.data_ptr() if bias is not None else None, int(gelu), M_valid))
        return C32, C16

    def dataflow_trace(self, capacity: int):
        """Record step time stamps of dataflow sweeps (capacity stamps; 0: off)."""
        _check(lib().qfs_dataflow_trace_enable(self._h, capacity))

    def dataflow_trace_read(self):
        """Stamps of the last traced sweep: (steps, starts, 4) uint64 ns (first chunk
        started, last chunk done, partials summed (updates only), step published) and
        (items, 4) per work item (dequeued, ready, processed, CTA index) or None."""
        st, S, it = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().qfs_dataflow_trace_read(self._h, None, 0, C.byref(st), C.byref(S), C.byref(it)))
        n = st.value * S.value * 4 + it.value * 4
        out = np.zeros(n, dtype=np.uint64)
        if n:
            _check(lib().qfs_dataflow_trace_read(self._h, out.ctypes.data, n, C.byref(st), C.byref(S), C.byref(it)))
        steps = out[:st.value * S.value * 4].reshape(st.value, S.value, 4)
        items = out[st.value * S.value * 4:].reshape(it.value, 4) if it.value else None
        return steps, items

    def batch_trace(self, capacity: int):
        """Record unit time stamps of batched runs (capacity stamps, 4 per unit; 0: off)."""
        _check(lib().qfs_batch_trace_enable(self._h, capacity))

    def batch_trace_read(self):
        """Stamps of the last traced batched run as a dict of per-unit arrays:
        t0, t1 (ns, unit taken and finished), problem, sm, s0 (first start),
        starts, G (lanes per start)."""
        nu = C.c_int64()
        _check(lib().qfs_batch_trace_read(self._h, None, 0, C.byref(nu)))
        out = np.zeros(4 * nu.value, dtype=np.uint64)
        if nu.value:
            _check(lib().qfs_batch_trace_read(self._h, out.ctypes.data, out.size, C.byref(nu)))
        r = out.reshape(-1, 4)
        return dict(t0=r[:, 0].copy(), t1=r[:, 1].copy(), problem=r[:, 2].astype(np.int64),
                    sm=(r[:, 3] >> np.uint64(32)).astype(np.int64),
                    s0=((r[:, 3] >> np.uint64(16)) & np.uint64(0xffff)).astype(np.int64),
                    starts=((r[:, 3] >> np.uint64(8)) & np.uint64(0xff)).astype(np.int64),
                    G=(r[:, 3] & np.uint64(0xff)).astype(np.int64))

    def profile(self, enable: bool):
        _check(lib().qfs_profile_enable(self._h, int(enable)))

    def profile_reset(self):
        _check(lib().qfs_profile_reset(self._h))

    def profile_read(self, kind: int = -1) -> dict:
        """Counters of one kernel kind (PROF_*), or of all with kind = -1."""
        l, t, ms, by = C.c_int64(), C.c_int64(), C.c_double(), C.c_double()
        _check(lib().qfs_profile_read(self._h, kind, C.byref(l), C.byref(t), C.byref(ms), C.byref(by)))
        return {"launches": l.value, "timed": t.value, "ms": ms.value, "bytes": by.value}

    def gate_update(self, envs, gates_old=None, beta=0.0):
        envs = _host_c128(envs).reshape(-1, 4, 4)
        out = np.zeros_like(envs)
        g = None if gates_old is None else _host_c128(gates_old).reshape(-1, 4, 4)
        _check(lib().qfs_gate_update(self._h, envs.shape[0], envs.ctypes.data,
                                     g.ctypes.data if g is not None else None, beta, out.ctypes.data))
        return out


class WarmStart:
    """The learned warm-start network (weights on the context's device)."""

    DIMS = [(256, 1024), (1024, 1024), (1024, 1024), (1024, 256)]   # (in, out) per layer

    def __init__(self, ctx: Context, seed: int = 0, batch_cap: int = 4096):
        self._h = _P()
        self.ctx = ctx
        _check(lib().qfs_ws_create(ctx._h, seed, batch_cap, C.byref(self._h)))

    def close(self):
        if self._h:
            lib().qfs_ws_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        n = C.c_int64()
        _check(lib().qfs_ws_params(self._h, None, None, C.byref(n)))
        out = np.zeros(n.value, dtype=np.float32)
        _check(lib().qfs_ws_params(self._h, out.ctypes.data, None, C.byref(n)))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        n = C.c_int64()
        _check(lib().qfs_ws_params(self._h, None, flat.ctypes.data, C.byref(n)))

    @classmethod
    def unflatten(cls, flat):
        """Flat parameter vector -> list of (W [out, in], b [out])."""
        out, off = [], 0
        for din, dout in cls.DIMS:
            W = flat[off:off + din * dout].reshape(dout, din)
            off += din * dout
            b = flat[off:off + dout]
            off += dout
            out.append((W, b))
        return out

    def loss_grad(self, targets, labels):
        t = _host_c128(targets)
        lab = np.ascontiguousarray(labels, dtype=np.float64)
        count = t.size // 256
        loss = C.c_double()
        n = C.c_int64()
        _check(lib().qfs_ws_params(self._h, None, None, C.byref(n)))
        g = np.zeros(n.value, dtype=np.float32)
        _check(lib().qfs_ws_loss_grad(self._h, count, t.ctypes.data, lab.ctypes.data, C.byref(loss), g.ctypes.data))
        return loss.value, g

    def train(self, targets, labels, epochs=1, batch=4096, lr=1e-3, seed=0, lr_final=None):
        t = _host_c128(targets)
        lab = np.ascontiguousarray(labels, dtype=np.float64)
        count = t.size // 256
        losses = np.zeros(epochs)
        _check(lib().qfs_ws_train(self._h, count, t.ctypes.data, lab.ctypes.data, epochs, batch, lr,
                                  lr if lr_final is None else lr_final, seed, losses.ctypes.data))
        return losses

    def instantiate(self, targets, params: Params, first_sweeps: int = 100, first_gates=None):
        """qfs_ws_instantiate: the two-stage policy (predicted first start,
        random multistarts as the fallback) for targets (P, 16, 16).  Returns
        (gates (P, 6, 4, 4), result records, stats dict)."""
        t = _host_c128(targets)
        P = t.size // 256
        fg = None if first_gates is None else _host_c128(first_gates, (P, 6, 4, 4))
        out = np.zeros((P, 6, 4, 4), dtype=np.complex128)
        res = (Result * P)()
        st = (C.c_int64 * 4)()
        _check(lib().qfs_ws_instantiate(self._h, P, t.ctypes.data, fg.ctypes.data if fg is not None else None,
                                        C.byref(params), first_sweeps, out.ctypes.data, res, st))
        r = np.frombuffer(res, dtype=np.dtype([("cost", "f8"), ("sweeps", "i4"), ("converged", "i4"),
                                                ("best_start", "i4"), ("fp64_sweeps", "i4"),
                                                ("training_states", "i4")], align=True), count=P).copy()
        return out, r, dict(first_converged=int(st[0]), first_start_sweeps=int(st[1]),
                            fallback_start_sweeps=int(st[2]), fallback_targets=int(st[3]))

    def predict(self, targets):
        t = _host_c128(targets)
        count = t.size // 256
        out = np.zeros((count, 6, 4, 4), dtype=np.complex128)
        _check(lib().qfs_ws_predict(self._h, count, t.ctypes.data, out.ctypes.data))
        return out
