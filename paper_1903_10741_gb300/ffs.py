"""Python binding of the C ABI in ``include/ffs.h`` (ctypes, argument marshalling only).

Every computation runs in ``libffs.so``'s CUDA kernels.  Device buffers are torch CUDA
tensors (PyTorch supplies device memory and streams); host results are numpy arrays.
There is no CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

FFS_OK = 0
ORDER_TOPO, ORDER_STAGE = 0, 1
MACH_GENE, MACH_EARLIEST = 0, 1
PLACE_INSERT = 4  # or-ed into a machine mode: idle-gap insertion placement
ST_FREE, ST_EXEC, ST_DONE, ST_FIXED = 0, 1, 2, 3
E_TIMEOUT = -5
E_STOPPED = -9  # a batched run ended early on ga_batch_stop
INJECT_NONE, INJECT_TABLE_COPY, INJECT_GEMM_LOADS = 0, 1, 2  # ffs_debug_inject (tests only)
KEEP_SLOT, KEEP_ISLAND, KEEP_ISLAND_OFFSPRING = 0, 1, 2  # keep rules of surrogate-assisted generations

_i32p = C.POINTER(C.c_int32)
_lib = None


class FFSError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = lib().ffs_strerror(code).decode() if _lib is not None else str(code)
        if _lib is not None and code == -4:
            msg += " [" + lib().ffs_last_error().decode() + "]"
        super().__init__(f"{what}: {msg} ({code})")


class Problem_c(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("n_stages", C.c_int32), ("machines_per_stage", _i32p),
                ("proc", _i32p), ("power", _i32p), ("release", _i32p), ("due", _i32p),
                ("peak_power", C.c_int32), ("wt", C.c_int32), ("proc_machine", _i32p),
                ("power_machine", _i32p)]


class Arrivals_c(C.Structure):
    _fields_ = [("job_count", C.c_int32), ("proc", _i32p), ("release", _i32p), ("due", _i32p),
                ("proc_machine", _i32p), ("power_machine", _i32p)]


def _arrivals_c(arrivals, keep: list):
    p, R, D = _i32(arrivals.p), _i32(arrivals.R), _i32(arrivals.D)
    pm = getattr(arrivals, "pm", None)
    qm = getattr(arrivals, "qm", None)
    pm = None if pm is None else _i32(pm)
    qm = None if qm is None else _i32(qm)
    keep.extend([p, R, D, pm, qm])
    return Arrivals_c(int(p.shape[0]), _p(p), _p(R), _p(D), None if pm is None else _p(pm),
                      None if qm is None else _p(qm))


class GAParams_c(C.Structure):
    _fields_ = [("pop", C.c_int32), ("island", C.c_int32), ("tournament_k", C.c_int32),
                ("pc_num", C.c_int32), ("pc_den", C.c_int32), ("pm_num", C.c_int32),
                ("pm_den", C.c_int32), ("order_mode", C.c_int32), ("machine_mode", C.c_int32),
                ("migrate_every", C.c_int32), ("instance_id", C.c_int32), ("seed", C.c_uint64),
                ("cuda_stream", C.c_void_p)]


class Result_c(C.Structure):
    _fields_ = [("objective", C.c_int64), ("total_tardiness", C.c_int64), ("makespan", C.c_int32),
                ("n_ops", C.c_int32), ("start", _i32p), ("machine", _i32p)]


class BatchConfig_c(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("smem_bytes", C.c_int32), ("ctas", C.c_int32),
                ("cluster", C.c_int32), ("ms_per_generation", C.c_float)]


class ServiceConfig_c(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("pad", C.c_int32), ("memory_bytes", C.c_int64),
                ("ga", GAParams_c)]


class RequestInfo_c(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("warm", C.c_int32), ("generations", C.c_int32),
                ("submit_ns", C.c_int64), ("admit_ns", C.c_int64), ("done_ns", C.c_int64),
                ("footprint", C.c_int64), ("n_ops", C.c_int32), ("pad", C.c_int32)]


class ServiceStats_c(C.Structure):
    _fields_ = [("active", C.c_int32), ("queued", C.c_int32), ("warm", C.c_int32), ("pad", C.c_int32),
                ("completed", C.c_int64), ("failed", C.c_int64), ("memory_bytes", C.c_int64),
                ("used_bytes", C.c_int64), ("peak_bytes", C.c_int64)]


class Info_c(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("n_stages", C.c_int32), ("n_machines", C.c_int32),
                ("n_genes", C.c_int32), ("rs", C.c_int32), ("horizon", C.c_int32),
                ("peak_power", C.c_int32), ("wt", C.c_int32)]


_SIGS = {
    "ffs_strerror": (C.c_char_p, [C.c_int]),
    "ffs_last_error": (C.c_char_p, []),
    "ffs_instance_create": (C.c_int, [C.POINTER(Problem_c), C.POINTER(C.c_void_p)]),
    "ffs_instance_destroy": (C.c_int, [C.c_void_p]),
    "ffs_instance_info": (C.c_int, [C.c_void_p, C.POINTER(Info_c)]),
    "ffs_instance_genes": (C.c_int, [C.c_void_p, _i32p, _i32p]),
    "ffs_instance_status": (C.c_int, [C.c_void_p, _i32p]),
    "ffs_commit": (C.c_int, [C.c_void_p, _i32p, _i32p]),
    "ffs_reschedule": (C.c_int, [C.c_void_p, C.POINTER(Arrivals_c), C.c_int32]),
    "ffs_reschedule_static": (C.c_int, [C.c_void_p, C.POINTER(Arrivals_c), C.c_int32]),
    "ffs_decode": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ffs_decode_schedule": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ffs_decode_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ffs_decode_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ga_population_create": (C.c_int, [C.c_void_p, C.POINTER(GAParams_c), C.POINTER(C.c_void_p)]),
    "ga_population_destroy": (C.c_int, [C.c_void_p]),
    "ga_population_create_warm": (C.c_int, [C.c_void_p, C.POINTER(GAParams_c), C.c_void_p, C.POINTER(C.c_void_p)]),
    "ga_population_footprint": (C.c_int, [C.c_void_p, C.POINTER(GAParams_c), C.POINTER(C.c_int64)]),
    "ffs_service_create": (C.c_int, [C.POINTER(ServiceConfig_c), C.POINTER(C.c_void_p)]),
    "ffs_service_destroy": (C.c_int, [C.c_void_p]),
    "ffs_service_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Arrivals_c), C.c_int32, C.c_int32,
                                     C.POINTER(C.c_int64)]),
    "ffs_service_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(RequestInfo_c), C.POINTER(Result_c)]),
    "ffs_service_forget": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ffs_service_stop_request": (C.c_int, [C.c_void_p, C.c_int64]),
    "ffs_service_stats_read": (C.c_int, [C.c_void_p, C.POINTER(ServiceStats_c)]),
    "ga_run": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Result_c)]),
    "ga_population_read": (C.c_int, [C.c_void_p] + [C.c_void_p] * 10),
    "ga_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "ga_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "ffs_kernel_launches": (C.c_int, [C.POINTER(C.c_uint64)]),
    "ffs_surrogate_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ffs_surrogate_destroy": (C.c_int, [C.c_void_p]),
    "ffs_surrogate_param_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "ffs_surrogate_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ffs_surrogate_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ffs_surrogate_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "ffs_surrogate_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ffs_surrogate_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p]),
    "ffs_debug_inject": (C.c_int, [C.c_int32]),
    "ffs_debug_bounds_faults": (C.c_int, [C.POINTER(C.c_uint32)]),
    "ga_population_surrogate_keep": (C.c_int, [C.c_void_p, C.c_int32]),
    "ffs_surrogate_score_exactly": (C.c_int, [C.c_void_p, C.c_int32]),
    "ga_profile_read_phases": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ga_population_read_candidates": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ffs_surrogate_read_activations": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                                 C.c_void_p]),
    "ga_population_attach_surrogate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_int32, C.c_int32]),
    "ffs_surrogate_pretrain": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p]),
    "ga_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(GAParams_c), C.POINTER(C.c_void_p)]),
    "ga_batch_destroy": (C.c_int, [C.c_void_p]),
    "ga_batch_run": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "ga_batch_stop": (C.c_int, [C.c_void_p]),
    "ga_batch_read": (C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 10),
    "ga_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "ga_batch_get_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ga_batch_set_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ffs_tensor_gemm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_int32, C.c_void_p]),
    "ga_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "ga_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}


def debug_inject(mode: int):
    """Failure injection for tests of the bounded device waits (``ffs_debug_inject``)."""
    _check(lib().ffs_debug_inject(int(mode)), "ffs_debug_inject")


def kernel_launches() -> int:
    """Kernels launched by libffs in this process so far."""
    n = C.c_uint64(0)
    _check(lib().ffs_kernel_launches(C.byref(n)), "ffs_kernel_launches")
    return int(n.value)


def bounds_faults() -> int:
    """Device indices found out of range since the last call (bounds-checked builds only)."""
    n = C.c_uint32()
    _check(lib().ffs_debug_bounds_faults(C.byref(n)), "ffs_debug_bounds_faults")
    return int(n.value)


def header_functions():
    """Names of the functions declared in include/ffs.h."""
    with open(os.path.join(_build.INCLUDE, "ffs.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(\w+)\s*\(", text, flags=re.M)))


def lib():
    """Loads libffs.so (building it first if it is missing or stale); with the environment
    variable FFS_CHECKED=1, the bounds-checked build instead."""
    global _lib
    if _lib is None:
        path = _build.build(checked=os.environ.get("FFS_CHECKED") == "1")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != FFS_OK:
        raise FFSError(rc, what)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dptr(t):
    return None if t is None else t.data_ptr()


class Instance:
    """An EDFFS instance held by the library (``ffs_instance``)."""

    def __init__(self, problem):
        self._keep = [_i32(problem.o), _i32(problem.p), _i32(problem.q), _i32(problem.R), _i32(problem.D)]
        o, p, q, R, D = self._keep
        pm, qm = getattr(problem, "pm", None), getattr(problem, "qm", None)
        pm = None if pm is None else _i32(pm)
        qm = None if qm is None else _i32(qm)
        self._keep += [pm, qm]
        pr = Problem_c(int(p.shape[0]), int(o.shape[0]), _p(o), _p(p), _p(q), _p(R), _p(D),
                       int(problem.Qmax), int(problem.WT), None if pm is None else _p(pm),
                       None if qm is None else _p(qm))
        h = C.c_void_p()
        _check(lib().ffs_instance_create(C.byref(pr), C.byref(h)), "ffs_instance_create")
        self._h = h
        self._keep = None

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ffs_instance_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = Info_c()
        _check(lib().ffs_instance_info(self._h, C.byref(i)), "ffs_instance_info")
        return {n: getattr(i, n) for n, _ in Info_c._fields_}

    @property
    def K(self) -> int:
        return self.info()["n_genes"]

    def genes(self):
        K = self.K
        gj = np.zeros(max(K, 1), np.int32)
        gs = np.zeros(max(K, 1), np.int32)
        _check(lib().ffs_instance_genes(self._h, _p(gj), _p(gs)), "ffs_instance_genes")
        return gj[:K], gs[:K]

    def status(self) -> np.ndarray:
        inf = self.info()
        st = np.zeros((inf["n_jobs"], inf["n_stages"]), np.int32)
        _check(lib().ffs_instance_status(self._h, _p(st)), "ffs_instance_status")
        return st

    def commit(self, S, M):
        S, M = _i32(S), _i32(M)
        _check(lib().ffs_commit(self._h, _p(S), _p(M)), "ffs_commit")

    def reschedule(self, arrivals, t_now: int, static: bool = False):
        """Rescheduling point t_now with new jobs (Sec. 4.1); ``static`` keeps the executed
        plan and schedules only the new jobs after it (``ffs_reschedule_static``)."""
        keep = []
        a = _arrivals_c(arrivals, keep)
        fn = lib().ffs_reschedule_static if static else lib().ffs_reschedule
        _check(fn(self._h, C.byref(a), int(t_now)), "ffs_reschedule_static" if static else "ffs_reschedule")

    def decode(self, y, x=None, order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST, stream=None,
               schedule=False, check=True):
        """Decodes device chromosomes ``y`` (int16 [count, K]) and ``x`` (int8, machine genes).
        Returns device tensors: obj (int64), tard, cmax, and with ``schedule`` S, M [count, N, g]."""
        import torch
        count = int(y.shape[0]) if y.dim() == 2 else 1
        dev = y.device
        obj = torch.empty(count, dtype=torch.int64, device=dev)
        st = _stream_ptr(stream)
        out = {"obj": obj}
        if schedule:
            inf = self.info()
            S = torch.empty((count, inf["n_jobs"], inf["n_stages"]), dtype=torch.int32, device=dev)
            M = torch.empty_like(S)
            _check(lib().ffs_decode_schedule(self._h, order_mode, mach_mode, _dptr(y), _dptr(x), count,
                                             _dptr(obj), _dptr(S), _dptr(M), st), "ffs_decode_schedule")
            out.update(S=S, M=M)
        else:
            tard = torch.empty(count, dtype=torch.int64, device=dev)
            cmax = torch.empty(count, dtype=torch.int32, device=dev)
            _check(lib().ffs_decode(self._h, order_mode, mach_mode, _dptr(y), _dptr(x), count,
                                    _dptr(obj), _dptr(tard), _dptr(cmax), st), "ffs_decode")
            out.update(tard=tard, cmax=cmax)
        if check:
            _check(lib().ffs_decode_check(self._h, st), "ffs_decode")
        return out

    def decode_noalloc(self, y, x=None, order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST, stream=None):
        """Decodes like ``decode`` through ``ffs_decode_noalloc``: the library uses only its
        fixed internal device scratch, never allocating, for callers that cannot allocate
        (a fixed device-memory budget, a framework allocator that owns the memory, loops
        that must not wait on the allocator).  The output tensors are allocated here, on
        the caller's side.  Synchronous."""
        import torch
        count = int(y.shape[0]) if y.dim() == 2 else 1
        obj = torch.empty(count, dtype=torch.int64, device=y.device)
        tard = torch.empty(count, dtype=torch.int64, device=y.device)
        cmax = torch.empty(count, dtype=torch.int32, device=y.device)
        _check(lib().ffs_decode_noalloc(self._h, order_mode, mach_mode, _dptr(y), _dptr(x), count,
                                        _dptr(obj), _dptr(tard), _dptr(cmax), _stream_ptr(stream)),
               "ffs_decode_noalloc")
        return {"obj": obj, "tard": tard, "cmax": cmax}


def ga_params(P: int, island: int = 64, tour_k: int = 2, pc=(4, 5), pm=(1, 10), order_mode=ORDER_STAGE,
              mach_mode=MACH_EARLIEST, migrate_every: int = 10, seed: int = 1, instance_id: int = 0,
              stream_ptr=None) -> GAParams_c:
    return GAParams_c(P, min(island, P), tour_k, pc[0], pc[1], pm[0], pm[1], order_mode, mach_mode,
                      migrate_every, instance_id, seed, stream_ptr)


def footprint(inst: Instance, P: int, **kw) -> int:
    """Device bytes of a population of ``inst`` (``ga_population_footprint``)."""
    n = C.c_int64()
    par = ga_params(P, **kw)
    _check(lib().ga_population_footprint(inst.handle, C.byref(par), C.byref(n)), "ga_population_footprint")
    return int(n.value)


def tensor_gemm(A, B, bias=None, relu_bf16: bool = False, stream=None):
    """C = A . B^T on the tcgen05 tensor cores (``ffs_tensor_gemm``): A [M, K] and B [N, K]
    BF16 CUDA tensors; FP32 [M, N] result, or relu(A . B^T + bias) as BF16."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.bfloat16 if relu_bf16 else torch.float32, device=A.device)
    _check(lib().ffs_tensor_gemm(_dptr(A), _dptr(B), M, N, K, _dptr(bias), _dptr(C), 1 if relu_bf16 else 0, 1,
                                 _stream_ptr(stream)), "ffs_tensor_gemm")
    return C


class Population:
    """A device-resident GA population (``ga_population``).  With ``prev`` (an earlier
    population of the same instance), generation 0 is ``prev``'s population carried over
    to the instance's present genes (``ga_population_create_warm``)."""

    def __init__(self, inst: Instance, P: int, island: int = 64, tour_k: int = 2, pc=(4, 5),
                 pm=(1, 10), order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST, migrate_every: int = 10,
                 seed: int = 1, instance_id: int = 0, stream=None, prev: "Population" = None):
        self.inst = inst
        island = min(island, P)
        self.P, self.island = P, island
        self.nisl = P // island
        self.mach_mode = mach_mode
        par = ga_params(P, island, tour_k, pc, pm, order_mode, mach_mode, migrate_every, seed, instance_id,
                        _stream_ptr(stream))
        h = C.c_void_p()
        if prev is None:
            _check(lib().ga_population_create(inst.handle, C.byref(par), C.byref(h)), "ga_population_create")
        else:
            _check(lib().ga_population_create_warm(inst.handle, C.byref(par), prev._h, C.byref(h)),
                   "ga_population_create_warm")
        self._h = h
        self.K = inst.K

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ga_population_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, generations: int, want_schedule: bool = True) -> dict:
        inf = self.inst.info()
        S = np.zeros((inf["n_jobs"], inf["n_stages"]), np.int32)
        M = np.zeros_like(S)
        r = Result_c(0, 0, 0, 0, _p(S) if want_schedule else None, _p(M) if want_schedule else None)
        _check(lib().ga_run(self._h, int(generations), C.byref(r)), "ga_run")
        out = dict(obj=int(r.objective), tard=int(r.total_tardiness), cmax=int(r.makespan))
        if want_schedule:
            out.update(S=S, M=M)
        return out

    def read(self) -> dict:
        P, K, n = self.P, self.K, self.nisl
        d = dict(Y=np.zeros((P, K), np.int16), X=np.zeros((P, K), np.int8), obj=np.zeros(P, np.int64),
                 fit=np.zeros(P, np.int64), bY=np.zeros((n, K), np.int16), bX=np.zeros((n, K), np.int8),
                 bobj=np.zeros(n, np.int64), bfit=np.zeros(n, np.int64))
        emax = C.c_int64()
        gen = C.c_int32()
        _check(lib().ga_population_read(self._h, *[d[k].ctypes.data for k in
                                                   ("Y", "X", "obj", "fit", "bY", "bX", "bobj", "bfit")],
                                        C.addressof(emax), C.addressof(gen)), "ga_population_read")
        d["emax"] = int(emax.value)
        d["gen"] = int(gen.value)
        return d

    def attach_surrogate(self, sur, oversample: int = 8, lr: float = 1e-3, train_steps: int = 1,
                         pretrain_steps: int = 0, screen: float = 1.0, keep: int = KEEP_SLOT):
        """Surrogate-assisted generations from now on (None detaches); optionally first
        trains the surrogate on the current population.  ``keep``: KEEP_SLOT (per-slot
        screening with probability ``screen``) or KEEP_ISLAND (each island keeps the
        best-scored 1/oversample of its candidates)."""
        if sur is not None and pretrain_steps > 0:
            loss = C.c_float()
            _check(lib().ffs_surrogate_pretrain(sur._h, self._h, int(pretrain_steps), float(lr), C.addressof(loss)),
                   "ffs_surrogate_pretrain")
        _check(lib().ga_population_attach_surrogate(self._h, sur._h if sur is not None else None, int(oversample),
                                                    float(lr), int(train_steps), int(round(screen * 1000))),
               "ga_population_attach_surrogate")
        if sur is not None:
            _check(lib().ga_population_surrogate_keep(self._h, int(keep)), "ga_population_surrogate_keep")
        self._sur = sur

    def candidates(self, oversample: int) -> dict:
        """The last surrogate-assisted generation's candidates (Y, X [P*F, K]), their scores
        and, under KEEP_ISLAND, the row kept for each slot."""
        n = self.P * oversample
        d = dict(Y=np.zeros((n, self.K), np.int16), X=np.zeros((n, self.K), np.int8),
                 score=np.zeros(n, np.float32), keep=np.zeros(self.P, np.int32))
        _check(lib().ga_population_read_candidates(self._h, d["Y"].ctypes.data, d["X"].ctypes.data,
                                                   d["score"].ctypes.data, d["keep"].ctypes.data),
               "ga_population_read_candidates")
        return d

    def set_profiling(self, enable):
        """False/0: untimed graph replays; True/1: eager launches, the fused kernel timed;
        2: graph replays (the normal launch mode), each replay timed."""
        mode = 1 if enable is True else (0 if enable is False else int(enable))
        _check(lib().ga_set_profiling(self._h, mode), "ga_set_profiling")

    def profile(self):
        """(summed milliseconds, launches) of the fused generation kernel while profiling."""
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().ga_profile_read(self._h, C.byref(ms), C.byref(n)), "ga_profile_read")
        return float(ms.value), int(n.value)

    def profile_phases(self) -> dict:
        """Summed milliseconds of the phases of surrogate-assisted generations while profiling."""
        ms = np.zeros(5, np.float64)
        _check(lib().ga_profile_read_phases(self._h, ms.ctypes.data), "ga_profile_read_phases")
        return dict(zip(("candidates", "scoring", "keep_rule", "exact_decode", "training"), ms.tolist()))

    def checkpoint(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().ga_checkpoint(self._h, None, C.byref(n)), "ga_checkpoint")
        buf = (C.c_char * n.value)()
        _check(lib().ga_checkpoint(self._h, buf, C.byref(n)), "ga_checkpoint")
        return bytes(buf)

    def restore(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(lib().ga_restore(self._h, buf, len(data)), "ga_restore")


class Batch:
    """Many instances' GAs advanced by one persistent launch (``ga_batch``)."""

    def __init__(self, insts, P: int, island: int = 64, tour_k: int = 2, pc=(4, 5), pm=(1, 10),
                 order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST, migrate_every: int = 10, seed: int = 1,
                 instance_id: int = 0, stream=None):
        self.insts = list(insts)
        island = min(island, P)
        self.P, self.island, self.nisl = P, island, P // island
        par = GAParams_c(P, island, tour_k, pc[0], pc[1], pm[0], pm[1], order_mode, mach_mode,
                         migrate_every, instance_id, seed, _stream_ptr(stream))
        arr = (C.c_void_p * len(self.insts))(*[i.handle.value for i in self.insts])
        h = C.c_void_p()
        _check(lib().ga_batch_create(arr, len(self.insts), C.byref(par), C.byref(h)), "ga_batch_create")
        self._h = h
        self.K = [i.K for i in self.insts]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ga_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stop(self):
        """Asks a run in progress (in another thread) to end at a generation boundary; that
        run then raises FFSError with code E_STOPPED."""
        _check(lib().ga_batch_stop(self._h), "ga_batch_stop")

    def run(self, generations: int, results: bool = False):
        if not results:
            _check(lib().ga_batch_run(self._h, int(generations), None), "ga_batch_run")
            return None
        n = len(self.insts)
        res = (Result_c * n)()
        bufs = []
        for i, inst in enumerate(self.insts):
            inf = inst.info()
            S = np.zeros((inf["n_jobs"], inf["n_stages"]), np.int32)
            M = np.zeros_like(S)
            bufs.append((S, M))
            res[i].start, res[i].machine = _p(S), _p(M)
        _check(lib().ga_batch_run(self._h, int(generations), res), "ga_batch_run")
        return [dict(obj=int(r.objective), tard=int(r.total_tardiness), cmax=int(r.makespan), S=S, M=M)
                for r, (S, M) in zip(res, bufs)]

    def read(self, index: int) -> dict:
        P, K, n = self.P, self.K[index], self.nisl
        d = dict(Y=np.zeros((P, K), np.int16), X=np.zeros((P, K), np.int8), obj=np.zeros(P, np.int64),
                 fit=np.zeros(P, np.int64), bY=np.zeros((n, K), np.int16), bX=np.zeros((n, K), np.int8),
                 bobj=np.zeros(n, np.int64), bfit=np.zeros(n, np.int64))
        emax = C.c_int64()
        gen = C.c_int32()
        _check(lib().ga_batch_read(self._h, int(index), *[d[k].ctypes.data for k in
                                                          ("Y", "X", "obj", "fit", "bY", "bX", "bobj", "bfit")],
                                   C.addressof(emax), C.addressof(gen)), "ga_batch_read")
        d["emax"] = int(emax.value)
        d["gen"] = int(gen.value)
        return d

    def tune(self, generations: int) -> dict:
        c = BatchConfig_c()
        _check(lib().ga_batch_tune(self._h, int(generations), C.byref(c)), "ga_batch_tune")
        return {n: getattr(c, n) for n, _ in BatchConfig_c._fields_}

    def config(self) -> dict:
        c = BatchConfig_c()
        _check(lib().ga_batch_get_config(self._h, C.byref(c)), "ga_batch_get_config")
        return {n: getattr(c, n) for n, _ in BatchConfig_c._fields_}

    def set_config(self, warps: int, smem_bytes: int, cluster: int = 0):
        c = BatchConfig_c(warps, smem_bytes, 0, cluster, 0.0)
        _check(lib().ga_batch_set_config(self._h, C.byref(c)), "ga_batch_set_config")


class Surrogate:
    """The learned fitness surrogate of one instance (``ffs_surrogate``)."""

    H = 256

    def __init__(self, inst: Instance, max_batch: int, seed: int = 0, stream=None):
        h = C.c_void_p()
        _check(lib().ffs_surrogate_create(inst.handle, int(max_batch), int(seed), _stream_ptr(stream), C.byref(h)),
               "ffs_surrogate_create")
        self._h = h
        self.K = inst.K
        n = C.c_int64()
        _check(lib().ffs_surrogate_param_count(self._h, C.byref(n)), "ffs_surrogate_param_count")
        self.n_params = int(n.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ffs_surrogate_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """Name -> (offset, shape) of the blocks of the parameter vector."""
        H, K = self.H, self.K
        out, off = {}, 0
        for name, shape in (("W1", (H, 3 * K)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)),
                            ("b3", (1,))):
            out[name] = (off, shape)
            off += int(np.prod(shape))
        return out

    def unpack(self, vec):
        return {k: np.asarray(vec[o:o + int(np.prod(s))]).reshape(s) for k, (o, s) in self.layout().items()}

    def pack(self, params):
        vec = np.zeros(self.n_params, np.float32)
        for k, (o, s) in self.layout().items():
            vec[o:o + int(np.prod(s))] = np.asarray(params[k], np.float32).ravel()
        return vec

    def get_params(self):
        v = np.zeros(self.n_params, np.float32)
        _check(lib().ffs_surrogate_get_params(self._h, v.ctypes.data), "ffs_surrogate_get_params")
        return v

    def set_params(self, vec):
        v = np.ascontiguousarray(vec, np.float32)
        _check(lib().ffs_surrogate_set_params(self._h, v.ctypes.data), "ffs_surrogate_set_params")

    def predict(self, y):
        import torch
        out = torch.empty(int(y.shape[0]), dtype=torch.float32, device=y.device)
        _check(lib().ffs_surrogate_predict(self._h, _dptr(y), int(y.shape[0]), _dptr(out)), "ffs_surrogate_predict")
        return out

    def gradients(self, y, obj):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        _check(lib().ffs_surrogate_gradients(self._h, _dptr(y), _dptr(obj), int(y.shape[0]), g.ctypes.data,
                                             C.addressof(loss)), "ffs_surrogate_gradients")
        return g, float(loss.value)

    def train(self, y, obj, lr: float = 1e-3) -> float:
        loss = C.c_float()
        _check(lib().ffs_surrogate_train(self._h, _dptr(y), _dptr(obj), int(y.shape[0]), float(lr),
                                         C.addressof(loss)), "ffs_surrogate_train")
        return float(loss.value)

    def score_exactly(self, on: bool = True):
        """Diagnostic: score candidates by their exact objectives (a perfect model)."""
        _check(lib().ffs_surrogate_score_exactly(self._h, 1 if on else 0), "ffs_surrogate_score_exactly")

    def activations(self, rows: int) -> dict:
        """Stored activations of the last forward pass over the surrogate's own batch: h1, h2
        [rows, 256] (BF16 values as float64), out and t [rows] (float64)."""
        h1 = np.zeros((rows, self.H), np.uint16)
        h2 = np.zeros((rows, self.H), np.uint16)
        out = np.zeros(rows, np.float32)
        t = np.zeros(rows, np.float32)
        _check(lib().ffs_surrogate_read_activations(self._h, int(rows), h1.ctypes.data, h2.ctypes.data,
                                                    out.ctypes.data, t.ctypes.data), "ffs_surrogate_read_activations")

        def widen(b):
            return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return dict(h1=widen(h1), h2=widen(h2), out=out.astype(np.float64), t=t.astype(np.float64))


class Service:
    """The rescheduling service (``ffs_service``): requests (instance, arrivals, t_now,
    generations) are queued, admitted by memory and run concurrently on the GPU by the
    library's worker thread; each instance's last population stays on the device."""

    def __init__(self, P: int, max_active: int = 8, memory_bytes: int = 8 << 30, **ga_kw):
        cfg = ServiceConfig_c(int(max_active), 0, int(memory_bytes), ga_params(P, **ga_kw))
        h = C.c_void_p()
        _check(lib().ffs_service_create(C.byref(cfg), C.byref(h)), "ffs_service_create")
        self._h = h
        self._n_ops = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ffs_service_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, inst: Instance, arrivals=None, t_now: int = 0, generations: int = 200) -> int:
        t = C.c_int64()
        if arrivals is None:
            _check(lib().ffs_service_submit(self._h, inst.handle, None, int(t_now), int(generations), C.byref(t)),
                   "ffs_service_submit")
        else:
            keep = []
            a = _arrivals_c(arrivals, keep)
            _check(lib().ffs_service_submit(self._h, inst.handle, C.byref(a), int(t_now), int(generations),
                                            C.byref(t)), "ffs_service_submit")
        return int(t.value)

    def info(self, ticket: int) -> dict:
        """State of a request without waiting."""
        i = RequestInfo_c()
        rc = lib().ffs_service_wait(self._h, int(ticket), 0, C.byref(i), None)
        if rc not in (FFS_OK, -5) and i.state != 3:
            _check(rc, "ffs_service_wait")
        return {n: getattr(i, n) for n, _ in RequestInfo_c._fields_ if n != "pad"}

    def wait(self, ticket: int, timeout_ms: int = -1, schedule: bool = True) -> dict:
        """Waits for a request; returns its info and best schedule (raises if it failed)."""
        i = RequestInfo_c()
        rc = lib().ffs_service_wait(self._h, int(ticket), int(timeout_ms), C.byref(i), None)
        _check(rc, "ffs_service_wait")
        S = np.zeros(max(i.n_ops, 1), np.int32)
        M = np.zeros_like(S)
        r = Result_c(0, 0, 0, 0, _p(S) if schedule else None, _p(M) if schedule else None)
        _check(lib().ffs_service_wait(self._h, int(ticket), 0, None, C.byref(r)), "ffs_service_wait")
        out = {n: getattr(i, n) for n, _ in RequestInfo_c._fields_ if n != "pad"}
        out.update(obj=int(r.objective), tard=int(r.total_tardiness), cmax=int(r.makespan))
        if schedule:
            out.update(S=S[:i.n_ops], M=M[:i.n_ops])
        return out

    def stop(self, ticket: int):
        """Ends a request early (ffs_service_stop_request)."""
        _check(lib().ffs_service_stop_request(self._h, int(ticket)), "ffs_service_stop_request")

    def forget(self, inst: Instance):
        _check(lib().ffs_service_forget(self._h, inst.handle), "ffs_service_forget")

    def stats(self) -> dict:
        s = ServiceStats_c()
        _check(lib().ffs_service_stats_read(self._h, C.byref(s)), "ffs_service_stats_read")
        return {n: getattr(s, n) for n, _ in ServiceStats_c._fields_ if n != "pad"}
