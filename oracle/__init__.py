"""CPU oracle for the EDFFS decoder and hybrid GA (arXiv 1903.10741).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The product
(``paper_1903_10741_gb300``) never does.  The arithmetic lives in ``ffs_oracle.c``
(plain single-threaded C); this module compiles it with gcc and marshals arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libffs_oracle.so")
_lock = threading.Lock()
_lib = None

ST_FREE, ST_EXEC, ST_DONE, ST_FIXED = 0, 1, 2, 3
ORDER_TOPO, ORDER_STAGE, ORDER_GIVEN = 0, 1, 2
MACH_GENE, MACH_EARLIEST = 0, 1
PLACE_INSERT = 4  # or-ed into the machine mode: back-fill machine idle gaps

_i32p = C.POINTER(C.c_int32)


class _Inst(C.Structure):
    _fields_ = [("N", C.c_int32), ("g", C.c_int32), ("Qmax", C.c_int32), ("WT", C.c_int32),
                ("RS", C.c_int32), ("o", _i32p), ("p", _i32p), ("q", _i32p), ("R", _i32p),
                ("D", _i32p), ("status", _i32p), ("S0", _i32p), ("M0", _i32p), ("pm", _i32p),
                ("qm", _i32p)]


class _Eval(C.Structure):
    _fields_ = [("obj", C.c_int64), ("tard", C.c_int64), ("cmax", C.c_int32),
                ("err", C.c_int32), ("probes", C.c_int64), ("span", C.c_int64),
                ("slots", C.c_int64)]


class _GAParams(C.Structure):
    _fields_ = [("P", C.c_int32), ("I", C.c_int32), ("tour_k", C.c_int32),
                ("pc_num", C.c_int32), ("pc_den", C.c_int32), ("pm_num", C.c_int32),
                ("pm_den", C.c_int32), ("order_mode", C.c_int32), ("mach_mode", C.c_int32),
                ("migrate_every", C.c_int32), ("instance_id", C.c_int32), ("pad", C.c_int32),
                ("seed", C.c_uint64)]


class _GAState(C.Structure):
    _fields_ = [("Y", C.c_void_p), ("X", C.c_void_p), ("obj", C.c_void_p), ("fit", C.c_void_p),
                ("bY", C.c_void_p), ("bX", C.c_void_p), ("bobj", C.c_void_p), ("bfit", C.c_void_p),
                ("emax", C.c_int64), ("gen", C.c_int32), ("K", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile ffs_oracle.c into a shared library (gcc, -O2, no tuning flags)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                               "-Wno-unused-function", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_draw.restype = C.c_uint32
        L.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_classify.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, C.c_int32, _i32p]
        L.orc_classify_static.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, C.c_int32, _i32p]
        L.orc_gene_count.restype = C.c_int32
        L.orc_gene_count.argtypes = [C.POINTER(_Inst)]
        L.orc_gene_map.argtypes = [C.POINTER(_Inst), _i32p, _i32p]
        L.orc_decode.restype = C.c_int32
        L.orc_decode.argtypes = [C.POINTER(_Inst), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, _i32p, _i32p, C.POINTER(_Eval)]
        L.orc_objective.restype = C.c_int64
        L.orc_objective.argtypes = [C.c_int32, _i32p, _i32p, C.c_int32, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int32)]
        L.orc_correct.argtypes = [C.c_int32, C.c_void_p]
        L.orc_crossover.argtypes = [C.c_int32] + [C.c_void_p] * 4 + [C.c_int32, C.c_int32] + [C.c_void_p] * 4
        L.orc_mutate.argtypes = [C.c_int32, _i32p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]
        L.orc_order.argtypes = [C.POINTER(_Inst), C.c_int32, C.c_void_p, C.c_void_p, _i32p]
        _i64p = C.POINTER(C.c_int64)
        L.orc_island_best_worst.argtypes = [_i64p, C.c_int32, C.c_int32, _i32p, _i32p]
        L.orc_tournament.restype = C.c_int32
        L.orc_tournament.argtypes = [_i64p, _i32p, C.c_int32]
        L.orc_l5_cells.argtypes = [C.c_int32, C.c_int32, _i32p]
        L.orc_select.restype = C.c_int32
        L.orc_select.argtypes = [_i64p, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, C.c_int32,
                                 C.c_int32]
        L.orc_island_replace.argtypes = [C.c_int32, C.c_int32, C.c_int32] + [C.c_void_p] * 8
        L.orc_migrate.argtypes = [C.c_int32, C.c_int32, C.c_int32] + [C.c_void_p] * 4
        L.orc_candidates.restype = C.c_int32
        L.orc_candidates.argtypes = [C.POINTER(_Inst), C.POINTER(_GAParams), C.POINTER(_GAState), C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_ga_init.restype = C.c_int32
        L.orc_ga_init.argtypes = [C.POINTER(_Inst), C.POINTER(_GAParams), C.POINTER(_GAState)]
        L.orc_ga_init_from.restype = C.c_int32
        L.orc_ga_init_from.argtypes = [C.POINTER(_Inst), C.POINTER(_GAParams), C.POINTER(_GAState)]
        L.orc_ga_step.restype = C.c_int32
        L.orc_ga_step.argtypes = [C.POINTER(_Inst), C.POINTER(_GAParams), C.POINTER(_GAState)]
        _lib = L
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


def _ptr(a):
    return None if a is None else a.ctypes.data


# ------------------------------------------------------------------ Philox

def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def draw(seed: int, purpose: int, instance: int, gen: int, slot: int, d: int) -> int:
    return int(lib().orc_draw(seed, purpose, instance, gen, slot, d))


# ------------------------------------------------------------------ instance

class Instance:
    """An EDFFS instance at a rescheduling point, with the committed plan of frozen ops."""

    def __init__(self, problem):
        self.o = np.ascontiguousarray(problem.o, dtype=np.int32)
        self.p = np.ascontiguousarray(problem.p, dtype=np.int32)
        self.q = np.ascontiguousarray(problem.q, dtype=np.int32)
        self.R = np.ascontiguousarray(problem.R, dtype=np.int32)
        self.D = np.ascontiguousarray(problem.D, dtype=np.int32)
        self.Qmax = int(problem.Qmax)
        self.WT = int(problem.WT)
        self.RS = 0
        # unrelated machines (Table 2): P_jsm and Q_jsm per job and global machine, or None
        pm, qm = getattr(problem, "pm", None), getattr(problem, "qm", None)
        self.pm = None if pm is None else np.ascontiguousarray(pm, dtype=np.int32)
        self.qm = None if qm is None else np.ascontiguousarray(qm, dtype=np.int32)
        N, g = self.p.shape
        self.status = np.zeros((N, g), dtype=np.int32)
        self.S0 = np.zeros((N, g), dtype=np.int32)
        self.M0 = np.zeros((N, g), dtype=np.int32)

    @property
    def N(self):
        return int(self.p.shape[0])

    @property
    def g(self):
        return int(self.p.shape[1])

    def _c(self) -> _Inst:
        for name in ("p", "status", "S0", "M0"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), dtype=np.int32))
        s = _Inst(self.N, self.g, self.Qmax, self.WT, self.RS, _p32(self.o), _p32(self.p),
                  _p32(self.q), _p32(self.R), _p32(self.D), _p32(self.status), _p32(self.S0),
                  _p32(self.M0), None if self.pm is None else _p32(self.pm),
                  None if self.qm is None else _p32(self.qm))
        return s

    @property
    def moff(self):
        return np.concatenate([[0], np.cumsum(self.o)]).astype(np.int64)

    def plan_durations(self):
        """[N, g] duration of every op on its committed machine (P_jsm of M0)."""
        if self.pm is None:
            return self.p
        mg = self.moff[:-1][None, :] + self.M0
        return np.take_along_axis(self.pm, mg, axis=1).astype(np.int32)

    def plan_powers(self):
        """[N, g] power of every op on its committed machine."""
        mg = self.moff[:-1][None, :] + self.M0
        if self.qm is None:
            return self.q[mg]
        return np.take_along_axis(self.qm, mg, axis=1).astype(np.int32)

    @property
    def K(self) -> int:
        c = self._c()
        return int(lib().orc_gene_count(C.byref(c)))

    def gene_map(self):
        K = self.K
        gj = np.zeros(max(K, 1), dtype=np.int32)
        gs = np.zeros(max(K, 1), dtype=np.int32)
        c = self._c()
        lib().orc_gene_map(C.byref(c), _p32(gj), _p32(gs))
        return gj[:K], gs[:K]

    def gene_machines(self) -> np.ndarray:
        _, gs = self.gene_map()
        return self.o[gs]

    def decode(self, y, x=None, order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST, given=None):
        y = np.ascontiguousarray(y, dtype=np.int16)
        K = self.K
        x = np.zeros(K, dtype=np.int8) if x is None else np.ascontiguousarray(x, dtype=np.int8)
        gv = None if given is None else np.ascontiguousarray(given, dtype=np.int32)
        S = np.zeros((self.N, self.g), dtype=np.int32)
        M = np.zeros((self.N, self.g), dtype=np.int32)
        ev = _Eval()
        c = self._c()
        rc = lib().orc_decode(C.byref(c), order_mode, mach_mode, _ptr(y), _ptr(x), _ptr(gv),
                              _p32(S), _p32(M), C.byref(ev))
        if rc != 0:
            raise ValueError(f"oracle decode rejected the chromosome (code {rc})")
        return dict(S=S, M=M, obj=int(ev.obj), tard=int(ev.tard), cmax=int(ev.cmax),
                    probes=int(ev.probes), span=int(ev.span), slots=int(ev.slots))

    def order(self, y, order_mode=ORDER_STAGE, given=None) -> np.ndarray:
        """Z of Alg. 1: the genes in the order the decoder assigns them."""
        y = np.ascontiguousarray(y, dtype=np.int16)
        K = self.K
        gv = None if given is None else np.ascontiguousarray(given, dtype=np.int32)
        out = np.zeros(max(K, 1), dtype=np.int32)
        c = self._c()
        lib().orc_order(C.byref(c), order_mode, _ptr(y), _ptr(gv), _p32(out))
        return out[:K]

    def commit(self, S, M):
        """Make (S, M) the plan being executed."""
        self.S0 = np.ascontiguousarray(S, dtype=np.int32).copy()
        self.M0 = np.ascontiguousarray(M, dtype=np.int32).copy()

    def reschedule(self, arrivals, t_now: int, static: bool = False):
        """Freeze at t_now using the committed plan (Alg. 1), append the new jobs.  With
        ``static``, the traditional static approach: every op of the plan not yet completed
        keeps its start and machine, and only the new jobs are scheduled."""
        if t_now < self.RS:
            raise ValueError("t_now must not precede the previous rescheduling point")
        st = np.zeros_like(self.status)
        fn = lib().orc_classify_static if static else lib().orc_classify
        dur = np.ascontiguousarray(self.plan_durations(), dtype=np.int32)
        fn(self.N, self.g, _p32(dur), _p32(self.S0), int(t_now), _p32(st))
        n = arrivals.n
        g = self.g
        self.status = np.concatenate([st, np.zeros((n, g), np.int32)])
        self.S0 = np.concatenate([self.S0, np.zeros((n, g), np.int32)])
        self.M0 = np.concatenate([self.M0, np.zeros((n, g), np.int32)])
        self.p = np.concatenate([self.p, arrivals.p.astype(np.int32)])
        if self.pm is not None:
            self.pm = np.concatenate([self.pm, np.asarray(arrivals.pm, np.int32)])
        if self.qm is not None:
            self.qm = np.concatenate([self.qm, np.asarray(arrivals.qm, np.int32)])
        self.R = np.concatenate([self.R, arrivals.R.astype(np.int32)])
        self.D = np.concatenate([self.D, arrivals.D.astype(np.int32)])
        self.RS = int(t_now)


def objective(C_j, D, WT):
    C_j = np.ascontiguousarray(C_j, dtype=np.int32)
    D = np.ascontiguousarray(D, dtype=np.int32)
    t = C.c_int64()
    cm = C.c_int32()
    obj = lib().orc_objective(len(C_j), _p32(C_j), _p32(D), int(WT), C.byref(t), C.byref(cm))
    return int(obj), int(t.value), int(cm.value)


def correct(y):
    y = np.ascontiguousarray(y, dtype=np.int16).copy()
    lib().orc_correct(len(y), _ptr(y))
    return y


def crossover(ya, xa, yb, xb, cx, cy):
    K = len(ya)
    ya, yb = (np.ascontiguousarray(v, dtype=np.int16) for v in (ya, yb))
    xa, xb = (np.ascontiguousarray(v, dtype=np.int8) for v in (xa, xb))
    y0, y1 = np.zeros(K, np.int16), np.zeros(K, np.int16)
    x0, x1 = np.zeros(K, np.int8), np.zeros(K, np.int8)
    lib().orc_crossover(K, _ptr(ya), _ptr(xa), _ptr(yb), _ptr(xb), int(cx), int(cy),
                        _ptr(y0), _ptr(x0), _ptr(y1), _ptr(x1))
    return y0, x0, y1, x1


def mutate(y, x, gene_o, xr, a, b):
    y = np.ascontiguousarray(y, dtype=np.int16).copy()
    x = np.ascontiguousarray(x, dtype=np.int8).copy()
    go = np.ascontiguousarray(gene_o, dtype=np.int32)
    xr = np.ascontiguousarray(xr, dtype=np.uint32)
    lib().orc_mutate(len(y), _p32(go), _ptr(y), _ptr(x), _ptr(xr), int(a), int(b))
    return y, x


# ------------------------------------------------------------------ GA operators (Sec. 4.4)

def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def island_best_worst(fit, lo: int, hi: int):
    """(best, worst) of fit[lo:hi]: largest / smallest fitness, lowest index among equals."""
    f = _i64(fit)
    b, w = C.c_int32(), C.c_int32()
    lib().orc_island_best_worst(f.ctypes.data_as(C.POINTER(C.c_int64)), lo, hi, C.byref(b), C.byref(w))
    return int(b.value), int(w.value)


def tournament(fit, entrants) -> int:
    """Winner among the entrant indices: largest fitness, ties to the lowest index."""
    f = _i64(fit)
    e = np.ascontiguousarray(entrants, dtype=np.int32)
    return int(lib().orc_tournament(f.ctypes.data_as(C.POINTER(C.c_int64)), _p32(e), len(e)))


def l5_cells(P: int, i: int):
    """Cell i and its N, S, W, E neighbours on the sqrt(P) x sqrt(P) torus."""
    out = np.zeros(5, np.int32)
    lib().orc_l5_cells(P, i, _p32(out))
    return out.tolist()


def select(fit, P: int, I: int, tour_k: int, seed: int, instance: int, gen: int, slot: int) -> int:
    """The parent the GA selects for `slot` at generation `gen`."""
    f = _i64(fit)
    return int(lib().orc_select(f.ctypes.data_as(C.POINTER(C.c_int64)), P, I, tour_k, seed, instance, gen, slot))


def island_replace(cY, cX, cobj, cfit, lo: int, I: int, bY, bX, bobj: int, bfit: int):
    """Elitist replacement of the island at slots lo..lo+I.  Returns the updated children
    (Y, X, obj, fit) and best-ever record (bY, bX, bobj, bfit) as new arrays."""
    cY = np.ascontiguousarray(cY, dtype=np.int16).copy()
    cX = np.ascontiguousarray(cX, dtype=np.int8).copy()
    cobj, cfit = _i64(cobj).copy(), _i64(cfit).copy()
    bY = np.ascontiguousarray(bY, dtype=np.int16).copy()
    bX = np.ascontiguousarray(bX, dtype=np.int8).copy()
    bo, bf = np.array([bobj], np.int64), np.array([bfit], np.int64)
    lib().orc_island_replace(cY.shape[1], lo, I, _ptr(cY), _ptr(cX), _ptr(cobj), _ptr(cfit), _ptr(bY), _ptr(bX),
                             _ptr(bo), _ptr(bf))
    return cY, cX, cobj, cfit, bY, bX, int(bo[0]), int(bf[0])


def migrate(cY, cX, cobj, cfit, I: int):
    """Single-ring migration over the islands of I slots; returns new arrays."""
    cY = np.ascontiguousarray(cY, dtype=np.int16).copy()
    cX = np.ascontiguousarray(cX, dtype=np.int8).copy()
    cobj, cfit = _i64(cobj).copy(), _i64(cfit).copy()
    lib().orc_migrate(cY.shape[1], I, len(cfit) // I, _ptr(cY), _ptr(cX), _ptr(cobj), _ptr(cfit))
    return cY, cX, cobj, cfit


# ------------------------------------------------------------------ GA

class GA:
    """The hybrid GA run on the CPU, one generation at a time."""

    def __init__(self, inst: Instance, P: int, island: int = 64, tour_k: int = 2,
                 pc=(4, 5), pm=(1, 10), order_mode=ORDER_STAGE, mach_mode=MACH_EARLIEST,
                 migrate_every: int = 10, seed: int = 1, instance_id: int = 0):
        self.inst = inst
        island = min(island, P)
        self.par = _GAParams(P, island, tour_k, pc[0], pc[1], pm[0], pm[1], order_mode,
                             mach_mode, migrate_every, instance_id, 0, seed)
        K = inst.K
        self.K = K
        nisl = P // island
        self.Y = np.zeros((P, max(K, 1)), np.int16)
        self.X = np.zeros((P, max(K, 1)), np.int8)
        self.obj = np.zeros(P, np.int64)
        self.fit = np.zeros(P, np.int64)
        self.bY = np.zeros((nisl, max(K, 1)), np.int16)
        self.bX = np.zeros((nisl, max(K, 1)), np.int8)
        self.bobj = np.zeros(nisl, np.int64)
        self.bfit = np.zeros(nisl, np.int64)
        self.st = _GAState(self.Y.ctypes.data, self.X.ctypes.data, self.obj.ctypes.data,
                           self.fit.ctypes.data, self.bY.ctypes.data, self.bX.ctypes.data,
                           self.bobj.ctypes.data, self.bfit.ctypes.data, 0, 0, K)
        self._inst_c = None

    def _ic(self):
        self._inst_c = self.inst._c()
        return self._inst_c

    def init(self):
        rc = lib().orc_ga_init(C.byref(self._ic()), C.byref(self.par), C.byref(self.st))
        if rc:
            raise RuntimeError(f"oracle GA init failed ({rc})")
        return self

    def init_from(self, Y, X=None):
        """Generation 0 from given rows (a warm start) instead of random ones."""
        P = self.Y.shape[0]
        self.Y[:, :self.K] = np.asarray(Y, dtype=np.int16).reshape(P, self.K)
        self.X[:, :self.K] = 0 if X is None else np.asarray(X, dtype=np.int8).reshape(P, self.K)
        rc = lib().orc_ga_init_from(C.byref(self._ic()), C.byref(self.par), C.byref(self.st))
        if rc:
            raise RuntimeError(f"oracle GA init failed ({rc})")
        return self

    def step(self, n: int = 1):
        for _ in range(n):
            rc = lib().orc_ga_step(C.byref(self._ic()), C.byref(self.par), C.byref(self.st))
            if rc:
                raise RuntimeError(f"oracle GA step failed ({rc})")
        return self

    def candidates(self, F: int):
        """The P*F offspring the next generation would build, F per slot (row f P + j is
        candidate f of slot j; F = 1 gives the children of `step`), and whether crossover or
        mutation changed each row."""
        P, K = self.Y.shape[0], self.K
        cY = np.zeros((P * F, max(K, 1)), np.int16)
        cX = np.zeros((P * F, max(K, 1)), np.int8)
        cnew = np.zeros(P * F, np.uint8)
        lib().orc_candidates(C.byref(self._ic()), C.byref(self.par), C.byref(self.st), int(F), cY.ctypes.data,
                             cX.ctypes.data, cnew.ctypes.data)
        return cY[:, :K], cX[:, :K], cnew

    @property
    def gen(self):
        return int(self.st.gen)

    @property
    def emax(self):
        return int(self.st.emax)

    def best(self):
        """Best-ever individual over all islands (largest fitness, lowest island)."""
        i = int(np.argmax(self.bfit))
        return self.bY[i, :self.K].copy(), self.bX[i, :self.K].copy(), int(self.bobj[i])


# ------------------------------------------------------------------ warm start

def gene_keys(inst: Instance) -> np.ndarray:
    """Identity of each gene across rescheduling points: job * g + stage (jobs only append)."""
    gj, gs = inst.gene_map()
    return gj.astype(np.int64) * inst.g + gs


def warm_remap(Y_old, X_old, keys_old, keys_new, P_new):
    """Warm-start population for a rescheduled instance (not in the paper, which restarts
    its GA at every rescheduling point, Sec. 4.1).

    Row r of the result comes from old row r mod P_old.  A gene present before and after
    keeps its machine gene, and the surviving genes keep their relative priority order,
    taking the top priorities n_new+1 .. K_new (ascending old priority -> ascending new
    one).  The n_new genes that did not exist before (operations of new jobs) take the
    priorities below them, n_new .. 1, in ascending gene index, with machine gene 0.
    """
    Y_old = np.asarray(Y_old)
    X_old = np.asarray(X_old)
    keys_old = list(np.asarray(keys_old).tolist())
    keys_new = list(np.asarray(keys_new).tolist())
    pos_old = {k: i for i, k in enumerate(keys_old)}
    surv = [i for i, k in enumerate(keys_new) if k in pos_old]
    fresh = [i for i, k in enumerate(keys_new) if k not in pos_old]
    n_new, K_new = len(fresh), len(keys_new)
    src = np.array([pos_old[keys_new[i]] for i in surv], dtype=np.int64)
    Y = np.zeros((P_new, K_new), np.int16)
    X = np.zeros((P_new, K_new), np.int8)
    for r in range(P_new):
        yo, xo = Y_old[r % len(Y_old)], X_old[r % len(X_old)]
        order = np.argsort(yo[src], kind="stable")          # survivors by old priority, ascending
        for rank, t in enumerate(order):
            Y[r, surv[t]] = n_new + 1 + rank
            X[r, surv[t]] = xo[src[t]]
        for q, i in enumerate(fresh):
            Y[r, i] = n_new - q
    return Y, X
