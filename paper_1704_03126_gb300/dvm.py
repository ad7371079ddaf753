"""ctypes binding of libdvm (include/dvm.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels.  Loading fails loudly when libdvm.so is
missing or no CUDA device is present; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdvm.so")

DVM_OK, DVM_EINVAL, DVM_ENOMEM, DVM_ECUDA, DVM_ENOCONV, DVM_ETIMEOUT, DVM_ENUMERIC, DVM_ESTATE = range(8)
PAIRING = {"auto": 0, "on": 1, "off": 2}  # dvm_pairing
QUAD_KINDS = {"gh": 0, "nc": 1, "cubic": 2}
STORAGE = {"auto": 0, "as_given": 1, "transposed": 2}
FP64, FP32_ACC64 = 0, 1


class DvmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_STATUS_NAMES = {0: "DVM_OK", 1: "DVM_EINVAL", 2: "DVM_ENOMEM", 3: "DVM_ECUDA", 4: "DVM_ENOCONV",
                 5: "DVM_ETIMEOUT", 6: "DVM_ENUMERIC", 7: "DVM_ESTATE"}


class Quad(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("vmax", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("ly", ctypes.c_double), ("kn", ctypes.c_double), ("delta", ctypes.c_double),
        ("quad", Quad), ("accommodation", ctypes.c_double), ("precision", ctypes.c_int),
        ("force", ctypes.c_double), ("store_distribution", ctypes.c_int), ("sweep_warps", ctypes.c_int),
        ("top_wall_u1", ctypes.c_double), ("storage", ctypes.c_int),
        ("dx1", ctypes.c_double), ("row_heights", ctypes.c_void_p), ("anderson_depth", ctypes.c_int),
        ("fp32_refine", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("eps", ctypes.c_double), ("est", ctypes.c_double),
                ("mass_shift", ctypes.c_double), ("Q", ctypes.c_double), ("status", ctypes.c_int),
                ("transposed", ctypes.c_int)]


_lib = None


def lib():
    """Load libdvm.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdvm.so not found at {LIB_PATH}; build it first (python -c "
                               "'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.dvm_params_init.argtypes = [ctypes.POINTER(Params)]
        L.dvm_create.argtypes = [P, ctypes.POINTER(Params), P, ctypes.POINTER(P)]
        L.dvm_set_delta_field.argtypes = [P, P]
        L.dvm_reset.argtypes = [P]
        L.dvm_solve.argtypes = [P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.dvm_iterate.argtypes = [P, I]
        L.dvm_flowrate.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.dvm_fields.argtypes = [P, P, P, P, P]
        L.dvm_get_info.argtypes = [P, ctypes.POINTER(Info)]
        L.dvm_distribution.argtypes = [P, P, I, P]
        L.dvm_quadrature.argtypes = [P, P, P]
        L.dvm_batch_solve.argtypes = [P, I, D, I, P]
        L.dvm_velocity_grid.argtypes = [ctypes.POINTER(Quad), P, P]
        L.dvm_batch_create.argtypes = [P, I, ctypes.POINTER(P)]
        L.dvm_batch_run.argtypes = [P, D, I, P]
        L.dvm_batch_iterate.argtypes = [P, I]
        L.dvm_batch_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
        L.dvm_batch_kernels_per_sweep.argtypes = [P]
        L.dvm_batch_kernels_per_sweep.restype = I
        L.dvm_batch_destroy.argtypes = [P]
        L.dvm_moments.argtypes = [ctypes.POINTER(Quad), P, P, I, D, P, P, P]
        L.dvm_adjoint.argtypes = [P, D, I, P, ctypes.POINTER(D), ctypes.POINTER(I)]
        L.dvm_moments_noalloc.argtypes = [ctypes.POINTER(Quad), P, P, I, D, P, P, P]
        L.dvm_last_error.argtypes = [P]
        L.dvm_last_error.restype = ctypes.c_char_p
        L.dvm_status_string.argtypes = [I]
        L.dvm_status_string.restype = ctypes.c_char_p
        L.dvm_destroy.argtypes = [P]
        L.dvm_batch_enqueue.argtypes = [P, I]
        L.dvm_batch_check.argtypes = [P]
        L.dvm_set_schedule.argtypes = [P, I, I]
        L.dvm_get_schedule.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
        L.dvm_batch_set_schedule.argtypes = [P, I, I]
        L.dvm_batch_get_schedule.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
        L.dvm_batch_autotune.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]
        L.dvm_selftest_wait.argtypes = [I, I, ctypes.POINTER(D)]
        L.dvm_probe_peaks.argtypes = [I, D, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(I)]
        L.dvm_batch_set_persistent.argtypes = [P, I]
        L.dvm_batch_get_persistent.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
        L.dvm_batch_set_pairing.argtypes = [P, I]
        L.dvm_batch_get_pairing.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
        for name in ("dvm_params_init", "dvm_create", "dvm_set_delta_field", "dvm_reset", "dvm_solve",
                     "dvm_iterate", "dvm_flowrate", "dvm_fields", "dvm_get_info", "dvm_distribution",
                     "dvm_quadrature", "dvm_batch_solve", "dvm_velocity_grid", "dvm_batch_create",
                     "dvm_batch_run", "dvm_batch_iterate", "dvm_batch_timing", "dvm_moments",
                     "dvm_moments_noalloc", "dvm_adjoint", "dvm_set_schedule", "dvm_get_schedule",
                     "dvm_batch_set_schedule", "dvm_batch_get_schedule", "dvm_batch_autotune",
                     "dvm_batch_enqueue", "dvm_batch_check", "dvm_selftest_wait", "dvm_probe_peaks",
                     "dvm_batch_set_persistent", "dvm_batch_get_persistent", "dvm_batch_set_pairing",
                     "dvm_batch_get_pairing"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Solver:
    """One geometry: wraps a dvm_ctx.

    mask: uint8 [ny][nx] (1 = solid); quad = (kind, n, vmax) with kind in {"gh", "nc", "cubic"};
    exactly one of kn (> 0, inf allowed) and delta (>= 0).  stream: a cudaStream_t as int (e.g.
    torch.cuda.current_stream().cuda_stream) or None.  schedule: None (automatic), or (kind,
    shape) for set_schedule.  accommodation: alpha in [0, 1] of Eq. (diffuse2); below 1 the
    walls reflect the rest specularly (column sweep only; no adjoint).  top_wall_u1: speed of the plate
    beyond the last row (Couette flow; column sweep only).  storage: "auto" (the library
    stores a grid wider than tall transposed, so that its sweeps walk the long axis), "as_given" or
    "transposed"; arguments and results keep the [ny][nx] layout either way.  dx1: x1 spacing (0 = square
    cells ly / ny); row_heights: [ny] heights of the rows along x2 (ly becomes their sum; needs dx1 > 0,
    runs on the column sweep, stored transposed; no adjoint).  anderson: depth of the Anderson mixing of
    the source iteration (0 = plain; 1..8; FP64 storage and accommodation 1 only).  refine: FP32 storage,
    the most passes of mixed-precision refinement after the FP32 iteration (None = the library's default,
    3; 0 = off; see dvm_params.fp32_refine).
    """

    def __init__(self, mask, periodic_x=True, periodic_y=False, kn=None, delta=None, quad=("gh", 12, 5.0),
                 precision="fp64", ly=1.0, force=1.0, store_distribution=False, sweep_warps=0, stream=None,
                 schedule=None, accommodation=1.0, top_wall_u1=0.0, storage="auto", dx1=0.0, row_heights=None,
                 anderson=0, refine=None):
        L = lib()
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self.mask = mask
        p = Params()
        L.dvm_params_init(ctypes.byref(p))
        p.ny, p.nx = mask.shape
        p.periodic_x = int(bool(periodic_x))
        p.periodic_y = int(bool(periodic_y))
        p.ly = float(ly)
        if (kn is None) == (delta is None):
            raise ValueError("give exactly one of kn and delta")
        p.kn = float(kn) if kn is not None else -1.0
        p.delta = float(delta) if delta is not None else -1.0
        p.quad.kind = QUAD_KINDS[quad[0]]
        p.quad.n = int(quad[1])
        p.quad.vmax = float(quad[2]) if len(quad) > 2 else 5.0
        p.precision = {"fp64": FP64, "fp32": FP32_ACC64}[precision]
        p.force = float(force)
        p.accommodation = float(accommodation)
        p.top_wall_u1 = float(top_wall_u1)
        if storage not in STORAGE:
            raise ValueError(f"storage must be one of {sorted(STORAGE)}")
        p.storage = STORAGE[storage]
        p.dx1 = float(dx1)
        p.anderson_depth = int(anderson)
        if refine is not None:
            p.fp32_refine = int(refine)
        rows = None
        if row_heights is not None:
            rows = np.ascontiguousarray(row_heights, dtype=np.float64)
            if rows.shape != (mask.shape[0],):
                raise ValueError("row_heights must have one entry per row")
            p.row_heights = rows.ctypes.data
        self._row_heights = rows  # keeps the array that params points to alive
        p.store_distribution = int(bool(store_distribution))
        p.sweep_warps = int(sweep_warps)
        self.params = p
        self.nv = p.quad.n
        # bumped by every call that changes the state (delta field, reset, sweeps): autograd checks it
        self.state_id = 0
        self.last_adjoint_status = None
        self._ctx = ctypes.c_void_p()
        st = L.dvm_create(_ptr(mask), ctypes.byref(p), ctypes.c_void_p(stream or 0), ctypes.byref(self._ctx))
        if st != DVM_OK:
            raise DvmError(st, L.dvm_last_error(None).decode())
        if schedule is not None:
            self.set_schedule(*schedule)

    def _check(self, st, allow=(DVM_OK,)):
        if st not in allow:
            raise DvmError(st, lib().dvm_last_error(self._ctx).decode())
        return st

    @property
    def shape(self):
        return self.mask.shape

    def set_delta_field(self, delta_c):
        self.state_id += 1
        if delta_c is None:
            return self._check(lib().dvm_set_delta_field(self._ctx, None))
        d = np.ascontiguousarray(delta_c, dtype=np.float64)
        assert d.shape == self.shape
        return self._check(lib().dvm_set_delta_field(self._ctx, _ptr(d)))

    def reset(self):
        self.state_id += 1
        return self._check(lib().dvm_reset(self._ctx))

    def set_schedule(self, kind="auto", shape=0):
        """Sweep kernel of this solver: "rows" (shape = chunk width 1..16, 0 = auto), "columns" (shape =
        threads per column 1, 2, 4, 0 = auto) or "auto"."""
        return self._check(lib().dvm_set_schedule(self._ctx, SWEEP_KINDS[kind], int(shape)))

    def schedule(self):
        k, v = ctypes.c_int(), ctypes.c_int()
        self._check(lib().dvm_get_schedule(self._ctx, ctypes.byref(k), ctypes.byref(v)))
        return SWEEP_NAMES[k.value], v.value

    def solve(self, tol=1e-10, max_iter=100000, raise_on_noconv=True):
        """Returns (status, sweeps run, error estimate)."""
        it = ctypes.c_int(0)
        est = ctypes.c_double(0.0)
        self.state_id += 1
        st = lib().dvm_solve(self._ctx, float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(est))
        self._check(st, (DVM_OK,) if raise_on_noconv else (DVM_OK, DVM_ENOCONV))
        return st, it.value, est.value

    def iterate(self, n):
        self.state_id += 1
        return self._check(lib().dvm_iterate(self._ctx, int(n)))

    def flowrate(self):
        q = ctypes.c_double()
        ka = ctypes.c_double()
        self._check(lib().dvm_flowrate(self._ctx, ctypes.byref(q), ctypes.byref(ka)))
        return q.value, ka.value

    def fields(self):
        out = {k: np.empty(self.shape) for k in ("rho", "u1", "u2", "tau")}
        self._check(lib().dvm_fields(self._ctx, _ptr(out["rho"]), _ptr(out["u1"]), _ptr(out["u2"]), _ptr(out["tau"])))
        return out

    def info(self):
        inf = Info()
        self._check(lib().dvm_get_info(self._ctx, ctypes.byref(inf)))
        return dict(iterations=inf.iterations, eps=inf.eps, est=inf.est, mass_shift=inf.mass_shift, Q=inf.Q,
                    status=inf.status, transposed=bool(inf.transposed))

    def adjoint(self, tol=1e-10, max_iter=100000):
        """dQ/d delta_c at the current forward state: (grad [ny][nx], F sum z v1, adjoint sweeps).

        An adjoint iteration that ran out of sweeps (DVM_ENOCONV) still returns its last gradient; the
        status is kept in last_adjoint_status (DVM_OK or DVM_ENOCONV)."""
        g = np.empty(self.shape)
        qid = ctypes.c_double()
        it = ctypes.c_int()
        st = lib().dvm_adjoint(self._ctx, float(tol), int(max_iter), _ptr(g), ctypes.byref(qid), ctypes.byref(it))
        self._check(st, (DVM_OK, DVM_ENOCONV))
        self.last_adjoint_status = st
        return g, qid.value, it.value

    def distribution(self, ks):
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        out = np.empty((len(ks),) + self.shape)
        self._check(lib().dvm_distribution(self._ctx, _ptr(ks), len(ks), _ptr(out)))
        return out

    def quadrature(self):
        x = np.empty(self.nv)
        w = np.empty(self.nv)
        self._check(lib().dvm_quadrature(self._ctx, _ptr(x), _ptr(w)))
        return x, w

    def close(self):
        if self._ctx:
            lib().dvm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        # at interpreter shutdown the CUDA runtime may already be torn down; the process exit frees all
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


SWEEP_KINDS = {"auto": 0, "rows": 1, "columns": 2}
SWEEP_NAMES = {v: k for k, v in SWEEP_KINDS.items()}


class Batch:
    """Several Solvers advanced by one launch of each kernel per sweep (dvm_batch_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._ctx.value for s in self.solvers])
        self._b = ctypes.c_void_p()
        st = lib().dvm_batch_create(arr, len(self.solvers), ctypes.byref(self._b))
        if st != DVM_OK:
            raise DvmError(st, lib().dvm_last_error(self.solvers[0]._ctx).decode())

    def _err(self, st):
        raise DvmError(st, lib().dvm_last_error(self.solvers[0]._ctx).decode())

    def _touch(self):
        for s in self.solvers:
            s.state_id += 1

    def run(self, tol=1e-10, max_iter=100000):
        per = np.zeros(len(self.solvers), dtype=np.int32)
        self._touch()
        st = lib().dvm_batch_run(self._b, float(tol), int(max_iter), _ptr(per))
        if st not in (DVM_OK, DVM_ENOCONV):
            self._err(st)
        return per

    def iterate(self, n=1):
        self._touch()
        st = lib().dvm_batch_iterate(self._b, int(n))
        if st != DVM_OK:
            self._err(st)

    def enqueue(self, n=1):
        """n sweeps of every member, enqueued without waiting (see check)."""
        self._touch()
        st = lib().dvm_batch_enqueue(self._b, int(n))
        if st != DVM_OK:
            self._err(st)

    def check(self):
        """Wait for the enqueued sweeps; raises on a failed member."""
        st = lib().dvm_batch_check(self._b)
        if st != DVM_OK:
            self._err(st)

    def timing(self):
        """(sweep_ms, finalize_ms) of the last single sweep."""
        a = ctypes.c_float()
        f = ctypes.c_float()
        st = lib().dvm_batch_timing(self._b, ctypes.byref(a), ctypes.byref(f))
        if st != DVM_OK:
            self._err(st)
        return a.value, f.value

    def kernels_per_sweep(self):
        return lib().dvm_batch_kernels_per_sweep(self._b)

    def set_schedule(self, kind="auto", shape=0):
        st = lib().dvm_batch_set_schedule(self._b, SWEEP_KINDS[kind], int(shape))
        if st != DVM_OK:
            self._err(st)

    def schedule(self):
        k, v = ctypes.c_int(), ctypes.c_int()
        st = lib().dvm_batch_get_schedule(self._b, ctypes.byref(k), ctypes.byref(v))
        if st != DVM_OK:
            self._err(st)
        return SWEEP_NAMES[k.value], v.value

    def set_persistent(self, on=True):
        """One persistent launch per up to 64 sweeps with a device-side scheduler (row sweep only); see
        dvm_batch_set_persistent."""
        self._touch()
        st = lib().dvm_batch_set_persistent(self._b, int(bool(on)))
        if st != DVM_OK:
            self._err(st)

    def persistent(self):
        """(on, blocks of the persistent launch)."""
        on, blocks = ctypes.c_int(), ctypes.c_int()
        st = lib().dvm_batch_get_persistent(self._b, ctypes.byref(on), ctypes.byref(blocks))
        if st != DVM_OK:
            self._err(st)
        return bool(on.value), blocks.value

    def set_pairing(self, mode):
        """Paired velocity groups in the FP32 row sweep: "auto", "on" or "off" (dvm_batch_set_pairing)."""
        self._touch()
        st = lib().dvm_batch_set_pairing(self._b, PAIRING[mode])
        if st != DVM_OK:
            self._err(st)

    def pairing(self):
        """(mode, sweep blocks of the planned launch that sweep paired groups)."""
        mode, blocks = ctypes.c_int(), ctypes.c_int()
        st = lib().dvm_batch_get_pairing(self._b, ctypes.byref(mode), ctypes.byref(blocks))
        if st != DVM_OK:
            self._err(st)
        return {v: k for k, v in PAIRING.items()}[mode.value], blocks.value

    def autotune(self, sweeps=5):
        """Time every fitting sweep kernel (the trial sweeps advance the state); keeps the fastest.
        Returns (kind, shape, median sweep ms); shape is the chunk width for "rows"."""
        k, v, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._touch()
        st = lib().dvm_batch_autotune(self._b, int(sweeps), ctypes.byref(k), ctypes.byref(v), ctypes.byref(ms))
        if st != DVM_OK:
            self._err(st)
        return SWEEP_NAMES[k.value], v.value, ms.value

    def close(self):
        if self._b:
            lib().dvm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        # at interpreter shutdown the CUDA runtime may already be torn down; the process exit frees all
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def batch_solve(solvers, tol=1e-10, max_iter=100000):
    """Solve several Solvers in one batched launch per sweep; returns the per-instance statuses."""
    n = len(solvers)
    arr = (ctypes.c_void_p * n)(*[s._ctx.value for s in solvers])
    per = np.zeros(n, dtype=np.int32)
    for s in solvers:
        s.state_id += 1
    st = lib().dvm_batch_solve(arr, n, float(tol), int(max_iter), _ptr(per))
    if st not in (DVM_OK, DVM_ENOCONV):
        raise DvmError(st, lib().dvm_last_error(solvers[0]._ctx).decode())
    return per


def selftest_wait(primitive: int, spin_limit: int = 0):
    """Run a sweep wait primitive (0: progress word, 1: mbarrier) on a flag nothing raises:
    (status, seconds); the expected status is DVM_ETIMEOUT."""
    sec = ctypes.c_double(0.0)
    st = lib().dvm_selftest_wait(int(primitive), int(spin_limit), ctypes.byref(sec))
    return st, sec.value


PROBE_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def probe_peaks(kind: str, seconds: float = 0.2):
    """Measured FMA rate of the current GPU (dvm_probe_peaks): (TFLOP/s, L2 bytes, SMs).
    kind: "fp32", "fp32x2" (packed pairs) or "fp64"."""
    tf = ctypes.c_double(0.0)
    l2 = ctypes.c_int(0)
    sms = ctypes.c_int(0)
    st = lib().dvm_probe_peaks(PROBE_KINDS[kind], float(seconds), ctypes.byref(tf), ctypes.byref(l2), ctypes.byref(sms))
    if st != DVM_OK:
        raise DvmError(st, "dvm_probe_peaks failed")
    return tf.value, l2.value, sms.value


def velocity_grid(kind: str, n: int, vmax: float = 5.0):
    """Library's 1D nodes and weights (host only, no GPU needed)."""
    q = Quad(QUAD_KINDS[kind], int(n), float(vmax))
    x = np.empty(n)
    w = np.empty(n)
    st = lib().dvm_velocity_grid(ctypes.byref(q), _ptr(x), _ptr(w))
    if st != DVM_OK:
        raise DvmError(st, lib().dvm_last_error(None).decode())
    return x, w


def moments(h_ptr, ncell, quad, mom_ptr, q_ptr, dA_over_L, mask_ptr=None, stream=None, noalloc=False):
    """dvm_moments (or dvm_moments_noalloc) on device pointers (ints, e.g. torch data_ptr()):
    h [n*n][ncell] FP64 -> mom [ncell][4], Q [1]."""
    q = Quad(QUAD_KINDS[quad[0]], int(quad[1]), float(quad[2]) if len(quad) > 2 else 5.0)
    fn = lib().dvm_moments_noalloc if noalloc else lib().dvm_moments
    st = fn(ctypes.byref(q), ctypes.c_void_p(h_ptr), ctypes.c_void_p(mask_ptr or 0), int(ncell),
            float(dA_over_L), ctypes.c_void_p(mom_ptr), ctypes.c_void_p(q_ptr), ctypes.c_void_p(stream or 0))
    if st != DVM_OK:
        raise DvmError(st, lib().dvm_last_error(None).decode() or "dvm_moments failed")


def kn_to_delta(kn: float) -> float:
    return 0.0 if math.isinf(kn) else math.sqrt(math.pi) / (2.0 * kn)
