"""Plain FP64 CPU oracle for the DVM solution of the steady linearized BGK equation.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA path: the arithmetic lives
in ``dvm_oracle.c`` (compiled here with gcc) and in ``dense.py`` (a direct linear solve of the same
discrete equations for tiny grids).

Paper: Lindsay, Su, Liu & Wu, "Comparative study of the discrete velocity and lattice Boltzmann
methods for rarefied gas flows through irregular channels", arXiv:1704.03126, Sec. II.A (DVM,
Eqs. BGK, diffuse2, nonuniform_v, iteration) and Sec. III (Q and k_a for Poiseuille flow).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvm_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENOCONV, ORC_ENUMERIC = 0, 1, 2, 4, 6

_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("dx", ctypes.c_double),
        ("mask", ctypes.c_void_p), ("delta", ctypes.c_void_p),
        ("nv", ctypes.c_int), ("xv", ctypes.c_void_p), ("wv", ctypes.c_void_p),
        ("alpha", ctypes.c_double), ("force", ctypes.c_double), ("top_u", ctypes.c_double),
        ("dy", ctypes.c_void_p), ("collision", ctypes.c_int),
    ]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("eps", ctypes.c_double), ("est", ctypes.c_double),
                ("c_shift", ctypes.c_double), ("Q", ctypes.c_double)]


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.orc_quad_gauss_hermite.argtypes = [ctypes.c_int, P, P]
        lib.orc_quad_newton_cotes.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
        lib.orc_quad_cubic.argtypes = [ctypes.c_int, P, P]
        lib.orc_solve.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, ctypes.c_int, P,
                                  ctypes.c_double, P, P, P, P, P, ctypes.POINTER(_Result)]
        lib.orc_sweep_selected.argtypes = [ctypes.POINTER(_Problem), P, ctypes.c_double, P,
                                           ctypes.c_int, P]
        lib.orc_adjoint.argtypes = [ctypes.POINTER(_Problem), P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, P, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int)]
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def quadrature(kind: str, n: int, vmax: float = 5.0):
    """1D nodes and weights (weights approximate int g exp(-x^2)/sqrt(pi) dx).

    kind: "gh" Gauss-Hermite, "nc" closed trapezoid on [-vmax, vmax], "cubic" Eq. (nonuniform_v).
    """
    x = np.zeros(n)
    w = np.zeros(n)
    lib = _lib()
    if kind == "gh":
        st = lib.orc_quad_gauss_hermite(n, _ptr(x), _ptr(w))
    elif kind == "nc":
        st = lib.orc_quad_newton_cotes(n, float(vmax), _ptr(x), _ptr(w))
    elif kind == "cubic":
        st = lib.orc_quad_cubic(n, _ptr(x), _ptr(w))
    else:
        raise ValueError(f"unknown quadrature kind {kind!r}")
    if st != ORC_OK:
        raise ValueError(f"quadrature {kind} n={n} rejected (status {st})")
    return x, w


@dataclass
class Problem:
    """A discrete problem: solid mask [ny][nx], periodicity, per-cell delta, 1D velocity rule."""

    mask: np.ndarray
    periodic_x: bool
    periodic_y: bool
    delta: np.ndarray           # [ny][nx]
    xv: np.ndarray
    wv: np.ndarray
    alpha: float = 1.0
    force: float = 1.0
    ly: float = 1.0
    top_u: float = 0.0          # speed of the plate beyond the last row (Couette flow), 0 = at rest
    dy: np.ndarray = None       # row heights [ny] (x2 spacing), or None for square cells ly / ny
    dx1: float = None           # x1 spacing when dy is given
    # "projection": L = delta psi . G^{-1} m, the projection onto the collision invariants in the
    # quadrature inner product (default); "literal": Eq. BGK as printed, delta [rho + 2 u.v + tau (|v|^2 - 1)]
    # with the quadrature moments.  They agree for a quadrature exact on psi_i psi_j f_eq.
    collision: str = "projection"

    @staticmethod
    def make(mask, periodic_x, periodic_y, delta, quad=("gh", 8, 5.0), alpha=1.0, force=1.0, ly=1.0, top_u=0.0,
             dy=None, dx1=None, collision="projection"):
        """dy: row heights (then ly = sum dy and dx1, the x1 spacing, must be given)."""
        if collision not in ("projection", "literal"):
            raise ValueError(f"unknown collision reading {collision!r}")
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        ny, nx = mask.shape
        d = np.broadcast_to(np.asarray(delta, dtype=np.float64), (ny, nx))
        kind, n = quad[0], quad[1]
        vmax = quad[2] if len(quad) > 2 else 5.0
        xv, wv = quadrature(kind, n, vmax)
        if top_u != 0.0 and periodic_y:
            raise ValueError("a moving top plate needs a non-periodic x2 axis")
        if dy is not None:
            dy = np.ascontiguousarray(dy, dtype=np.float64)
            if dy.shape != (ny,) or not np.all(dy > 0) or dx1 is None or not dx1 > 0:
                raise ValueError("dy needs ny positive row heights and a positive x1 spacing dx1")
            ly = float(dy.sum())
            dx1 = float(dx1)
        return Problem(mask, bool(periodic_x), bool(periodic_y), np.ascontiguousarray(d), xv, wv,
                       float(alpha), float(force), float(ly), float(top_u), dy, dx1, collision)

    @property
    def nx(self):
        return self.mask.shape[1]

    @property
    def ny(self):
        return self.mask.shape[0]

    @property
    def nv(self):
        return len(self.xv)

    @property
    def dx(self):
        """x1 spacing (the square cell size ly / ny unless row heights are given)."""
        return self.dx1 if self.dy is not None else self.ly / self.ny

    def row_heights(self):
        return self.dy if self.dy is not None else np.full(self.ny, self.dx)

    def velocities(self):
        """Tensor-product table: v1[k], v2[k], W[k] with k = a*nv + b."""
        v1 = np.repeat(self.xv, self.nv)
        v2 = np.tile(self.xv, self.nv)
        W = np.outer(self.wv, self.wv).ravel()
        return v1, v2, W

    def _c(self):
        self._keep = (self.mask, self.delta, self.xv, self.wv, self.dy)
        return _Problem(self.nx, self.ny, int(self.periodic_x), int(self.periodic_y), self.dx,
                        self.mask.ctypes.data, self.delta.ctypes.data, self.nv,
                        self.xv.ctypes.data, self.wv.ctypes.data, self.alpha, self.force, self.top_u,
                        self.dy.ctypes.data if self.dy is not None else None,
                        1 if self.collision == "literal" else 0)


def delta_from_kn(kn: float) -> float:
    """delta = sqrt(pi) / (2 Kn), the coefficient of the BGK operator (Eq. BGK); Kn = inf -> 0."""
    return 0.0 if math.isinf(kn) else math.sqrt(math.pi) / (2.0 * kn)


def solve(prob: Problem, tol: float = 1e-10, max_iter: int = 100000, h0=None, c0: float = 0.0,
          inplace: bool = False):
    """Source iteration (Eq. iteration) to the stopping rule; returns a dict of results.

    h0: starting state [K][ny][nx] (zeros when None); with inplace=True it is advanced in place."""
    K = prob.nv * prob.nv
    if h0 is None:
        h = np.zeros((K, prob.ny, prob.nx))
    elif inplace:
        h = h0
        if h.dtype != np.float64 or not h.flags.c_contiguous or h.shape != (K, prob.ny, prob.nx):
            raise ValueError("in-place state must be a C-contiguous float64 array [K][ny][nx]")
    else:
        h = np.array(h0, dtype=np.float64, copy=True)
    rho, u1, u2, tau = (np.zeros((prob.ny, prob.nx)) for _ in range(4))
    eps_hist = np.zeros(max_iter)
    res = _Result()
    pc = prob._c()
    st = _lib().orc_solve(ctypes.byref(pc), tol, max_iter, _ptr(h), c0, _ptr(rho), _ptr(u1),
                          _ptr(u2), _ptr(tau), _ptr(eps_hist), ctypes.byref(res))
    if st == ORC_EINVAL:
        raise ValueError("oracle rejected the problem")
    if st == ORC_ENOMEM:
        raise MemoryError("oracle out of memory")
    return dict(h=h, rho=rho, u1=u1, u2=u2, tau=tau, Q=res.Q, c=res.c_shift, iters=res.iters,
                eps=res.eps, est=res.est, eps_hist=eps_hist[:res.iters], converged=(st == ORC_OK),
                status=st)


def sweep_selected(prob: Problem, h_in: np.ndarray, c_shift: float, ks):
    """One sweep of the listed velocities from the full state h_in (no projection)."""
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    h_in = np.ascontiguousarray(h_in, dtype=np.float64)
    out = np.zeros((len(ks), prob.ny, prob.nx))
    pc = prob._c()
    st = _lib().orc_sweep_selected(ctypes.byref(pc), _ptr(h_in), c_shift, _ptr(ks), len(ks), _ptr(out))
    if st != ORC_OK:
        raise ValueError(f"orc_sweep_selected status {st}")
    return out


def adjoint(prob: Problem, h: np.ndarray, c_shift: float, tol: float = 1e-10, max_iter: int = 100000):
    """Adjoint of the projected iteration: (dQ/d delta [ny][nx], Q identity value, iterations)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    grad = np.zeros((prob.ny, prob.nx))
    q_id = ctypes.c_double(0.0)
    iters = ctypes.c_int(0)
    pc = prob._c()
    st = _lib().orc_adjoint(ctypes.byref(pc), _ptr(h), c_shift, tol, max_iter, _ptr(grad),
                            ctypes.byref(q_id), ctypes.byref(iters))
    if st == ORC_EINVAL:
        raise ValueError("oracle rejected the adjoint problem")
    return grad, q_id.value, iters.value, st == ORC_OK


def flow_rate(prob: Problem, u1: np.ndarray) -> float:
    """Q = sum_gas u1 dA / Lx (Sec. III), dA = dx dy_j."""
    gas = prob.mask == 0
    dA = prob.dx * prob.row_heights()[:, None] * np.ones((1, prob.nx))
    return float((u1 * dA)[gas].sum() / (prob.nx * prob.dx))
