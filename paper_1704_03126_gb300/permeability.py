"""Apparent and intrinsic gas permeability of a porous medium (Sec. III).

* k_a = sqrt(4/pi) Q Kn, normalised by H^2 (Eq. k_a), from a converged solve: the library's
  dvm_flowrate returns it beside Q.
* k_inf, the intrinsic permeability, is the apparent permeability in the limit Kn -> 0 (Sec. III).
  The DVM cannot run at Kn = 0 (delta = sqrt(pi)/(2 Kn) is unbounded), so k_inf is extrapolated from
  the smallest Knudsen numbers solved: in the slip regime k_a = k_inf + b Kn + c Kn^2 + ...
  (first-order slip gives the linear term), and a polynomial in Kn through those points, of degree
  one less than their number (two at most), is evaluated at Kn = 0.  For the plane channel the limit
  is H^2 / 12.  Near the continuum the mean free path shrinks below the cell size; the upwind sweep
  resolves the flow only while delta dx stays below about one, so these solves run on the same
  staircase refined `fit_refine` times, with a Gauss-Hermite velocity grid (the near-equilibrium
  distribution needs no velocities beyond |v| ~ 4 and no resolution of discontinuities).
* H* = H sqrt(12 k_inf / phi) and Kn* = Kn H / H* = Kn sqrt(phi / (12 k_inf)) (Sec. III), phi the
  porosity; for the plane channel (phi = 1, k_inf = 1/12) Kn* = Kn.

`permeability_curve` runs the fit points of one medium as one batch on the GPU and the curve points
as another (the sweep, moments, projection and stopping test are the library's kernels); only the
three-point fit and the two formulas above run on the host.
"""
from __future__ import annotations

import math

import numpy as np

from .inputs import refine_mask


def apparent_permeability(q: float, kn: float) -> float:
    """k_a = sqrt(4/pi) Q Kn (Eq. k_a)."""
    return math.sqrt(4.0 / math.pi) * q * kn


def intrinsic_permeability(kns, kas, degree: int | None = None) -> float:
    """k_inf: the polynomial in Kn through (or, with more points than degree + 1, least squares over)
    the pairs (Kn, k_a), evaluated at Kn = 0.  degree defaults to min(len - 1, 2)."""
    kns = np.asarray(kns, dtype=np.float64)
    kas = np.asarray(kas, dtype=np.float64)
    if kns.shape != kas.shape or kns.ndim != 1 or len(kns) < 2:
        raise ValueError("need at least two (Kn, k_a) pairs")
    if np.any(kns <= 0.0) or len(set(kns.tolist())) != len(kns):
        raise ValueError("Knudsen numbers must be positive and distinct")
    if degree is None:
        degree = min(len(kns) - 1, 2)
    if not 1 <= degree <= len(kns) - 1:
        raise ValueError("degree must be between 1 and the number of points - 1")
    coef = np.polynomial.polynomial.polyfit(kns, kas, degree)
    return float(coef[0])


def characteristic_length(k_inf: float, phi: float, H: float = 1.0) -> float:
    """H* = H sqrt(12 k_inf / phi) (Sec. III)."""
    if not (k_inf > 0.0 and 0.0 < phi <= 1.0):
        raise ValueError("need k_inf > 0 and 0 < phi <= 1")
    return H * math.sqrt(12.0 * k_inf / phi)


def equivalent_knudsen(kn, k_inf: float, phi: float):
    """Kn* = Kn sqrt(phi / (12 k_inf)) (Sec. III); kn may be a scalar or an array."""
    return np.asarray(kn, dtype=np.float64) / characteristic_length(k_inf, phi)


def solve_batch(masks, kns, quad, precision="fp32", tol=None, max_iter=200000, schedule="autotune", stream=None,
                anderson=0):
    """Force-driven flow through each (mask, Kn) pair (both axes periodic, H = 1), all advanced as one
    batch on the GPU from h = 0 until every stopping test passes (anderson > 0: mixed iterates of that
    depth).  Returns (k_a, iterations, status) lists in the order of the pairs."""
    from . import dvm

    if tol is None:
        tol = 1e-10 if precision == "fp64" else 1e-6
    sols = [dvm.Solver(m, True, True, kn=k, quad=quad, precision=precision, stream=stream, anderson=anderson)
            for m, k in zip(masks, kns)]
    batch = dvm.Batch(sols)
    try:
        if schedule == "autotune":
            batch.autotune(3)
            for s in sols:
                s.reset()
        status = [int(x) for x in batch.run(tol=tol, max_iter=max_iter)]
        ka = [s.flowrate()[1] for s in sols]
        iters = [s.info()["iterations"] for s in sols]
    finally:
        batch.close()
        for s in sols:
            s.close()
    return ka, iters, status


def curve_from_values(kns, kas, fit_kns, fit_kas, phi):
    """k_inf from the fit points, then H*, Kn* and k_a / k_inf of the curve points."""
    k_inf = intrinsic_permeability(fit_kns, fit_kas)
    return {
        "kn": [float(k) for k in kns], "k_a": [float(k) for k in kas],
        "fit_kn": [float(k) for k in fit_kns], "fit_k_a": [float(k) for k in fit_kas],
        "k_inf": k_inf, "phi": float(phi), "H_star": characteristic_length(k_inf, phi),
        "kn_star": equivalent_knudsen(kns, k_inf, phi).tolist(),
        "k_a_over_k_inf": [float(k) / k_inf for k in kas],
    }


def permeability_curve(mask, kns, fit_kns=(0.005, 0.01, 0.02), quad=("cubic", 32, 4.0),
                       fit_quad=("gh", 12, 0.0), fit_refine=2, precision="fp32", porosity=None, tol=None,
                       max_iter=200000, schedule="autotune", stream=None, anderson=0):
    """k_a(Kn), k_inf and k_a / k_inf against Kn* for the force-driven flow through one periodic medium.

    mask: uint8 [ny][nx], both axes periodic, height H = 1.  kns: the Knudsen numbers of the curve,
    solved on `mask` with `quad`; fit_kns: the small ones k_inf is extrapolated from, solved on the
    mask refined `fit_refine` times with `fit_quad`.  Each set runs as one batch (`dvm.Batch`; the
    sweep kernel picked by the library's autotuner unless schedule is "none").  Returns a dict with
    the Knudsen numbers, k_a, k_inf, phi, H*, Kn*, the ratios and the solves' iterations and statuses.
    anderson: depth of the mixed iteration for every solve (0 = plain).
    """
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    phi = float(1.0 - mask.mean()) if porosity is None else float(porosity)
    kns = sorted(float(k) for k in kns)
    fit = sorted(float(k) for k in fit_kns)
    fine = refine_mask(mask, fit_refine) if fit_refine > 1 else mask
    fka, fit_iters, fit_status = solve_batch([fine] * len(fit), fit, fit_quad, precision, tol, max_iter, schedule,
                                             stream, anderson)
    ka, iters, status = solve_batch([mask] * len(kns), kns, quad, precision, tol, max_iter, schedule, stream,
                                    anderson)
    out = curve_from_values(kns, ka, fit, fka, phi)
    out["iterations"] = {f"{k:g}": i for k, i in zip(fit + kns, fit_iters + iters)}
    out["status"] = {f"{k:g}": s for k, s in zip(fit + kns, fit_status + status)}
    return out
