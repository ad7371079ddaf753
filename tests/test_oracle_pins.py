"""Pins for the CPU oracle: closed forms, library routines, a second solution route, invariants.

None of these re-types the oracle's own formulas: each compares it with something the paper or the
mathematics fixes independently.
  * Gauss-Hermite rule          vs numpy.polynomial.hermite.hermgauss (library routine)
  * quadrature moment sums      vs erf closed forms
  * free-molecular plates       vs the exact discrete solution h = v1 d / |v2| (stencil exact on lines)
  * continuum limit             vs Q = delta/12 + sigma_P/2 with the published BGK slip coefficient
  * iterative fixed point       vs a direct dense LAPACK solve of the same discrete equations
  * adjoint gradient            vs the dense transposed solve and central finite differences
  * symmetry and conservation   mirror symmetries of symmetric geometries, zero mass shift for
                                exact quadrature
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1704_03126_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature (Sec. II.A)

@pytest.mark.parametrize("n", [2, 4, 8, 12, 16, 24, 32, 48])
def test_gauss_hermite_matches_numpy(n):
    x, w = oracle.quadrature("gh", n)
    xr, wr = np.polynomial.hermite.hermgauss(n)
    assert np.max(np.abs(x - xr)) < 1e-12 * max(1.0, np.abs(xr).max())
    assert np.max(np.abs(w - wr / math.sqrt(math.pi))) < 1e-14


def test_newton_cotes_moments_match_erf():
    x, w = oracle.quadrature("nc", 32, 5.0)
    assert np.allclose(x, np.linspace(-5, 5, 32), atol=1e-15, rtol=0)
    # exact truncated moments of exp(-x^2)/sqrt(pi) on [-5, 5]
    m0 = math.erf(5.0)
    m2 = 0.5 * math.erf(5.0) - 5.0 * math.exp(-25.0) / math.sqrt(math.pi)
    # trapezoid error (Euler-Maclaurin, first term): h^2/12 (f'(5) - f'(-5))
    hstep = 10.0 / 31.0
    fp = lambda t: -2.0 * t * math.exp(-t * t) / math.sqrt(math.pi)
    fp2 = lambda t: (2.0 * t - 2.0 * t ** 3) * math.exp(-t * t) / math.sqrt(math.pi)
    assert abs(w.sum() - (m0 + hstep ** 2 / 12.0 * (fp(5.0) - fp(-5.0)))) < 5e-13
    assert abs((w * x * x).sum() - (m2 + hstep ** 2 / 12.0 * (fp2(5.0) - fp2(-5.0)))) < 2e-11


@pytest.mark.parametrize("n,tol0,tol2,tol4", [(16, 1e-4, 1e-3, 2e-3), (32, 1e-7, 1e-6, 2e-5),
                                            (48, 1e-7, 1e-6, 2e-5)])
def test_cubic_grid_nodes_and_moments(n, tol0, tol2, tol4):
    x, w = oracle.quadrature("cubic", n)
    # Eq. (nonuniform_v): extreme nodes at +-4, symmetric, clustered at 0
    assert abs(x[-1] - 4.0) < 1e-14 and abs(x[0] + 4.0) < 1e-14
    assert np.allclose(x, -x[::-1], atol=1e-15)
    assert abs(x[n // 2]) < 4.0 / (n - 1) ** 3 * 1.0000001
    # moments 1, 1/2, 3/4 of exp(-x^2)/sqrt(pi); the rule is a trapezoid in s of a smooth
    # integrand truncated at |v| = 4 (erfc(4) ~ 1.5e-8), so the defects shrink quickly with n
    assert abs(w.sum() - 1.0) < tol0
    assert abs((w * x * x).sum() - 0.5) < tol2
    assert abs((w * x ** 4).sum() - 0.75) < tol4


# ---------------------------------------------------------------- free-molecular plates

@pytest.mark.parametrize("quad", [("gh", 12, 0.0), ("nc", 32, 5.0)])
def test_free_molecular_plates_exact(quad):
    """delta = 0 between diffuse plates: v2 dh/dy = v1 with h = 0 at the wall the molecule left
    (rho_w = 0 by oddness in v1), so h = v1 d / |v2| with d the distance from that wall; the
    second-order upwind stencils (interior, one- and two-point wall forms) are exact on it."""
    ny = 32
    p = oracle.Problem.make(inputs.plates_mask(4, ny), True, False, 0.0, quad)
    # a fixed number of sweeps: the u1-based stop ends earlier, while grazing velocities still
    # carry lagged seam values around the periodic x axis
    r = oracle.solve(p, tol=0.0, max_iter=600)
    v1, v2, W = p.velocities()
    y = (np.arange(ny) + 0.5) / ny
    d = np.where(v2[:, None] > 0, y[None, :], 1.0 - y[None, :])
    h_exact = v1[:, None] * d / np.abs(v2)[:, None]
    assert np.max(np.abs(r["h"][:, :, 0] - h_exact)) < 1e-10 * np.abs(h_exact).max()
    q_exact = 0.5 * np.sum(W * v1 * v1 / np.abs(v2))
    assert abs(r["Q"] - q_exact) < 1e-11 * q_exact


# ---------------------------------------------------------------- continuum limit (Sec. III k_a)

def test_continuum_limit_slip_coefficient():
    """k_a = sqrt(4/pi) Q Kn -> 1/12 needs Q -> delta/12; the next term is sigma_P/2 (BGK slip).
    Richardson in 1/delta from delta = 10 and 20 removes the O(1/delta) term."""
    gold = json.load(open(os.path.join(GOLDEN, "bgk_slip_coefficient.json")))
    qs = {}
    for delta, ny in [(10.0, 64), (20.0, 128)]:
        p = oracle.Problem.make(inputs.plates_mask(2, ny), True, False, delta, ("gh", 16, 0.0))
        r = oracle.solve(p, tol=1e-10, max_iter=100000)
        assert r["converged"]
        qs[delta] = r["Q"] - delta / 12.0
    slip_half = 2.0 * qs[20.0] - qs[10.0]
    assert abs(slip_half - gold["value"] / 2.0) < gold["abs_uncertainty_for_test"] / 2.0
    # apparent permeability of the plates approaches H^2/12 from above
    for delta in (10.0, 20.0):
        kn = math.sqrt(math.pi) / (2 * delta)
        k_a = math.sqrt(4 / math.pi) * (qs[delta] + delta / 12.0) * kn
        assert 1.0 / 12.0 < k_a < 1.0 / 12.0 * (1.0 + 12.0 / delta)


# ---------------------------------------------------------------- dense direct solve

def _tiny_cases():
    block = np.zeros((6, 6), np.uint8)
    block[2:4, 2:4] = 1
    notch = np.zeros((8, 4), np.uint8)
    notch[0:2, 1] = 1
    notch[7, 2:4] = 1
    dvar = np.full((6, 6), 1.3)
    dvar[0, 0] = 0.4
    dvar[5, 1] = 2.6
    return [
        ("block_periodic_cubic6", block, True, True, dvar, ("cubic", 6, 4.0), 1.0),
        ("block_periodic_gh6_alpha0.6", block, True, True, 2.0, ("gh", 6, 0.0), 0.6),
        ("plates_gh8", np.zeros((8, 4), np.uint8), True, False, 0.7, ("gh", 8, 0.0), 1.0),
        ("notched_nc6", notch, True, False, 5.0, ("nc", 6, 4.0), 1.0),
        ("block_periodic_nc8_small_delta", block, True, True, 0.05, ("nc", 8, 4.0), 1.0),
    ]


@pytest.mark.parametrize("case", _tiny_cases(), ids=lambda c: c[0])
def test_iteration_matches_dense_solve(case):
    name, mask, px, py, delta, quad, alpha = case
    p = oracle.Problem.make(mask, px, py, delta, quad, alpha=alpha)
    ds = dense.solve(p)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - ds["Q"]) < 1e-11 * abs(ds["Q"])
    assert np.max(np.abs(r["h"] - ds["h"])) < 1e-10 * max(1.0, np.abs(ds["h"]).max())
    assert abs(r["c"] - ds["c"]) < 1e-11
    # the projection holds mean density at zero
    assert abs(r["rho"][mask == 0].mean()) < 1e-13


def test_dense_free_molecular_cubic_closed_form():
    """The cubic grid's grazing velocities make the lagged iteration slow at delta = 0; the direct
    solve of the same equations still reproduces Q = 1/2 sum W v1^2 / |v2| exactly."""
    p = oracle.Problem.make(inputs.plates_mask(2, 8), True, False, 0.0, ("cubic", 8, 4.0))
    ds = dense.solve(p)
    v1, v2, W = p.velocities()
    q_exact = 0.5 * np.sum(W * v1 * v1 / np.abs(v2))
    assert abs(ds["Q"] - q_exact) < 1e-10 * q_exact


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("case", _tiny_cases()[:4], ids=lambda c: c[0])
def test_adjoint_matches_dense_transpose(case):
    name, mask, px, py, delta, quad, alpha = case
    p = oracle.Problem.make(mask, px, py, delta, quad, alpha=alpha)
    ds = dense.solve(p)
    g_dense = dense.adjoint_gradient(p, ds)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_it, q_id, iters, ok = oracle.adjoint(p, r["h"], r["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_dense).max()
    assert np.max(np.abs(g_it - g_dense)) < 1e-9 * scale
    # forward/adjoint identity Q = F sum z v1
    assert abs(q_id - r["Q"]) < 1e-10 * abs(r["Q"])
    assert np.all(g_it[mask == 1] == 0.0)


def test_adjoint_matches_central_differences():
    name, mask, px, py, delta, quad, alpha = _tiny_cases()[0]
    p = oracle.Problem.make(mask, px, py, delta, quad, alpha=alpha)
    g = dense.adjoint_gradient(p)
    for (j, i) in [(0, 0), (5, 1), (1, 4), (4, 5)]:
        step = 1e-5 * p.delta[j, i]
        qs = []
        for sgn in (1, -1):
            d = p.delta.copy()
            d[j, i] += sgn * step
            qs.append(dense.solve(oracle.Problem(p.mask, px, py, d, p.xv, p.wv, alpha))["Q"])
        fd = (qs[0] - qs[1]) / (2 * step)
        assert abs(fd - g[j, i]) < 1e-6 * np.abs(g).max()


# ---------------------------------------------------------------- invariants

def test_plates_invariants_and_zero_mass_shift():
    """Plates: rho = tau = u2 = 0 (h odd in v1), x-invariance, u1 symmetric about the mid-plane;
    with Gauss-Hermite weights (exact low moments) the scheme conserves mass, so c = 0."""
    p = oracle.Problem.make(inputs.plates_mask(4, 32), True, False, oracle.delta_from_kn(0.1), ("gh", 12, 0.0))
    r = oracle.solve(p, tol=1e-12, max_iter=100000)
    assert r["converged"]
    for f in ("rho", "tau", "u2"):
        assert np.abs(r[f]).max() < 1e-12
    u1 = r["u1"]
    assert np.abs(u1 - u1[:, :1]).max() < 1e-12
    assert np.abs(u1[:, 0] - u1[::-1, 0]).max() < 1e-12
    assert abs(r["c"]) < 1e-13
    assert r["Q"] > oracle.delta_from_kn(0.1) / 12.0  # slip only adds flow


def test_rough_channel_mirror_symmetries():
    """Blocks centred in x on both walls: u1 even in x and y, u2 odd in both, rho odd in x."""
    mask = inputs.rough_channel_mask(32)
    p = oracle.Problem.make(mask, True, False, oracle.delta_from_kn(1.0), ("nc", 8, 4.0))
    r = oracle.solve(p, tol=1e-12, max_iter=100000)
    assert r["converged"]
    gas = mask == 0
    u1, u2, rho = r["u1"], r["u2"], r["rho"]
    tol = 1e-10 * np.abs(u1).max()
    assert np.abs((u1 - u1[:, ::-1])[gas]).max() < tol
    assert np.abs((u1 - u1[::-1, :])[gas]).max() < tol
    assert np.abs((u2 + u2[:, ::-1])[gas]).max() < tol
    assert np.abs((u2 + u2[::-1, :])[gas]).max() < tol
    assert np.abs((rho + rho[:, ::-1])[gas]).max() < tol


def test_porous_medium_iteration_converges():
    """Narrow pores between small disks: the iteration must converge (a near-wall stencil that puts a
    negative weight on the lagged wall value makes it diverge with an oscillating mode)."""
    mask = inputs.porous_disks_mask(48, 0.6, 4, 7, seed=3)[0]
    p = oracle.Problem.make(mask, True, True, oracle.delta_from_kn(0.5), ("cubic", 12, 4.0))
    r = oracle.solve(p, tol=1e-10, max_iter=5000)
    assert r["converged"] and r["status"] == 0
    assert np.isfinite(r["Q"]) and r["Q"] > 0
    # mass: the projection keeps the mean gas density at zero
    assert abs(r["rho"][mask == 0].mean()) < 1e-12


def test_sweep_selected_reproduces_fixed_point():
    """At convergence one more sweep of any velocity returns the same h (fixed point of Eq. iteration)."""
    mask = inputs.rough_channel_mask(16)
    p = oracle.Problem.make(mask, True, False, 2.0, ("nc", 8, 4.0))
    r = oracle.solve(p, tol=1e-14, max_iter=100000)
    ks = [0, 5, 17, 40, 63]
    out = oracle.sweep_selected(p, r["h"], r["c"], ks)
    assert np.abs(out - r["h"][ks]).max() < 1e-11 * np.abs(r["h"]).max()


# ---------------------------------------------------------------- collision operator (Sec. II.A, Eq. BGK)
#
# Eq. BGK writes the collision term as delta [rho + 2 u.v + tau (|v|^2 - 1)] with the moments of Sec.
# II.A.  The oracle (and the library) use the W-orthogonal projection of h onto span{1, v1, v2, |v|^2}
# instead; the two coincide when the quadrature integrates psi_i psi_j f_eq exactly.  These tests hold
# the literal form against the projection: equal for Gauss-Hermite, small differences on the configs'
# grids, and on inexact grids a departure from the paper's Q_s = 0.5 (Sec. II.B) that the projection
# does not have.


@pytest.mark.parametrize("case", ["block_periodic", "couette_rough"])
def test_collision_readings_coincide_for_an_exact_quadrature(case):
    """Gauss-Hermite 8 integrates polynomials of degree <= 15 against f_eq exactly, so the Gram matrix
    is that of the continuous inner product and G^{-1} m reproduces rho - tau, 2 u, tau: both readings
    give the same discrete system (dense solve) and the same fixed point (iteration)."""
    mask = np.zeros((6, 6), np.uint8)
    if case == "block_periodic":
        mask[2:4, 2:4] = 1
        kw = dict(force=1.0)
        px, py = True, True
    else:
        mask[0, 1:3] = 1
        mask[1, 2] = 1
        kw = dict(force=0.0, top_u=1.0)
        px, py = True, False
    sols = {}
    for col in ("projection", "literal"):
        p = oracle.Problem.make(mask, px, py, 1.1, ("gh", 8, 0.0), collision=col, **kw)
        sols[col] = (dense.solve(p), oracle.solve(p, tol=1e-14, max_iter=400000))
    (d0, r0), (d1, r1) = sols["projection"], sols["literal"]
    assert np.max(np.abs(d0["B"] - d1["B"])) < 1e-12
    assert abs(d0["Q"] - d1["Q"]) < 1e-12 * abs(d0["Q"])
    assert r0["converged"] and r1["converged"]
    assert abs(r0["Q"] - r1["Q"]) < 1e-12 * abs(r0["Q"])
    assert np.max(np.abs(r1["h"] - d1["h"])) < 1e-10 * max(1.0, np.abs(d1["h"]).max())


def test_literal_collision_loses_momentum_on_an_inexact_grid():
    """On the cubic grid of Eq. (nonuniform_v) (32 nodes), m0 m2 = 0.4999992 differs from 1/2.  The literal
    form then maps the uniform drift v1 to 2 m0 m2 v1, so the momentum sum of L - delta h is
    delta U (2 m0 m2 - 1) instead of 0: a spurious body force proportional to delta, which drives a
    Poiseuille-like flow of order delta^2 (2 m0 m2 - 1).  Smooth Couette plates therefore lose the
    paper's Q_s = 0.5 at every Kn (Sec. II.B) by a growing amount as Kn falls, while the projection
    keeps Q_s = U H m0 m2 exactly (measured with these solves on 32 rows: literal - m0 m2 = -1.1e-6 at
    Kn 1, -1.8e-5 at Kn 0.1 and -1.1e-3 at Kn 0.01; projection within 1e-13)."""
    x, w = oracle.quadrature("cubic", 32, 4.0)
    m0, m2 = float(w.sum()), float((w * x * x).sum())
    # the literal kernel applied to v1 is 2 m0 m2 v1 (a dense check of the operator itself)
    p = oracle.Problem.make(np.zeros((2, 2), np.uint8), True, False, 1.0, ("cubic", 32, 4.0), collision="literal")
    v1, v2, W = p.velocities()
    Ml = dense.collision_kernel(v1, v2, W, "literal")
    Mp = dense.collision_kernel(v1, v2, W, "projection")
    assert np.max(np.abs(Ml @ v1 - 2.0 * m0 * m2 * v1)) < 1e-12
    assert np.max(np.abs(Mp @ v1 - v1)) < 1e-12
    dev = {}
    for kn in (1.0, 0.1):
        for col in ("projection", "literal"):
            q = oracle.Problem.make(inputs.plates_mask(4, 32), True, False, oracle.delta_from_kn(kn), ("cubic", 32, 4.0),
                                    force=0.0, top_u=1.0, collision=col)
            r = oracle.solve(q, tol=1e-13, max_iter=400000)
            assert r["converged"]
            dev[(kn, col)] = r["Q"] - m0 * m2
    assert abs(dev[(1.0, "projection")]) < 1e-11 and abs(dev[(0.1, "projection")]) < 1e-11
    # the literal form falls below m0 m2 (and below 1/2) by more than the quadrature's own defect
    # |m0 m2 - 1/2| = 8.1e-7, and by about delta^2 more at the smaller Knudsen number
    assert dev[(1.0, "literal")] < -abs(m0 * m2 - 0.5)
    ratio = dev[(0.1, "literal")] / dev[(1.0, "literal")]
    assert 8.0 < ratio < 40.0  # measured 16.7; delta grows 10x


@pytest.mark.parametrize("case", ["rough_nc32", "porous_cubic48", "couette_cubic32"])
def test_collision_readings_on_the_configured_grids(case):
    """Both readings converge on the configs' velocity grids, and their fixed points differ by a
    grid-dependent amount: the Newton-Cotes rule is exact to about 1e-10 on the moments involved, the
    cubic rules to about 1e-6.  Measured relative differences in Q (Kn 1 here; the larger figures at
    smaller Kn are in the design notes): NC32 rough channel 1.0e-10, cubic48 porous 24 x 24 1.2e-7,
    cubic32 Couette over a WM wall 2.2e-6."""
    if case == "rough_nc32":
        mask, px, py, quad, kw, bound = inputs.rough_channel_mask(32), True, False, ("nc", 32, 5.0), {}, 1e-9
    elif case == "porous_cubic48":
        mask = inputs.porous_disks_mask(24, 0.7, 2, 4, seed=1)[0]
        px, py, quad, kw, bound = True, True, ("cubic", 48, 4.0), {}, 2e-6
    else:
        mask, ly = inputs.couette_rough_mask(24, 2.0, 0.02)
        px, py, quad, kw, bound = True, False, ("cubic", 32, 4.0), dict(ly=ly, top_u=1.0, force=0.0), 1e-5
    qs = {}
    for col in ("projection", "literal"):
        p = oracle.Problem.make(mask, px, py, oracle.delta_from_kn(1.0), quad, collision=col, **kw)
        r = oracle.solve(p, tol=1e-12, max_iter=100000)
        assert r["converged"]
        qs[col] = r["Q"]
    rel = abs(qs["projection"] - qs["literal"]) / abs(qs["projection"])
    assert rel < bound


def test_oracle_adjoint_rejects_the_literal_reading():
    """The oracle's adjoint transposes the projection; it refuses the literal reading."""
    p = oracle.Problem.make(inputs.plates_mask(4, 8), True, False, 1.0, ("gh", 6, 0.0), collision="literal")
    r = oracle.solve(p, tol=1e-12, max_iter=10000)
    with pytest.raises(ValueError):
        oracle.adjoint(p, r["h"], r["c"])


# ---------------------------------------------------------------- Couette flow (Sec. II, Eq. diffuse1)

@pytest.mark.parametrize("quad", [("gh", 8, 0.0), ("nc", 8, 4.0), ("cubic", 8, 4.0)])
@pytest.mark.parametrize("kn", [0.1, 1.0, 10.0])
def test_plane_couette_flow_rate_is_half(kn, quad):
    """Smooth plates, the top one moving with U = 1: the linearized problem with walls at (0, U) is the
    one with walls at (-U/2, U/2) plus the uniform drift 2 (U/2) v1, which the collision operator,
    the transport and the diffuse walls all leave invariant (rho_w of the drift vanishes on a
    symmetric grid); the former is odd under the mirror (x2 -> H - x2, v -> -v).  So u1 is the drift's
    U sum_k W_k v1_k^2 = U m0 m2 (m0 = sum w_a, m2 = sum w_a x_a^2 of the 1D rule) plus an odd part,
    and Q = U H m0 m2 at every Kn: the paper's Q_s = 0.5 (Sec. II) for a rule exact on x^2 (Gauss-
    Hermite), and the rule's own second moment otherwise."""
    ny = 16
    p = oracle.Problem.make(np.zeros((ny, 4), np.uint8), True, False, oracle.delta_from_kn(kn), quad,
                            force=0.0, top_u=1.0)
    m0, m2 = float(p.wv.sum()), float((p.wv * p.xv ** 2).sum())
    r = oracle.solve(p, tol=1e-13, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - m0 * m2) < 1e-10
    if quad[0] == "gh":
        gold = json.load(open(os.path.join(GOLDEN, "couette_smooth_flow_rate.json")))
        assert abs(m0 * m2 - gold["value"]) < 1e-14
        assert abs(r["Q"] - gold["value"]) < 1e-10 + gold["abs_uncertainty_for_test"]
    u1 = r["u1"][:, 0]
    assert np.max(np.abs(u1 + u1[::-1] - 2.0 * m0 * m2)) < 1e-10
    assert np.all(np.diff(u1) > 0)  # the shear profile rises towards the moving plate


@pytest.mark.parametrize("alpha", [0.5, 0.8])
def test_plane_couette_with_partially_specular_plates(alpha):
    """The uniform drift 2 (U/2) v1 is also left unchanged by specular reflection (v1 keeps its sign),
    so the argument above holds for any accommodation: Q = U H m0 m2 and the mirrored profile."""
    ny = 14
    p = oracle.Problem.make(np.zeros((ny, 3), np.uint8), True, False, oracle.delta_from_kn(0.5), ("gh", 8, 0.0),
                            alpha=alpha, force=0.0, top_u=1.0)
    m0, m2 = float(p.wv.sum()), float((p.wv * p.xv ** 2).sum())
    r = oracle.solve(p, tol=1e-13, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - m0 * m2) < 1e-10
    u1 = r["u1"][:, 0]
    assert np.max(np.abs(u1 + u1[::-1] - 2.0 * m0 * m2)) < 1e-10
    # partially specular plates drag less: the slip at each plate grows as alpha falls
    full = oracle.solve(oracle.Problem.make(np.zeros((ny, 3), np.uint8), True, False, oracle.delta_from_kn(0.5),
                                            ("gh", 8, 0.0), force=0.0, top_u=1.0), tol=1e-13, max_iter=400000)
    assert u1[0] > full["u1"][0, 0]


@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_couette_iteration_matches_dense_solve(alpha):
    """A rough bottom under a moving plate: the iteration's fixed point against the direct solve
    (the moving plate enters the dense system as a source term)."""
    mask = np.zeros((6, 6), np.uint8)
    mask[0, 1:3] = 1
    mask[1, 2] = 1
    p = oracle.Problem.make(mask, True, False, 1.2, ("gh", 6, 0.0), alpha=alpha, force=0.0, top_u=1.0)
    ds = dense.solve(p)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - ds["Q"]) < 1e-11 * abs(ds["Q"])
    assert np.max(np.abs(r["h"] - ds["h"])) < 1e-10 * max(1.0, np.abs(ds["h"]).max())


def test_couette_force_and_moving_plate_superpose():
    """The problem is linear: force-driven plus moving-plate flow rates add."""
    mask = inputs.couette_rough_mask(8, aspect=2.0, eps=0.05)[0]
    quad = ("gh", 6, 0.0)
    q = {}
    for name, force, u in (("force", 1.0, 0.0), ("plate", 0.0, 1.0), ("both", 1.0, 1.0)):
        p = oracle.Problem.make(mask, True, False, 1.0, quad, force=force, top_u=u, ly=mask.shape[0] / 8)
        q[name] = oracle.solve(p, tol=1e-13, max_iter=400000)["Q"]
    assert abs(q["both"] - q["force"] - q["plate"]) < 1e-10 * abs(q["both"])


def test_wm_roughness_has_the_requested_rms():
    mask, ly = inputs.couette_rough_mask(40, aspect=5.0, eps=0.02)
    ny, nx = mask.shape
    assert nx == 200 and abs(ly - ny / 40) < 1e-12
    # the staircase height of every column tracks base + r(x) to within a cell
    dx = 1.0 / 40
    x = (np.arange(nx) + 0.5) * dx
    r = inputs.wm_roughness(x, n_max=int(math.floor(math.log(20.0) / math.log(1.5))))
    r *= 0.02 / math.sqrt(np.mean(r * r))
    heights = mask.sum(axis=0) * dx
    base = heights.mean() - r.mean()
    assert np.max(np.abs(heights - (base + r))) <= dx
    assert mask[-1].sum() == 0  # the top rows are gas: the moving plate lies beyond the last row


def test_wm_profile_sum_against_an_independent_series():
    """Eq. (WM) as a plain loop over its terms (unit A) equals the generator's vectorised sum, and each
    term's amplitude gamma^((D - 2) n) falls with the frequency for D < 2."""
    x = np.linspace(0.0, 5.0, 37)
    ref = np.zeros_like(x)
    for n in range(-4, 7):
        ref += [math.cos(2 * math.pi * 1.5 ** n * xi) * 1.5 ** (-(2 - 1.5) * n) for xi in x]
    assert np.max(np.abs(inputs.wm_roughness(x, 1.5, 1.5, -4, 6) - ref)) < 1e-12
    assert 1.5 ** (-(2 - 1.5) * 6) < 1.5 ** (-(2 - 1.5) * -4)


def test_paper_grid_couette_generator():
    """Sec. II.A's grid: 1500 equal columns over aspect 5, 60 equal rows across the band of the zero-mean
    WM profile scaled to rms eps H, 100 equal rows above it up to the plate at x2 = H; a band cell is
    solid exactly when its centre lies below the profile, and no cell above the band is solid."""
    mask, dy, dx1 = inputs.couette_paper_grid()
    assert mask.shape == (160, 1500) and abs(dx1 - 5.0 / 1500) < 1e-15
    x = (np.arange(1500) + 0.5) * dx1
    r = inputs.wm_roughness(x, n_max=int(math.floor(math.log(1.0 / (2 * dx1)) / math.log(1.5))))
    r -= r.mean()
    r *= 0.02 / math.sqrt(np.mean(r * r))
    assert abs(math.sqrt(np.mean(r * r)) - 0.02) < 1e-15 and abs(r.mean()) < 1e-15
    lo, hi = r.min(), r.max()
    assert np.allclose(dy[:60], (hi - lo) / 60, rtol=0, atol=1e-15)
    assert np.allclose(dy[60:], (1.0 - hi) / 100, rtol=0, atol=1e-15)
    assert abs(lo + dy.sum() - 1.0) < 1e-13  # the grid spans min r .. H
    yc = lo + np.cumsum(dy) - 0.5 * dy
    assert np.array_equal(mask, (yc[:, None] < r[None, :]).astype(np.uint8))
    assert mask[60:].sum() == 0 and mask[0].sum() > 0


# ---------------------------------------------------------------- rows of unequal height (Sec. II.A grid)

def _stretched_rows(ny, seed, symmetric=False):
    """Seeded row heights in [0.4, 1.6] (relative), normalised to H = 1; mirrored when symmetric."""
    rng = inputs.SplitMix64(seed)
    h = np.array([0.4 + 1.2 * rng.uniform() for _ in range(ny)])
    if symmetric:
        h = 0.5 * (h + h[::-1])
    return h / h.sum()


@pytest.mark.parametrize("quad", [("gh", 8, 0.0), ("nc", 12, 5.0)])
def test_free_molecular_plates_exact_on_unequal_rows(quad):
    """delta = 0: h = v1 d / |v2| is linear in x2, and the unequal-row stencils (Lagrange derivatives
    through the same points) are exact on linear fields, so the discrete solution is exact on any row
    heights; Q = 1/2 sum W v1^2 / |v2| (midpoint areas integrate a linear profile exactly)."""
    ny = 24
    dy = _stretched_rows(ny, 11)
    p = oracle.Problem.make(inputs.plates_mask(4, ny), True, False, 0.0, quad, dy=dy, dx1=0.03)
    r = oracle.solve(p, tol=0.0, max_iter=600)
    v1, v2, W = p.velocities()
    y = np.cumsum(dy) - 0.5 * dy
    d = np.where(v2[:, None] > 0, y[None, :], 1.0 - y[None, :])
    h_exact = v1[:, None] * d / np.abs(v2)[:, None]
    assert np.max(np.abs(r["h"][:, :, 0] - h_exact)) < 1e-10 * np.abs(h_exact).max()
    q_exact = 0.5 * np.sum(W * v1 * v1 / np.abs(v2))
    assert abs(r["Q"] - q_exact) < 1e-11 * q_exact
    assert abs(oracle.flow_rate(p, r["u1"]) - r["Q"]) < 1e-14


def test_equal_row_heights_reproduce_square_cells():
    """Heights all equal to the x1 spacing: the general stencils reduce to the square-cell ones."""
    mask = inputs.rough_channel_mask(24)
    ny = mask.shape[0]
    a = oracle.solve(oracle.Problem.make(mask, True, False, 1.3, ("nc", 8, 4.0)), tol=1e-13, max_iter=100000)
    b = oracle.solve(oracle.Problem.make(mask, True, False, 1.3, ("nc", 8, 4.0), dy=np.full(ny, 1.0 / ny),
                                         dx1=1.0 / ny), tol=1e-13, max_iter=100000)
    assert abs(a["Q"] - b["Q"]) < 1e-12 * abs(a["Q"])
    assert np.nanmax(np.abs(a["u1"] - b["u1"])) < 1e-11


def _unequal_row_cases():
    notch = np.zeros((8, 4), np.uint8)
    notch[0:2, 1] = 1
    notch[7, 2:4] = 1
    return [
        ("plates_gh6", np.zeros((7, 3), np.uint8), True, False, 0.7, ("gh", 6, 0.0), 1.0, 0.0),
        ("notched_nc6", notch, True, False, 3.0, ("nc", 6, 4.0), 1.0, 0.0),
        ("notched_gh6_alpha0.6", notch, True, False, 1.0, ("gh", 6, 0.0), 0.6, 0.0),
        ("couette_notched_cubic6", notch, True, False, 1.5, ("cubic", 6, 4.0), 1.0, 1.0),
        ("periodic_rows_block_gh6", np.pad(np.ones((2, 2), np.uint8), 2), True, True, 2.0, ("gh", 6, 0.0), 1.0, 0.0),
    ]


@pytest.mark.parametrize("case", _unequal_row_cases(), ids=lambda c: c[0])
def test_unequal_rows_iteration_matches_dense_solve(case):
    """The iteration (closed-form Lagrange weights in C) and the dense solve (weights from a
    Vandermonde solve) reach the same fixed point on rows of unequal height."""
    name, mask, px, py, delta, quad, alpha, top_u = case
    dy = _stretched_rows(mask.shape[0], 5)
    p = oracle.Problem.make(mask, px, py, delta, quad, alpha=alpha, force=0.0 if top_u else 1.0, top_u=top_u,
                            dy=dy, dx1=0.11)
    ds = dense.solve(p)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - ds["Q"]) < 1e-11 * abs(ds["Q"])
    assert np.max(np.abs(r["h"] - ds["h"])) < 1e-10 * max(1.0, np.abs(ds["h"]).max())


@pytest.mark.parametrize("kn", [0.1, 1.0])
def test_plane_couette_on_symmetric_unequal_rows(kn):
    """Rows mirrored about the mid-plane keep the mirror symmetry of the Couette argument, so
    Q = U H m0 m2 and u1(x2) + u1(H - x2) = 2 U m0 m2 hold on them too."""
    ny = 20
    dy = _stretched_rows(ny, 3, symmetric=True)
    p = oracle.Problem.make(np.zeros((ny, 3), np.uint8), True, False, oracle.delta_from_kn(kn), ("gh", 8, 0.0),
                            force=0.0, top_u=1.0, dy=dy, dx1=0.05)
    m0, m2 = float(p.wv.sum()), float((p.wv * p.xv ** 2).sum())
    r = oracle.solve(p, tol=1e-13, max_iter=400000)
    assert r["converged"]
    assert abs(r["Q"] - m0 * m2) < 1e-10
    u1 = r["u1"][:, 0]
    assert np.max(np.abs(u1 + u1[::-1] - 2.0 * m0 * m2)) < 1e-10


def test_couette_mean_profile_integrates_to_the_flow_rate():
    """The mean streamwise profile (solid cells as zero) integrates to Q over the rows, on equal and on
    stretched rows over a notched wall; between smooth plates it is mirror-symmetric about m0 m2."""
    from paper_1704_03126_gb300 import couette
    notch = np.zeros((10, 6), np.uint8)
    notch[0:2, 2] = 1
    for dy in (None, _stretched_rows(10, 9)):
        kw = dict(dy=dy, dx1=0.1) if dy is not None else {}
        p = oracle.Problem.make(notch, True, False, 1.2, ("gh", 6, 0.0), force=0.0, top_u=1.0, **kw)
        r = oracle.solve(p, tol=1e-13, max_iter=200000)
        y, ub = couette.mean_profile(r["u1"], notch, p.ly, dy)
        assert abs(float((ub * p.row_heights()).sum()) - r["Q"]) < 1e-13
        assert np.all(np.diff(y) > 0) and abs(y[-1] + 0.5 * p.row_heights()[-1] - p.ly) < 1e-14
    p = oracle.Problem.make(np.zeros((12, 3), np.uint8), True, False, 0.8, ("gh", 8, 0.0), force=0.0, top_u=1.0)
    r = oracle.solve(p, tol=1e-13, max_iter=200000)
    y, ub = couette.mean_profile(r["u1"], p.mask)
    m0m2 = float(p.wv.sum() * (p.wv * p.xv ** 2).sum())
    assert np.max(np.abs(ub + ub[::-1] - 2 * m0m2)) < 1e-10
    assert abs(couette.profile_at(y, ub, [0.5])[0] - m0m2) < 1e-10
    assert abs(couette.q_star(0.45, 0.5) - 0.9) < 1e-15


def test_couette_adjoint_matches_dense_transpose_and_differences():
    """The moving plate only adds a constant source, so the adjoint operator is the one of a plate at
    rest: the iterative adjoint at the Couette state matches the dense transposed solve and central
    differences of dense Couette solves (the Q identity is F sum z v1 = 0 here: no force)."""
    mask = np.zeros((8, 6), np.uint8)
    mask[0:2, 2] = 1
    dfield = np.full((8, 6), 1.1)
    dfield[3, 4] = 0.6
    p = oracle.Problem.make(mask, True, False, dfield, ("gh", 6, 0.0), force=0.0, top_u=1.0)
    ds = dense.solve(p)
    g_dense = dense.adjoint_gradient(p, ds)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_it, q_id, iters, ok = oracle.adjoint(p, r["h"], r["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_dense).max()
    assert scale > 0.0
    assert np.max(np.abs(g_it - g_dense)) < 1e-9 * scale
    assert abs(q_id) < 1e-14
    for (j, i) in [(3, 4), (6, 1), (2, 3)]:
        step = 1e-5 * dfield[j, i]
        qs = []
        for sgn in (1, -1):
            d = dfield.copy()
            d[j, i] += sgn * step
            qs.append(dense.solve(oracle.Problem.make(mask, True, False, d, ("gh", 6, 0.0), force=0.0,
                                                       top_u=1.0))["Q"])
        assert abs((qs[0] - qs[1]) / (2 * step) - g_dense[j, i]) < 1e-6 * scale


@pytest.mark.parametrize("top_u", [0.0, 1.0])
def test_adjoint_on_unequal_rows_matches_dense_transpose(top_u):
    """The adjoint on rows of unequal height (the forward Lagrange weights transposed, the flow-rate
    functional weighted by the row heights) matches the dense transposed solve and central
    differences of dense solves."""
    mask = np.zeros((9, 5), np.uint8)
    mask[0:2, 2] = 1
    mask[8, 3] = 1
    dy = _stretched_rows(9, 13)
    dfield = np.full((9, 5), 1.3)
    dfield[4, 1] = 0.7
    kw = dict(dy=dy, dx1=0.09, force=0.0 if top_u else 1.0, top_u=top_u)
    p = oracle.Problem.make(mask, True, False, dfield, ("gh", 6, 0.0), **kw)
    ds = dense.solve(p)
    g_dense = dense.adjoint_gradient(p, ds)
    r = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_it, q_id, iters, ok = oracle.adjoint(p, r["h"], r["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_dense).max()
    assert np.max(np.abs(g_it - g_dense)) < 1e-9 * scale
    if not top_u:
        assert abs(q_id - r["Q"]) < 1e-10 * abs(r["Q"])  # Q = F sum z v1
    for (j, i) in [(4, 1), (0, 0), (7, 4)]:
        step = 1e-5 * dfield[j, i]
        qs = []
        for sgn in (1, -1):
            d = dfield.copy()
            d[j, i] += sgn * step
            qs.append(dense.solve(oracle.Problem.make(mask, True, False, d, ("gh", 6, 0.0), **kw))["Q"])
        assert abs((qs[0] - qs[1]) / (2 * step) - g_dense[j, i]) < 1e-6 * scale
