"""GPU adjoint (dvm_adjoint, transposed sweeps through the C ABI) against the FP64 oracle's adjoint of
the same projected iteration, the forward/adjoint identity Q = F sum z v1, and central differences of
GPU forward solves."""
import functools

import numpy as np
import pytest

import oracle
from paper_1704_03126_gb300 import build as dvm_build
from paper_1704_03126_gb300 import dvm, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    dvm_build.build()
    return dvm.lib()


def _block(nx, ny):
    m = np.zeros((ny, nx), np.uint8)
    m[ny // 3: ny // 3 + 3, nx // 2: nx // 2 + 4] = 1
    return m


CASES = [
    ("plates_gh8", inputs.plates_mask(4, 16), True, False, 0.7, ("gh", 8, 0.0)),
    ("rough24_nc8", inputs.rough_channel_mask(24), True, False, 1.5, ("nc", 8, 4.0)),
    ("block_periodic_cubic10", _block(20, 16), True, True, 1.0, ("cubic", 10, 4.0)),
    ("porous40_cubic12", inputs.porous_disks_mask(40, 0.6, 4, 6, seed=5)[0], True, True, 2.0, ("cubic", 12, 4.0)),
    ("closed_box_nc8", _block(12, 12), False, False, 1.0, ("nc", 8, 4.0)),
]


def _delta_field(mask, base, seed):
    rng = np.random.default_rng(seed)
    return base * rng.uniform(0.5, 1.5, size=mask.shape)


SCHEDULES = [("rows", 0), ("columns", 1), ("columns", 2), ("columns", 4)]


@functools.lru_cache(maxsize=None)
def _oracle_gradient(name):
    _, mask, px, py, delta, quad = next(c for c in CASES if c[0] == name)
    d = _delta_field(mask, delta, 3)
    p = oracle.Problem.make(mask, px, py, d, quad)
    ref = oracle.solve(p, tol=1e-13, max_iter=200000)
    return oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=200000)


@pytest.mark.parametrize("schedule", SCHEDULES, ids=["rows", "cols1", "cols2", "cols4"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoint_gradient_matches_oracle(case, schedule):
    name, mask, px, py, delta, quad = case
    d = _delta_field(mask, delta, 3)
    sol = dvm.Solver(mask, px, py, delta=delta, quad=quad, precision="fp64", store_distribution=True,
                     schedule=schedule)
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=200000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=200000)
    g_ref, q_ref_id, _, ok = _oracle_gradient(name)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale, np.abs(grad - g_ref).max() / scale
    q, _ = sol.flowrate()
    assert abs(q_id - q) < 1e-9 * abs(q)
    assert np.all(grad[mask == 1] == 0.0)


def test_adjoint_matches_central_differences_of_gpu_solves():
    mask = inputs.rough_channel_mask(16)
    quad = ("nc", 8, 4.0)
    d = _delta_field(mask, 1.0, 9)
    sol = dvm.Solver(mask, True, False, delta=1.0, quad=quad, precision="fp64", store_distribution=True)
    sol.set_delta_field(d)
    sol.solve(tol=1e-14, max_iter=200000)
    grad, _, _ = sol.adjoint(tol=1e-13, max_iter=200000)
    gas = np.flatnonzero(mask.ravel() == 0)
    for cell in gas[[0, 17, 60, len(gas) - 1]]:
        step = 1e-4 * d.ravel()[cell]
        qs = []
        for sgn in (1, -1):
            dd = d.copy().ravel()
            dd[cell] += sgn * step
            s = dvm.Solver(mask, True, False, delta=1.0, quad=quad, precision="fp64")
            s.set_delta_field(dd.reshape(mask.shape))
            s.solve(tol=1e-14, max_iter=200000)
            qs.append(s.flowrate()[0])
        fd = (qs[0] - qs[1]) / (2 * step)
        assert abs(fd - grad.ravel()[cell]) < 1e-6 * np.abs(grad).max()


def test_adjoint_requires_stored_distribution():
    sol = dvm.Solver(inputs.plates_mask(4, 8), True, False, kn=1.0, quad=("gh", 4, 0.0))
    sol.solve(tol=1e-10)
    with pytest.raises(dvm.DvmError) as ei:
        sol.adjoint()
    assert ei.value.status == dvm.DVM_ESTATE


def test_autograd_flow_rate_backward():
    import torch

    from paper_1704_03126_gb300.autograd import flow_rate

    mask = inputs.porous_disks_mask(32, 0.65, 3, 5, seed=4)[0]
    quad = ("cubic", 8, 4.0)
    sol = dvm.Solver(mask, True, True, delta=1.0, quad=quad, precision="fp64", store_distribution=True)
    d0 = _delta_field(mask, 1.2, 11)
    delta = torch.tensor(d0, dtype=torch.float64, device="cuda", requires_grad=True)
    q = flow_rate(delta, sol, tol=1e-13)
    q.backward()
    g_auto = delta.grad.cpu().numpy()
    # the same gradient from the oracle's adjoint
    p = oracle.Problem.make(mask, True, True, d0, quad)
    ref = oracle.solve(p, tol=1e-13, max_iter=200000)
    g_ref, _, _, _ = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=200000)
    assert abs(q.item() - ref["Q"]) < 1e-10 * abs(ref["Q"])
    assert np.abs(g_auto - g_ref).max() < 1e-8 * np.abs(g_ref).max()
    # one directional derivative along a random direction
    rng = np.random.default_rng(2)
    dirn = rng.standard_normal(mask.shape) * (mask == 0)
    eps = 1e-5
    qp = flow_rate(torch.tensor(d0 + eps * dirn, device="cuda"), sol, tol=1e-14).item()
    qm = flow_rate(torch.tensor(d0 - eps * dirn, device="cuda"), sol, tol=1e-14).item()
    assert abs((qp - qm) / (2 * eps) - float((g_auto * dirn).sum())) < 1e-6 * np.abs(g_auto).sum()


def test_autograd_backward_after_the_solver_moved_on():
    """One solver, two graph nodes: forward(d1), forward(d2), then backward of the first.  The first
    node's gradient must be the one at d1 (backward re-solves at d1), equal to that of a fresh
    forward(d1) + backward; and an adjoint cut short by max_iter raises unless allowed."""
    import torch

    from paper_1704_03126_gb300.autograd import flow_rate

    mask = inputs.porous_disks_mask(24, 0.7, 2, 4, seed=5)[0]
    quad = ("cubic", 8, 4.0)
    sol = dvm.Solver(mask, True, True, delta=1.0, quad=quad, precision="fp64", store_distribution=True)
    d1 = _delta_field(mask, 1.2, 21)
    d2 = _delta_field(mask, 0.4, 22)
    t1 = torch.tensor(d1, dtype=torch.float64, device="cuda", requires_grad=True)
    t2 = torch.tensor(d2, dtype=torch.float64, device="cuda", requires_grad=True)
    q1 = flow_rate(t1, sol, tol=1e-13)
    q2 = flow_rate(t2, sol, tol=1e-13)
    q1.backward()
    g1 = t1.grad.cpu().numpy()
    p = oracle.Problem.make(mask, True, True, d1, quad)
    ref = oracle.solve(p, tol=1e-13, max_iter=200000)
    g_ref, _, _, _ = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=200000)
    assert np.abs(g1 - g_ref).max() < 1e-8 * np.abs(g_ref).max()
    q2.backward()
    g2 = t2.grad.cpu().numpy()
    p2 = oracle.Problem.make(mask, True, True, d2, quad)
    ref2 = oracle.solve(p2, tol=1e-13, max_iter=200000)
    g_ref2, _, _, _ = oracle.adjoint(p2, ref2["h"], ref2["c"], tol=1e-13, max_iter=200000)
    assert np.abs(g2 - g_ref2).max() < 1e-8 * np.abs(g_ref2).max()
    # an adjoint iteration stopped by max_iter: error by default, a warning when allowed
    t3 = torch.tensor(d1, dtype=torch.float64, device="cuda", requires_grad=True)
    q3 = flow_rate(t3, sol, tol=1e-13, adjoint_max_iter=3)
    with pytest.raises(dvm.DvmError) as ei:
        q3.backward()
    assert ei.value.status == dvm.DVM_ENOCONV
    t4 = torch.tensor(d1, dtype=torch.float64, device="cuda", requires_grad=True)
    q4 = flow_rate(t4, sol, tol=1e-13, adjoint_max_iter=3, allow_noconv=True)
    with pytest.warns(RuntimeWarning):
        q4.backward()


@pytest.mark.parametrize("storage", ["as_given", "transposed"])
@pytest.mark.parametrize("schedule", SCHEDULES[:2], ids=["rows", "cols1"])
@pytest.mark.parametrize("name", ["rough24_nc8", "block_periodic_cubic10"])
def test_adjoint_gradient_in_either_storage_order(name, schedule, storage):
    """The transposed grid takes the adjoint source g = W v_flow dA / L along its x2; the gradient comes
    back in the caller's layout."""
    _, mask, px, py, delta, quad = next(c for c in CASES if c[0] == name)
    d = _delta_field(mask, delta, 3)
    sol = dvm.Solver(mask, px, py, delta=delta, quad=quad, precision="fp64", store_distribution=True,
                     schedule=schedule, storage=storage)
    assert sol.info()["transposed"] == (storage == "transposed")
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=200000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=200000)
    g_ref, q_ref_id, _, ok = _oracle_gradient(name)
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale
    assert abs(q_id - sol.flowrate()[0]) < 1e-9 * abs(q_id)


def test_adjoint_after_a_mixed_forward_solve():
    """Anderson-mixed forward iterates (FP64) converge to the same state, so the adjoint taken there
    matches the oracle's gradient."""
    name = "rough24_nc8"
    _, mask, px, py, delta, quad = next(c for c in CASES if c[0] == name)
    d = _delta_field(mask, delta, 3)
    sol = dvm.Solver(mask, px, py, delta=delta, quad=quad, precision="fp64", store_distribution=True, anderson=5)
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=200000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=200000)
    g_ref, _, _, ok = _oracle_gradient(name)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale
    assert abs(q_id - sol.flowrate()[0]) < 1e-9 * abs(q_id)


@pytest.mark.parametrize("storage", ["as_given", "transposed"])
def test_couette_adjoint_matches_oracle(storage):
    """Gradient of the Couette flow rate (plate moving with U = 1 over a notched wall, no force) with
    respect to a per-cell collision rate: the GPU adjoint against the oracle's adjoint at its own
    converged state."""
    mask = np.zeros((10, 8), np.uint8)
    mask[0:2, 3] = 1
    mask[0, 5] = 1
    d = _delta_field(mask, 1.2, 5)
    quad = ("cubic", 8, 4.0)
    sol = dvm.Solver(mask, True, False, delta=1.2, quad=quad, precision="fp64", store_distribution=True, force=0.0,
                     top_wall_u1=1.0, storage=storage)
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=200000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=200000)
    p = oracle.Problem.make(mask, True, False, d, quad, force=0.0, top_u=1.0)
    ref = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_ref, _, _, ok = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale
    assert abs(q_id) < 1e-14


# ------------------------------------------------------------------ partially specular walls, unequal rows

def _stretched_rows(ny, seed):
    rng = inputs.SplitMix64(seed)
    h = np.array([0.4 + 1.2 * rng.uniform() for _ in range(ny)])
    return h / h.sum()


def _notch(nx, ny):
    m = np.zeros((ny, nx), np.uint8)
    m[0:2, nx // 3] = 1
    m[ny - 1, nx // 2: nx // 2 + 2] = 1
    return m


SPEC_ADJ_CASES = [
    # name, mask, periodic_x, periodic_y, delta, quad, alpha
    ("plates_gh8_a0.6", inputs.plates_mask(4, 16), True, False, 0.7, ("gh", 8, 0.0), 0.6),
    ("rough24_nc8_a0.5", inputs.rough_channel_mask(24), True, False, 1.5, ("nc", 8, 4.0), 0.5),
    ("block_periodic_cubic10_a0.8", _block(20, 16), True, True, 1.0, ("cubic", 10, 4.0), 0.8),
    ("closed_box_nc8_a0.3", _block(12, 12), False, False, 1.0, ("nc", 8, 4.0), 0.3),
]


@functools.lru_cache(maxsize=None)
def _oracle_spec_gradient(name):
    _, mask, px, py, delta, quad, alpha = next(c for c in SPEC_ADJ_CASES if c[0] == name)
    p = oracle.Problem.make(mask, px, py, _delta_field(mask, delta, 4), quad, alpha=alpha)
    ref = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_ref, _, _, ok = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=400000)
    return g_ref, ok


@functools.lru_cache(maxsize=None)
def _oracle_unequal_gradient(name):
    _, mask, px, delta, quad, alpha, top_u = next(c for c in UNEQUAL_ADJ_CASES if c[0] == name)
    p = oracle.Problem.make(mask, px, False, _delta_field(mask, delta, 6), quad, alpha=alpha,
                            force=0.0 if top_u else 1.0, top_u=top_u, dy=_stretched_rows(mask.shape[0], 23), dx1=0.07)
    ref = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_ref, _, _, ok = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=400000)
    return g_ref, ok


@pytest.mark.parametrize("schedule", [("columns", 1), ("columns", 2), ("columns", 4)], ids=["cols1", "cols2", "cols4"])
@pytest.mark.parametrize("case", SPEC_ADJ_CASES, ids=[c[0] for c in SPEC_ADJ_CASES])
def test_partially_specular_adjoint_matches_oracle(case, schedule):
    """Accommodation alpha < 1 (Eq. diffuse2 with a specular part): the transposed sweep reflects
    (1 - alpha) 2 |v_a|/dx z of the mirrored velocity at each wall face into the next one; the GPU
    gradient against the oracle's adjoint of the same iteration."""
    name, mask, px, py, delta, quad, alpha = case
    d = _delta_field(mask, delta, 4)
    sol = dvm.Solver(mask, px, py, delta=delta, quad=quad, precision="fp64", store_distribution=True,
                     schedule=schedule, accommodation=alpha)
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=400000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=400000)
    g_ref, ok = _oracle_spec_gradient(name)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale, np.abs(grad - g_ref).max() / scale
    q, _ = sol.flowrate()
    assert abs(q_id - q) < 1e-9 * abs(q)
    assert np.all(grad[mask == 1] == 0.0)


UNEQUAL_ADJ_CASES = [
    # name, mask, periodic_x, delta, quad, alpha, top_u
    ("plates_gh8", np.zeros((18, 5), np.uint8), True, 0.6, ("gh", 8, 0.0), 1.0, 0.0),
    ("plates8x4_gh4", np.zeros((8, 4), np.uint8), True, 0.9, ("gh", 4, 0.0), 1.0, 0.0),
    ("notched_nc8", _notch(9, 14), True, 1.2, ("nc", 8, 4.0), 1.0, 0.0),
    ("notched_nc8_a0.6", _notch(9, 14), True, 1.2, ("nc", 8, 4.0), 0.6, 0.0),
    ("couette_notched_cubic8_a0.7", _notch(9, 14), True, 1.0, ("cubic", 8, 4.0), 0.7, 1.0),
]


@pytest.mark.parametrize("schedule", [("columns", 1), ("columns", 2), ("columns", 4)], ids=["cols1", "cols2", "cols4"])
@pytest.mark.parametrize("case", UNEQUAL_ADJ_CASES, ids=[c[0] for c in UNEQUAL_ADJ_CASES])
def test_unequal_rows_adjoint_matches_oracle(case, schedule):
    """Rows of seeded unequal heights (stored transposed: columns of unequal width): the transposed
    sweep pulls z of its two forward-downstream columns with their stretched weights; the source
    g = W v1 dA / Lx carries each row's height."""
    name, mask, px, delta, quad, alpha, top_u = case
    dy = _stretched_rows(mask.shape[0], 23)
    force = 0.0 if top_u else 1.0
    d = _delta_field(mask, delta, 6)
    sol = dvm.Solver(mask, px, False, delta=delta, quad=quad, precision="fp64", store_distribution=True,
                     schedule=schedule, accommodation=alpha, top_wall_u1=top_u, force=force, dx1=0.07,
                     row_heights=dy)
    assert sol.info()["transposed"]
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=400000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=400000)
    g_ref, ok = _oracle_unequal_gradient(name)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale, np.abs(grad - g_ref).max() / scale
    if force:
        assert abs(q_id - sol.flowrate()[0]) < 1e-9 * abs(q_id)
    else:
        assert abs(q_id) < 1e-14


@pytest.mark.parametrize("schedule", [("rows", 0), ("columns", 1), ("columns", 2)], ids=["rows", "cols1", "cols2"])
@pytest.mark.parametrize("storage", ["as_given", "transposed"])
def test_rectangular_cells_adjoint_matches_oracle(storage, schedule):
    """Equal rows of height ly / ny with a different x1 spacing (cells not square)."""
    mask = _notch(12, 10)
    ny = mask.shape[0]
    d = _delta_field(mask, 1.1, 8)
    sol = dvm.Solver(mask, True, False, delta=1.1, quad=("nc", 8, 4.0), precision="fp64", store_distribution=True,
                     schedule=schedule, dx1=0.043, storage=storage)
    sol.set_delta_field(d)
    sol.solve(tol=1e-13, max_iter=400000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=400000)
    p = oracle.Problem.make(mask, True, False, d, ("nc", 8, 4.0), dy=np.full(ny, 1.0 / ny), dx1=0.043)
    ref = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_ref, _, _, ok = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale, np.abs(grad - g_ref).max() / scale
    assert abs(q_id - sol.flowrate()[0]) < 1e-9 * abs(q_id)


@pytest.mark.parametrize("schedule", [("columns", 1), ("columns", 4)], ids=["cols1", "cols4"])
def test_unequal_rows_adjoint_with_a_uniform_collision_rate(schedule):
    """Unequal rows with one collision rate for every cell (no delta field): the transposed sweep still
    takes per-cell denominators, since the stretched columns change the stencil's diagonal."""
    mask = _notch(9, 14)
    dy = _stretched_rows(mask.shape[0], 29)
    sol = dvm.Solver(mask, True, False, delta=0.9, quad=("nc", 8, 4.0), precision="fp64", store_distribution=True,
                     schedule=schedule, dx1=0.07, row_heights=dy)
    sol.solve(tol=1e-13, max_iter=400000)
    grad, q_id, iters = sol.adjoint(tol=1e-13, max_iter=400000)
    p = oracle.Problem.make(mask, True, False, 0.9, ("nc", 8, 4.0), dy=dy, dx1=0.07)
    ref = oracle.solve(p, tol=1e-14, max_iter=400000)
    g_ref, _, _, ok = oracle.adjoint(p, ref["h"], ref["c"], tol=1e-13, max_iter=400000)
    assert ok
    scale = np.abs(g_ref).max()
    assert np.abs(grad - g_ref).max() < 1e-8 * scale, np.abs(grad - g_ref).max() / scale
    assert abs(q_id - sol.flowrate()[0]) < 1e-9 * abs(q_id)
