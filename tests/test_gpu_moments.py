"""dvm_moments: moments and flow rate of a caller-held distribution (C ABI, device pointers)."""
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


def reference_moments(h, mask, quad, dA_over_L):
    """Plain quadrature sums (Sec. II.A): h [K][ncell]."""
    x, w = oracle.quadrature(*quad)
    n = len(x)
    v1 = np.repeat(x, n)
    v2 = np.tile(x, n)
    W = np.outer(w, w).ravel()
    rho = W @ h
    u1 = (W * v1) @ h
    u2 = (W * v2) @ h
    tau = (W * (v1 * v1 + v2 * v2)) @ h - rho
    gas = np.ones(h.shape[1], bool) if mask is None else mask.ravel() == 0
    mom = np.stack([rho, u1, u2, tau], axis=1)
    mom[~gas] = 0.0
    return mom, u1[gas].sum() * dA_over_L


def run_moments(h, mask, quad, dA_over_L):
    import torch

    dev = torch.device("cuda")
    th = torch.from_numpy(np.ascontiguousarray(h)).to(dev)
    tm = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask.ravel().astype(np.uint8))).to(dev)
    mom = torch.empty((h.shape[1], 4), dtype=torch.float64, device=dev)
    q = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    dvm.moments(th.data_ptr(), h.shape[1], quad, mom.data_ptr(), q.data_ptr(), dA_over_L,
                mask_ptr=None if tm is None else tm.data_ptr(), stream=stream)
    return mom.cpu().numpy(), float(q.cpu().item())


@pytest.mark.parametrize("ncell,quad,with_mask", [
    (37 * 29, ("nc", 10, 4.0), True),
    (300_001, ("gh", 4, 0.0), False),     # more cells than blocks x threads: grid-stride and ragged tail
    (1, ("cubic", 6, 4.0), False),
])
def test_moments_match_numpy(ncell, quad, with_mask):
    rng = np.random.default_rng(11)
    K = quad[1] ** 2
    h = rng.standard_normal((K, ncell))
    mask = (rng.random(ncell) < 0.2).astype(np.uint8) if with_mask else None
    dA = 1.0 / 29.0 / 37.0
    mom, q = run_moments(h, mask, quad, dA)
    ref, qref = reference_moments(h, mask, quad, dA)
    assert np.abs(mom - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert abs(q - qref) < 1e-12 * max(1.0, abs(qref))
    mom2, q2 = run_moments(h, mask, quad, dA)
    assert q2 == q and np.array_equal(mom2, mom)  # deterministic


def test_moments_of_solver_state_match_its_fields():
    mask = inputs.rough_channel_mask(24)
    quad = ("nc", 8, 4.0)
    sol = dvm.Solver(mask, True, False, kn=1.0, quad=quad, precision="fp64", store_distribution=True)
    sol.solve(tol=1e-10, max_iter=10000)
    K = quad[1] ** 2
    h = sol.distribution(np.arange(K)).reshape(K, -1)
    ny, nx = mask.shape
    dA = (1.0 / ny) ** 2 / (nx / ny)
    mom, q = run_moments(h, mask, quad, dA)
    f = sol.fields()
    gas = mask.ravel() == 0
    for i, name in enumerate(("rho", "u1", "u2", "tau")):
        assert np.abs(mom[gas, i] - f[name].ravel()[gas]).max() < 1e-11
    assert abs(q - sol.flowrate()[0]) < 1e-11 * abs(q)
