"""Paired velocity groups in the FP32 row sweep (dvm_batch_set_pairing): two groups of a quadrant per
warp, packed FP32x2 arithmetic.  The update is the same source iteration, so a paired launch reaches
the same fixed point as a launch with one group per warp (to FP32 rounding) and the oracle's (to the
refined FP32 tolerance), across periodic seams, walls, ragged chunks, several pairs per block, an odd
group left over per quadrant, and the stored distribution."""
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


# name, mask, periodic_x, periodic_y, kn, quad: every case has at least two groups per quadrant
CASES = [
    ("rough40_cubic16", inputs.rough_channel_mask(40), True, False, 0.5, ("cubic", 16, 4.0)),
    ("block_periodic_37x23_cubic12", _block(37, 23), True, True, 1.0, ("cubic", 12, 4.0)),
    ("porous48_cubic24_odd_groups", inputs.porous_disks_mask(48, 0.6, 4, 6, seed=5)[0], True, True, 2.0,
     ("cubic", 24, 4.0)),
    ("plates_16x40_cubic32_four_pairs_per_block", inputs.plates_mask(16, 40), True, False, 0.3, ("cubic", 32, 4.0)),
]


def _solve(case, pairing, store=False, schedule=("rows", 0), persistent=False):
    _, mask, px, py, kn, quad = case
    sol = dvm.Solver(mask, px, py, kn=kn, quad=quad, precision="fp32", store_distribution=store)
    b = dvm.Batch([sol])
    b.set_schedule(*schedule)
    b.set_pairing(pairing)
    if persistent:
        b.set_persistent(True)
    mode, blocks = b.pairing()
    st = b.run(tol=1e-7, max_iter=200000)
    assert all(v == dvm.DVM_OK for v in st)
    return sol, b, blocks


@pytest.mark.parametrize("schedule", [("rows", 0), ("rows", 8), ("rows", 4)], ids=["rows", "rows8", "rows4"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_paired_groups_match_single_groups_and_the_oracle(case, schedule):
    name, mask, px, py, kn, quad = case
    on, _, blocks_on = _solve(case, "on", schedule=schedule)
    off, _, blocks_off = _solve(case, "off", schedule=schedule)
    assert blocks_on > 0 and blocks_off == 0
    q_on, q_off = on.flowrate()[0], off.flowrate()[0]
    assert abs(q_on - q_off) < 1e-6 * abs(q_off), (q_on, q_off)
    f_on, f_off = on.fields(), off.fields()
    gas = mask == 0
    for nm in ("rho", "u1", "u2", "tau"):
        scale = max(1.0, np.abs(f_off[nm][gas]).max())
        assert np.abs(f_on[nm][gas] - f_off[nm][gas]).max() < 1e-5 * scale, nm
    orc = oracle.solve(oracle.Problem.make(mask, px, py, dvm.kn_to_delta(kn), quad), tol=1e-12, max_iter=400000)
    assert orc["converged"]
    assert abs(q_on - orc["Q"]) < 1e-5 * abs(orc["Q"]), (q_on, orc["Q"])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_paired_groups_in_the_persistent_launch(case):
    """The persistent launch hands out paired tiles like single ones: the same sweeps as per-kernel
    launches with pairs (same sweep count; sums in another order), the same fixed point as launches
    without pairs (the FP32 stopping test ends on rounding noise, which pairing changes: no sweep count
    there)."""
    on, b, blocks_on = _solve(case, "on", persistent=True)
    assert b.persistent()[0] and blocks_on > 0
    kern, _, _ = _solve(case, "on")
    off, _, _ = _solve(case, "off")
    assert abs(on.info()["iterations"] - kern.info()["iterations"]) <= 2, \
        (on.info()["iterations"], kern.info()["iterations"], off.info()["iterations"])
    q_on, q_kern, q_off = on.flowrate()[0], kern.flowrate()[0], off.flowrate()[0]
    assert abs(q_on - q_kern) < 1e-7 * abs(q_kern), (q_on, q_kern)
    assert abs(q_on - q_off) < 1e-6 * abs(q_off), (q_on, q_off)
    gas = case[1] == 0
    for nm in ("rho", "u1"):
        f_on, f_off = on.fields()[nm], off.fields()[nm]
        assert np.abs(f_on[gas] - f_off[gas]).max() < 1e-5 * max(1.0, np.abs(f_off[gas]).max()), nm


def test_persistent_batch_of_paired_and_single_members():
    """All four geometries in one persistent batch (paired and leftover single tiles of several members
    in one scheduler, members retiring at different sweeps) against separate unpaired solves."""
    def members():
        return [dvm.Solver(c[1], c[2], c[3], kn=c[4], quad=c[5], precision="fp32") for c in CASES]
    sols = members()
    b = dvm.Batch(sols)
    b.set_schedule("rows", 0)
    b.set_pairing("on")
    b.set_persistent(True)
    assert b.pairing()[1] > 0
    assert all(v == dvm.DVM_OK for v in b.run(tol=1e-7, max_iter=200000))
    for s, case in zip(sols, CASES):
        off, _, _ = _solve(case, "off")
        assert abs(s.flowrate()[0] - off.flowrate()[0]) < 1e-6 * abs(off.flowrate()[0]), case[0]


def test_paired_sweep_stores_the_same_distribution():
    """One paired sweep from the same state writes the distribution the single-group sweep writes."""
    case = CASES[1]
    _, mask, px, py, kn, quad = case
    out = []
    for pairing in ("on", "off"):
        sol = dvm.Solver(mask, px, py, kn=kn, quad=quad, precision="fp32", store_distribution=True)
        b = dvm.Batch([sol])
        b.set_schedule("rows", 0)
        b.set_pairing(pairing)
        b.iterate(7)
        ks = np.arange(0, quad[1] * quad[1], 5)
        out.append(sol.distribution(ks))
    scale = np.abs(out[1]).max()
    assert np.abs(out[0] - out[1]).max() < 1e-5 * scale


def test_pairing_policy():
    """AUTO pairs only launches with at least three waves of single-group blocks; OFF never; a bad mode
    is rejected; FP64 batches are never paired."""
    case = CASES[0]
    _, mask, px, py, kn, quad = case
    sol = dvm.Solver(mask, px, py, kn=kn, quad=quad, precision="fp32")
    b = dvm.Batch([sol])
    b.set_schedule("rows", 0)
    assert b.pairing() == ("auto", 0)  # one small member: too few blocks to pair
    b.set_pairing("on")
    assert b.pairing()[1] > 0
    b.set_schedule("rows", 8)  # the policy survives a schedule change
    assert b.pairing()[0] == "on" and b.pairing()[1] > 0
    assert dvm.lib().dvm_batch_set_pairing(b._b, 7) == dvm.DVM_EINVAL
    assert b.pairing()[0] == "on"
    d = dvm.Solver(mask, px, py, kn=kn, quad=quad, precision="fp64")
    bd = dvm.Batch([d])
    bd.set_schedule("rows", 0)
    bd.set_pairing("on")
    assert bd.pairing()[1] == 0
    # many members: AUTO pairs by itself
    many = [dvm.Solver(inputs.rough_channel_mask(96), True, False, kn=kn, quad=("cubic", 32, 4.0), precision="fp32")
            for kn in np.geomspace(0.1, 10.0, 16)]
    bm = dvm.Batch(many)
    bm.set_schedule("rows", 16)
    assert bm.pairing()[1] > 0
    # a solve drops the pairs once the members still iterating fill fewer than three waves, and the
    # next solve plans them again; the fixed points are those of a launch that never pairs
    assert all(v == dvm.DVM_OK for v in bm.run(tol=1e-6, max_iter=50000))
    assert bm.pairing()[0] == "auto"
    ref = [dvm.Solver(inputs.rough_channel_mask(96), True, False, kn=kn, quad=("cubic", 32, 4.0), precision="fp32")
           for kn in np.geomspace(0.1, 10.0, 16)]
    br = dvm.Batch(ref)
    br.set_schedule("rows", 16)
    br.set_pairing("off")
    assert all(v == dvm.DVM_OK for v in br.run(tol=1e-6, max_iter=50000))
    for a, r in zip(many, ref):
        assert abs(a.flowrate()[0] - r.flowrate()[0]) < 1e-6 * abs(r.flowrate()[0])
    for s in many:
        s.reset()
    assert all(v == dvm.DVM_OK for v in bm.run(tol=1e-6, max_iter=50000))
    for a, r in zip(many, ref):
        assert abs(a.flowrate()[0] - r.flowrate()[0]) < 1e-6 * abs(r.flowrate()[0])
