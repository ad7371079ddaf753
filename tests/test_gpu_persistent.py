"""The persistent batched launch (dvm_batch_set_persistent): one kernel advances every member with a
device-side scheduler.  It computes the same source iteration as the per-kernel launches, so its fixed
points, iteration counts and the oracle parity are the same (sums in another order: rounding)."""
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


def _members(precision):
    """Mixed widths (several velocity groups per block for the narrow ones), both geometries, three
    velocity grids, Knudsen numbers from near-continuum to rarefied."""
    out = [inputs.rough_instance(0.1, n=32, nv=8), inputs.rough_instance(2.0, n=64, nv=12),
           inputs.porous_instance(0.5, n=48, nv=10, porosity=0.6, seed=3, rmin=3, rmax=6),
           inputs.plates_instance(0.2, nx=4, ny=24, nv=8)]
    return [dvm.Solver(i.mask, i.periodic_x, i.periodic_y, kn=i.kn, quad=i.quad, precision=precision) for i in out], out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_batch_matches_per_kernel_launches(precision):
    tol = 1e-11 if precision == "fp64" else 1e-7
    ref, insts = _members(precision)
    b0 = dvm.Batch(ref)
    b0.set_schedule("rows", 0)
    st0 = b0.run(tol=tol, max_iter=100000)
    per, _ = _members(precision)
    b1 = dvm.Batch(per)
    b1.set_schedule("rows", 0)
    b1.set_persistent(True)
    on, blocks = b1.persistent()
    assert on and blocks >= 1
    st1 = b1.run(tol=tol, max_iter=100000)
    assert all(v == 0 for v in st0) and all(v == 0 for v in st1)
    rel = 1e-10 if precision == "fp64" else 1e-7
    for a, c, inst in zip(ref, per, insts):
        qa, qc = a.flowrate()[0], c.flowrate()[0]
        assert abs(qa - qc) < rel * abs(qa), (inst.name, qa, qc)
        # each member stops on its own test: the same sweep count as in the per-kernel batch (the
        # stopping test sits on a knife edge only at the rounding level)
        assert abs(a.info()["iterations"] - c.info()["iterations"]) <= 2
        fa, fc = a.fields()["u1"], c.fields()["u1"]
        gas = inst.mask == 0
        assert np.abs(fa[gas] - fc[gas]).max() < rel * max(1.0, np.abs(fa[gas]).max())
    # against the oracle (FP64)
    if precision == "fp64":
        for s, inst in zip(per, insts):
            orc = oracle.solve(oracle.Problem.make(inst.mask, inst.periodic_x, inst.periodic_y, dvm.kn_to_delta(inst.kn),
                                                   inst.quad), tol=1e-12, max_iter=200000)
            assert abs(s.flowrate()[0] - orc["Q"]) < 1e-10 * abs(orc["Q"])


def test_persistent_members_stop_on_their_own():
    """A fast and a slow member in one persistent launch: the fast one retires inside the launch after
    its own sweeps (same count as solved alone), while the slow one runs on."""
    fast = inputs.rough_instance(5.0, n=32, nv=8)
    slow = inputs.rough_instance(0.05, n=32, nv=8)
    alone = []
    for inst in (fast, slow):
        s = dvm.Solver(inst.mask, True, False, kn=inst.kn, quad=inst.quad, precision="fp64", schedule=("rows", 0))
        s.solve(tol=1e-10, max_iter=100000)
        alone.append(s.info()["iterations"])
    sols = [dvm.Solver(i.mask, True, False, kn=i.kn, quad=i.quad, precision="fp64") for i in (fast, slow)]
    b = dvm.Batch(sols)
    b.set_schedule("rows", 0)
    b.set_persistent(True)
    st = b.run(tol=1e-10, max_iter=100000)
    assert all(v == 0 for v in st)
    its = [s.info()["iterations"] for s in sols]
    assert abs(its[0] - alone[0]) <= 1 and abs(its[1] - alone[1]) <= 1, (its, alone)
    assert its[1] > 5 * its[0]


def test_persistent_enqueued_sweeps_match_iterate():
    """n enqueued single sweeps (the benchmark's timed steps) and n sweeps by iterate reach the same state."""
    insts = [inputs.rough_instance(kn, n=32, nv=8) for kn in (0.1, 1.0)]
    qs = []
    for mode in ("iterate", "enqueue"):
        sols = [dvm.Solver(i.mask, True, False, kn=i.kn, quad=i.quad, precision="fp64") for i in insts]
        b = dvm.Batch(sols)
        b.set_schedule("rows", 0)
        b.set_persistent(True)
        if mode == "iterate":
            b.iterate(70)
        else:
            for _ in range(70):
                b.enqueue(1)
            b.check()
            sweep_ms, fin_ms = b.timing()
            assert sweep_ms > 0.0 and fin_ms >= 0.0
        assert all(s.info()["iterations"] == 70 for s in sols)
        qs.append([s.flowrate()[0] for s in sols])
    assert np.allclose(qs[0], qs[1], rtol=1e-12, atol=0.0)


def test_persistent_launch_restrictions():
    """Column sweep, moving plates and Anderson mixing stay on per-kernel launches."""
    mask, ly = inputs.couette_rough_mask(12, aspect=3.0, eps=0.05)
    s = dvm.Solver(mask, True, False, kn=0.5, quad=("cubic", 8, 4.0), precision="fp64", ly=ly, force=0.0,
                   top_wall_u1=1.0)
    b = dvm.Batch([s])
    with pytest.raises(dvm.DvmError) as ei:
        b.set_persistent(True)
    assert ei.value.status == dvm.DVM_EINVAL
    p = inputs.plates_instance(0.3, nx=4, ny=12, nv=8)
    a = dvm.Solver(p.mask, True, False, kn=p.kn, quad=p.quad, precision="fp64", anderson=3)
    b = dvm.Batch([a])
    b.set_schedule("rows", 0)
    with pytest.raises(dvm.DvmError):
        b.set_persistent(True)


def test_persistent_scheduler_wait_gives_up():
    """The scheduler's poll on an active instance whose work never appears gives up (DVM_ETIMEOUT) in
    about a second, with no fault and no hang; the device stays usable."""
    st, sec = dvm.selftest_wait(2, 0)
    assert st == dvm.DVM_ETIMEOUT and sec < 10.0, (st, sec)
    inst = inputs.plates_instance(kn=0.3, nx=4, ny=12, nv=8)
    sol = dvm.Solver(inst.mask, True, False, kn=inst.kn, quad=inst.quad, precision="fp64")
    b = dvm.Batch([sol])
    b.set_schedule("rows", 0)
    b.set_persistent(True)
    assert all(v == 0 for v in b.run(tol=1e-12, max_iter=100000))
    orc = oracle.solve(oracle.Problem.make(inst.mask, True, False, dvm.kn_to_delta(inst.kn), inst.quad), tol=1e-12,
                       max_iter=100000)
    assert abs(sol.flowrate()[0] - orc["Q"]) < 1e-10 * abs(orc["Q"])


def test_destroying_a_member_first_detaches_the_batch():
    """A batch whose member is destroyed first (as garbage collection of a reference cycle may do)
    releases its launches while the member's stream still exists; it then answers DVM_ESTATE and can
    still be destroyed."""
    insts = [inputs.rough_instance(kn, n=32, nv=8) for kn in (0.5, 2.0)]
    sols = [dvm.Solver(i.mask, True, False, kn=i.kn, quad=i.quad, precision="fp64") for i in insts]
    for persistent in (False, True):
        b = dvm.Batch(sols)
        b.set_schedule("rows", 0)
        b.set_persistent(persistent)
        b.iterate(3)
        if persistent:
            sols[0].close()
            with pytest.raises(dvm.DvmError) as ei:
                b.iterate(1)
            assert ei.value.status == dvm.DVM_ESTATE
            assert b.kernels_per_sweep() == 0
        b.close()
    # the surviving member still solves
    sols[1].solve(tol=1e-10, max_iter=100000)
    orc = oracle.solve(oracle.Problem.make(insts[1].mask, True, False, dvm.kn_to_delta(insts[1].kn), insts[1].quad),
                       tol=1e-12, max_iter=100000)
    assert abs(sols[1].flowrate()[0] - orc["Q"]) < 1e-10 * abs(orc["Q"])
