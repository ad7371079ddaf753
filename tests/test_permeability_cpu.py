"""Host logic of Sec. III's permeability curves and the synthetic media (no GPU).

* k_inf extrapolation: exact on polynomials of its degree; on the oracle's plane-channel flow rates it
  approaches the closed form H^2 / 12 (the plane Poiseuille permeability) within the size of the
  neglected O(Kn^2) term.
* H* and Kn*: the plane channel (phi = 1, k_inf = 1/12) has H* = H and Kn* = Kn.
* Media generators: porosity, periodic non-overlap with the stated gap, connection along x1,
  determinism under the seed; the winding test on hand-made masks.
"""
import functools
import math

import numpy as np
import pytest

import oracle
from paper_1704_03126_gb300 import inputs
from paper_1704_03126_gb300 import permeability as perm


def test_intrinsic_permeability_is_exact_on_polynomials():
    k_inf, b, c = 0.0123, 0.4, -0.9
    kns = [0.01, 0.02, 0.04]
    kas = [k_inf + b * k + c * k * k for k in kns]
    assert abs(perm.intrinsic_permeability(kns, kas) - k_inf) < 1e-15
    # two points: the line through them
    assert abs(perm.intrinsic_permeability([0.1, 0.3], [1.0 + 0.1, 1.0 + 0.3]) - 1.0) < 1e-14
    # least squares over more points than the degree needs
    kns = [0.01, 0.02, 0.03, 0.04, 0.05]
    assert abs(perm.intrinsic_permeability(kns, [2.0 - 3.0 * k for k in kns], degree=1) - 2.0) < 1e-14
    with pytest.raises(ValueError):
        perm.intrinsic_permeability([0.1], [1.0])
    with pytest.raises(ValueError):
        perm.intrinsic_permeability([0.1, 0.1], [1.0, 1.0])
    with pytest.raises(ValueError):
        perm.intrinsic_permeability([0.0, 0.1], [1.0, 1.0])


@functools.lru_cache(maxsize=None)
def _plates_k_a(delta, ny):
    p = oracle.Problem.make(inputs.plates_mask(2, ny), True, False, delta, ("gh", 16, 0.0))
    r = oracle.solve(p, tol=1e-10, max_iter=100000)
    assert r["converged"]
    kn = math.sqrt(math.pi) / (2.0 * delta)
    return kn, perm.apparent_permeability(r["Q"], kn)


def test_plane_channel_intrinsic_permeability_is_h2_over_12():
    """Oracle solves at delta = 10 and 20 (Kn = 0.089, 0.044); the line through them meets Kn = 0 at
    1/12 up to the O(Kn^2) term it neglects (measured -1.9 %).  Extrapolating in delta instead of Kn,
    or from Q instead of k_a, misses by more than 50 %."""
    pts = [_plates_k_a(10.0, 64), _plates_k_a(20.0, 128)]
    k_inf = perm.intrinsic_permeability([p[0] for p in pts], [p[1] for p in pts])
    assert abs(k_inf - 1.0 / 12.0) < 0.03 / 12.0, k_inf
    # apparent permeability exceeds the intrinsic one (slip adds flow)
    assert all(p[1] > k_inf for p in pts)


def test_plane_channel_characteristic_length_and_equivalent_knudsen():
    assert abs(perm.characteristic_length(1.0 / 12.0, 1.0) - 1.0) < 1e-15
    kn = np.array([0.01, 0.1, 1.0, 10.0])
    assert np.allclose(perm.equivalent_knudsen(kn, 1.0 / 12.0, 1.0), kn, rtol=1e-15, atol=0)
    # Kn* = lambda / H*: a medium with half the plane-channel permeability per unit porosity has a
    # smaller H* and a larger Kn*
    assert abs(perm.equivalent_knudsen(1.0, 1.0 / 24.0, 1.0) - math.sqrt(2.0)) < 1e-14
    assert abs(perm.equivalent_knudsen(1.0, 0.6 / 12.0, 0.6) - 1.0) < 1e-14
    with pytest.raises(ValueError):
        perm.characteristic_length(0.0, 0.5)


@pytest.mark.parametrize("kind", inputs.MEDIA)
@pytest.mark.parametrize("n", [64, 256])
def test_media_reach_the_porosity_and_connect_along_x1(kind, n):
    mask, phi = inputs.medium_mask(kind, n)
    assert mask.shape == (n, n) and mask.dtype == np.uint8
    assert 0.55 < phi <= 0.6 + 1.0 / n ** 2
    assert abs((1.0 - mask.mean()) - phi) < 1e-15
    assert inputs.percolates_x(mask)
    again, _ = inputs.medium_mask(kind, n)
    assert np.array_equal(mask, again)


def test_square_solids_keep_their_gap():
    """Every solid component is one square, and two squares never come within the gap (max norm,
    periodic)."""
    n, gap = 96, 2
    mask, _ = inputs.porous_squares_mask(n, 0.65, 6, 14, seed=4, gap=gap)
    # dilate each square by gap - 1 cells: squares closer than gap would merge into one component
    labels = _periodic_components(mask)
    for lab in range(1, labels.max() + 1):
        ys, xs = np.nonzero(labels == lab)
        # the component is a full square (periodic extents)
        hx = _periodic_extent(xs, n)
        hy = _periodic_extent(ys, n)
        assert hx == hy and hx * hy == len(xs)
    assert _min_periodic_gap(mask, labels, n) >= gap + 1


def _periodic_components(mask):
    n = mask.shape[0]
    labels = np.zeros(mask.shape, np.int64)
    cur = 0
    for j, i in zip(*np.nonzero(mask)):
        if labels[j, i]:
            continue
        cur += 1
        labels[j, i] = cur
        stack = [(j, i)]
        while stack:
            a, b = stack.pop()
            for da, db in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)):
                aa, bb = (a + da) % n, (b + db) % n
                if mask[aa, bb] and not labels[aa, bb]:
                    labels[aa, bb] = cur
                    stack.append((aa, bb))
    return labels


def _periodic_extent(coords, n):
    present = np.zeros(n, bool)
    present[np.unique(coords)] = True
    if present.all():
        return n
    # length of the occupied arc: n minus the longest empty run (cyclic)
    empty = ~present
    best = run = 0
    for v in np.concatenate([empty, empty]):
        run = run + 1 if v else 0
        best = max(best, min(run, n))
    return n - best


def _min_periodic_gap(mask, labels, n):
    """Smallest max-norm distance between cells of different squares (cells of the same square: 0)."""
    cells = [np.argwhere(labels == lab) for lab in range(1, labels.max() + 1)]
    best = n
    for a in range(len(cells)):
        for b in range(a + 1, len(cells)):
            d = np.abs(cells[a][:, None, :] - cells[b][None, :, :])
            d = np.minimum(d, n - d).max(axis=2)
            best = min(best, int(d.min()))
    return best


def test_winding_test_on_hand_made_masks():
    wall = np.zeros((10, 10), np.uint8)
    wall[:, 5] = 1
    assert not inputs.percolates_x(wall)
    wall[3, 5] = 0
    assert inputs.percolates_x(wall)
    # a diagonal step is not a 4-neighbour connection
    diag = np.ones((4, 4), np.uint8)
    for k in range(4):
        diag[k, k] = 0
    assert not inputs.percolates_x(diag)
    # a closed channel (walls at both ends of x2) still winds along x1
    assert inputs.percolates_x(np.zeros((3, 5), np.uint8), periodic_y=False)
    # a pocket enclosed by solid does not
    pocket = np.ones((5, 5), np.uint8)
    pocket[2, 2] = 0
    assert not inputs.percolates_x(pocket)
