"""Seeded synthetic geometries and workload lists.

This module only builds inputs: solid masks, Knudsen numbers, velocity-grid choices and sampled
cell lists.  It holds none of the solver's arithmetic, so both the CUDA path and the CPU oracle can
be fed from it.

The paper's own geometries are a Weierstrass-Mandelbrot rough wall (Sec. II, Eq. WM) and three
porous media shown only as images (Sec. III, Fig. 4).  The generators below make stand-ins with
the same structure: a staircase wall on a Cartesian grid (Sec. II.A, "stair case") and periodic
cells of irregular, square or circular solids.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma, then two xor-shift-multiply mixes."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


def plates_mask(nx: int = 4, ny: int = 32) -> np.ndarray:
    """Two parallel plates: all cells gas; the walls sit just outside rows 0 and ny-1 (y not periodic)."""
    return np.zeros((ny, nx), dtype=np.uint8)


def rough_channel_mask(n: int = 128, height_frac: float = 0.2, width_frac: float = 0.25) -> np.ndarray:
    """Plates with one rectangular block per period on both walls.

    The period is n x n cells (Lx = H).  Each block is round(height_frac n) rows high and
    round(width_frac n) columns wide, centred at x = Lx/2, on the bottom and the top wall.
    """
    mask = np.zeros((n, n), dtype=np.uint8)
    hb = int(round(height_frac * n))
    wb = int(round(width_frac * n))
    x0 = n // 2 - wb // 2
    mask[:hb, x0:x0 + wb] = 1
    mask[n - hb:, x0:x0 + wb] = 1
    return mask


def porous_disks_mask(n: int = 256, porosity: float = 0.6, rmin: int = 8, rmax: int = 20,
                      seed: int = 1, gap: int = 1, max_reject: int = 100000):
    """Periodic n x n cell of random non-overlapping disks (both axes periodic).

    Disks with integer radius U{rmin..rmax} and centre U[0, n)^2 are added in sequence; a disk is
    rejected when its periodic centre distance to an earlier disk is below r1 + r2 + gap.  Adding
    stops when the gas fraction reaches the target.  A cell is solid when its centre lies inside a
    disk.  Returns (mask, achieved porosity).  Raises ValueError after max_reject rejections in a row.
    """
    rng = SplitMix64(seed)
    mask = np.zeros((n, n), dtype=np.uint8)
    disks = []
    yc, xc = np.mgrid[0:n, 0:n]
    xc = xc + 0.5
    yc = yc + 0.5
    rejects = 0
    while (1.0 - mask.mean()) > porosity:
        r = rng.randint(rmin, rmax)
        cx = rng.uniform() * n
        cy = rng.uniform() * n
        ok = True
        for (ox, oy, orad) in disks:
            dxp = abs(cx - ox)
            dyp = abs(cy - oy)
            dxp = min(dxp, n - dxp)
            dyp = min(dyp, n - dyp)
            if dxp * dxp + dyp * dyp < (r + orad + gap) ** 2:
                ok = False
                break
        if not ok:
            rejects += 1
            if rejects > max_reject:
                raise ValueError("porous_disks_mask: cannot reach the target porosity")
            continue
        rejects = 0
        disks.append((cx, cy, r))
        ddx = np.abs(xc - cx)
        ddy = np.abs(yc - cy)
        ddx = np.minimum(ddx, n - ddx)
        ddy = np.minimum(ddy, n - ddy)
        mask[(ddx * ddx + ddy * ddy) < r * r] = 1
    return mask, float(1.0 - mask.mean())


def porous_squares_mask(n: int = 256, porosity: float = 0.6, smin: int = 12, smax: int = 36, seed: int = 2,
                        gap: int = 2, max_reject: int = 100000):
    """Periodic n x n cell of non-overlapping axis-aligned square solids (the shape of medium 2 of Sec. III).

    Squares with integer side U{smin..smax} and lower-left cell U{0..n-1}^2 are added in sequence (both
    axes periodic); a square is rejected when one of its cells lies within `gap` cells (max norm) of an
    earlier square.  Adding stops when the gas fraction reaches the target.  Returns (mask, porosity).
    """
    rng = SplitMix64(seed)
    mask = np.zeros((n, n), dtype=np.uint8)
    halo = np.zeros((n, n), dtype=bool)  # earlier squares dilated by gap
    rejects = 0
    while (1.0 - mask.mean()) > porosity:
        side = rng.randint(smin, smax)
        x0 = rng.randint(0, n - 1)
        y0 = rng.randint(0, n - 1)
        xs = (x0 + np.arange(side)) % n
        ys = (y0 + np.arange(side)) % n
        if halo[np.ix_(ys, xs)].any():
            rejects += 1
            if rejects > max_reject:
                raise ValueError("porous_squares_mask: cannot reach the target porosity")
            continue
        rejects = 0
        mask[np.ix_(ys, xs)] = 1
        hx = (x0 - gap + np.arange(side + 2 * gap)) % n
        hy = (y0 - gap + np.arange(side + 2 * gap)) % n
        halo[np.ix_(hy, hx)] = True
    return mask, float(1.0 - mask.mean())


def porous_irregular_mask(n: int = 256, porosity: float = 0.6, corr: float = 10.0, seed: int = 3):
    """Periodic n x n cell of irregular solids (the kind of medium 1 of Sec. III): a Gaussian-filtered
    field of SplitMix64 uniforms (periodic, filter width `corr` cells) thresholded so that the gas
    fraction is the target; gas cells are the field's lowest values.  Raises ValueError when the gas
    does not connect across the cell along x1.  Returns (mask, porosity)."""
    rng = SplitMix64(seed)
    noise = np.array([rng.uniform() for _ in range(n * n)]).reshape(n, n) - 0.5
    k = np.fft.fftfreq(n)
    kern = np.exp(-2.0 * (math.pi * corr) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    field = np.real(np.fft.ifft2(np.fft.fft2(noise) * kern))
    order = np.argsort(field, axis=None, kind="stable")
    mask = np.ones(n * n, dtype=np.uint8)
    mask[order[: int(round(porosity * n * n))]] = 0
    mask = mask.reshape(n, n)
    if not percolates_x(mask):
        raise ValueError("porous_irregular_mask: the gas does not connect along x1; try another seed")
    return mask, float(1.0 - mask.mean())


def percolates_x(mask: np.ndarray, periodic_y: bool = True) -> bool:
    """Whether the gas of a cell periodic along x1 contains a path that winds once around x1.

    Breadth-first search over gas cells with 4-neighbours, tracking the unwrapped x1 coordinate of each
    visit: reaching a cell again at an unwrapped position differing by a multiple of nx closes such a path.
    """
    ny, nx = mask.shape
    seen = np.full((ny, nx), np.iinfo(np.int64).min, dtype=np.int64)
    for sj, si in zip(*np.nonzero(mask == 0)):
        if seen[sj, si] != np.iinfo(np.int64).min:
            continue
        seen[sj, si] = si
        queue = [(sj, si, si)]
        while queue:
            j, i, u = queue.pop()
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jj, uu = j + dj, u + di
                if not periodic_y and (jj < 0 or jj >= ny):
                    continue
                jj %= ny
                ii = uu % nx
                if mask[jj, ii]:
                    continue
                if seen[jj, ii] == np.iinfo(np.int64).min:
                    seen[jj, ii] = uu
                    queue.append((jj, ii, uu))
                elif seen[jj, ii] != uu:
                    return True
    return False


def wm_roughness(x: np.ndarray, D: float = 1.5, gamma: float = 1.5, n1: int = -4, n_max: int = 8) -> np.ndarray:
    """Weierstrass-Mandelbrot profile of Eq. (WM) with unit scale A: sum over n = n1 .. n_max of
    cos(2 pi gamma^n x) / gamma^((2 - D) n), x in units of H.  The paper sums to infinity; a grid
    resolves frequencies up to its Nyquist limit, so the caller truncates there."""
    r = np.zeros_like(np.asarray(x, dtype=np.float64))
    for n in range(n1, n_max + 1):
        r += np.cos(2.0 * math.pi * gamma ** n * x) / gamma ** ((2.0 - D) * n)
    return r


def couette_rough_mask(gap_cells: int = 100, aspect: float = 5.0, eps: float = 0.02, D: float = 1.5,
                       gamma: float = 1.5, n1: int = -4):
    """Staircase bottom wall with the WM roughness of Sec. II below a smooth top plate (Couette flow).

    The channel is aspect * H long and has a mean gap H = gap_cells cells; the profile of Eq. (WM) is
    sampled at the cell centres, truncated at the grid's Nyquist frequency (gamma^n <= 1 / (2 dx)),
    and scaled so that its root mean square is eps * H (Eq. for epsilon).  A cell is solid when its
    centre lies below base + r(x), with a base of whole rows under the deepest valley.
    Returns (mask [ny][nx], ly): ly = ny dx is the domain height to pass as the grid height.
    """
    dx = 1.0 / gap_cells
    nx = int(round(aspect * gap_cells))
    x = (np.arange(nx) + 0.5) * dx
    n_max = int(math.floor(math.log(1.0 / (2.0 * dx)) / math.log(gamma)))
    r = wm_roughness(x, D, gamma, n1, n_max)
    r *= eps / math.sqrt(float(np.mean(r * r)))
    base_rows = int(math.ceil(max(0.0, -float(r.min())) / dx)) + 1
    ny = gap_cells + base_rows
    yc = (np.arange(ny) + 0.5) * dx
    mask = (yc[:, None] < base_rows * dx + r[None, :]).astype(np.uint8)
    return mask, ny * dx


def couette_paper_grid(nx: int = 1500, band_rows: int = 60, rest_rows: int = 100, aspect: float = 5.0,
                       eps: float = 0.02, D: float = 1.5, gamma: float = 1.5, n1: int = -4):
    """The Couette channel of Sec. II on the paper's grid: nx equal columns over aspect * H, the rough
    band min r <= x2 < max r split into band_rows equal rows and max r <= x2 <= H into rest_rows.

    r is Eq. (WM) sampled at the column centres, truncated at the columns' Nyquist frequency, shifted
    to zero mean (the bottom plate's mean position is x2 = 0, the top plate at x2 = H = 1) and scaled to
    rms eps H.  A cell of the band is solid when its centre lies below r.  Returns (mask [ny][nx], row
    heights [ny] bottom to top, dx1); the grid spans x2 from min r to 1.
    """
    dx1 = aspect / nx
    x = (np.arange(nx) + 0.5) * dx1
    n_max = int(math.floor(math.log(1.0 / (2.0 * dx1)) / math.log(gamma)))
    r = wm_roughness(x, D, gamma, n1, n_max)
    r -= r.mean()
    r *= eps / math.sqrt(float(np.mean(r * r)))
    lo, hi = float(r.min()), float(r.max())
    dy = np.concatenate([np.full(band_rows, (hi - lo) / band_rows), np.full(rest_rows, (1.0 - hi) / rest_rows)])
    yc = lo + np.cumsum(dy) - 0.5 * dy
    mask = (yc[:, None] < r[None, :]).astype(np.uint8)
    return mask, dy, dx1


def couette_instance(kn: float, gap_cells: int = 100, aspect: float = 5.0, eps: float = 0.02, nv: int = 32,
                     rough: bool = True, grid: str = "square") -> Instance:
    """Couette flow of Sec. II: smooth top plate moving with U = 1 (in units of v_m), bottom plate at
    rest, rough (WM staircase) or smooth, x1 periodic, no body force; cubic nv x nv velocities.

    grid "square": square cells, gap_cells across the mean gap.  grid "paper": the paper's grid, 1500
    columns and 60 + 100 rows (couette_paper_grid) for the rough channel, 1500 x 100 equal rows for
    the smooth one (x1 spacing H / 300)."""
    if grid == "paper":
        nx = 1500
        if rough:
            mask, dy, dx1 = couette_paper_grid(nx, 60, 100, aspect, eps)
        else:
            mask, dy, dx1 = plates_mask(nx, 100), np.full(100, 0.01), aspect / nx
        name = f"couette{'_wm' if rough else '_smooth'}{nx}x{mask.shape[0]}_paper_cubic{nv}_kn{kn:g}"
        return Instance(name, mask, True, False, kn, ("cubic", nv, 4.0),
                        {"ly": float(dy.sum()), "top_u": 1.0, "force": 0.0, "eps": eps if rough else 0.0,
                         "dx1": dx1, "row_heights": dy})
    if rough:
        mask, ly = couette_rough_mask(gap_cells, aspect, eps)
    else:
        mask, ly = plates_mask(int(round(aspect * gap_cells)), gap_cells), 1.0
    name = f"couette{'_wm' if rough else '_smooth'}{mask.shape[1]}x{mask.shape[0]}_cubic{nv}_kn{kn:g}"
    return Instance(name, mask, True, False, kn, ("cubic", nv, 4.0),
                    {"ly": ly, "top_u": 1.0, "force": 0.0, "eps": eps if rough else 0.0})


def kn_to_delta(kn: float) -> float:
    """Rarefaction delta = sqrt(pi) / (2 Kn) (coefficient of the BGK operator); Kn = inf gives 0."""
    return 0.0 if math.isinf(kn) else math.sqrt(math.pi) / (2.0 * kn)


@dataclass
class Instance:
    """One solve: geometry, periodicity, Knudsen number and velocity grid."""

    name: str
    mask: np.ndarray
    periodic_x: bool
    periodic_y: bool
    kn: float
    quad: tuple            # (kind, n, vmax): kind in {"gh", "nc", "cubic"}
    extra: dict = field(default_factory=dict)


def plates_instance(kn: float = 0.1, nx: int = 4, ny: int = 32, nv: int = 12) -> Instance:
    """Force-driven Poiseuille flow between two diffuse plates; Gauss-Hermite nv x nv velocities."""
    return Instance(f"plates{nx}x{ny}_gh{nv}_kn{kn:g}", plates_mask(nx, ny), True, False, kn, ("gh", nv, 0.0))


def rough_instance(kn: float, n: int = 128, nv: int = 32, vmax: float = 5.0) -> Instance:
    """Rough channel, n x n cells, trapezoid Newton-Cotes nv x nv velocities on [-vmax, vmax]."""
    return Instance(f"rough{n}_nc{nv}_kn{kn:g}", rough_channel_mask(n), True, False, kn, ("nc", nv, vmax))


def porous_instance(kn: float, n: int = 256, nv: int = 48, porosity: float = 0.6, seed: int = 1,
                    rmin: int = 8, rmax: int = 20) -> Instance:
    """Periodic disk medium, n x n cells, cubic nv x nv velocities (Eq. nonuniform_v)."""
    mask, phi = porous_disks_mask(n, porosity, rmin, rmax, seed)
    return Instance(f"porous{n}_phi{porosity:g}_s{seed}_cubic{nv}_kn{kn:g}", mask, True, True, kn,
                    ("cubic", nv, 4.0), {"porosity": phi, "seed": seed})


MEDIA = ("irregular", "squares", "disks")


def medium_mask(kind: str, n: int = 256, porosity: float = 0.6):
    """The three synthetic media standing in for media 1-3 of Sec. III (irregular, square and circular
    solids), n x n cells over the height H, periodic in both axes, a dozen grains or fewer (pores of
    about 0.1 H); feature sizes scale with n / 256.  Grains are added until the gas fraction is at or
    below `porosity`; the achieved value is returned with the mask."""
    f = n / 256.0
    if kind == "irregular":
        return porous_irregular_mask(n, porosity, corr=20.0 * f, seed=3)
    if kind == "squares":
        return porous_squares_mask(n, porosity, max(3, int(round(32 * f))), max(4, int(round(80 * f))), seed=2,
                                   gap=max(1, int(round(4 * f))))
    if kind == "disks":
        return porous_disks_mask(n, porosity, max(3, int(round(20 * f))), max(4, int(round(48 * f))), seed=1,
                                 gap=max(1, int(round(2 * f))))
    raise ValueError(f"unknown medium {kind!r}")


def refine_mask(mask: np.ndarray, factor: int) -> np.ndarray:
    """The same staircase geometry on a grid `factor` times finer: every cell becomes factor x factor."""
    return np.kron(np.asarray(mask, dtype=np.uint8), np.ones((factor, factor), dtype=np.uint8))


def medium_instance(kind: str, kn: float, n: int = 256, nv: int = 32, porosity: float = 0.6) -> Instance:
    """Force-driven (Poiseuille) flow through one synthetic medium, cubic nv x nv velocities."""
    mask, phi = medium_mask(kind, n, porosity)
    return Instance(f"{kind}{n}_phi{porosity:g}_cubic{nv}_kn{kn:g}", mask, True, True, kn, ("cubic", nv, 4.0),
                    {"porosity": phi, "medium": kind})


def batched_instances(count: int = 64, seed0: int = 0):
    """Mixed batch: side in {64..256}, rough or porous, Kn log-uniform in [0.01, 10], cubic Nv in {16..48}.

    Instance i uses SplitMix64(seed0 + i) for every choice.  Porous media have porosity U[0.6, 0.75]
    and disk radii scaled by side/256 (at least 4 cells), so that small cells still reach the target.
    """
    sides = [64, 96, 128, 192, 256]
    nvs = [16, 24, 32, 40, 48]
    out = []
    for i in range(count):
        rng = SplitMix64(seed0 + i)
        side = sides[rng.randint(0, len(sides) - 1)]
        nv = nvs[rng.randint(0, len(nvs) - 1)]
        kn = 10.0 ** (-2.0 + 3.0 * rng.uniform())
        if rng.uniform() < 0.5:
            inst = Instance(f"b{i}_rough{side}_cubic{nv}_kn{kn:.4g}", rough_channel_mask(side), True, False,
                            kn, ("cubic", nv, 4.0))
        else:
            phi = 0.6 + 0.15 * rng.uniform()
            rmin = max(4, int(round(8 * side / 256)))
            rmax = max(rmin + 1, int(round(20 * side / 256)))
            mask, ach = porous_disks_mask(side, phi, rmin, rmax, seed=1000 + i)
            inst = Instance(f"b{i}_porous{side}_cubic{nv}_kn{kn:.4g}", mask, True, True, kn,
                            ("cubic", nv, 4.0), {"porosity": ach})
        out.append(inst)
    return out


def sample_gas_cells(mask: np.ndarray, count: int, seed: int = 7) -> np.ndarray:
    """count distinct gas-cell flat indices drawn with SplitMix64 (partial Fisher-Yates)."""
    gas = np.flatnonzero(mask.ravel() == 0)
    rng = SplitMix64(seed)
    gas = gas.copy()
    count = min(count, len(gas))
    for t in range(count):
        j = t + int(rng.uniform() * (len(gas) - t))
        gas[t], gas[j] = gas[j], gas[t]
    return np.sort(gas[:count])
