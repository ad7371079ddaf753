"""Direct dense solve of the discrete DVM equations on tiny grids (second route to the fixed point).

TEST INFRASTRUCTURE ONLY.  Written independently of ``dvm_oracle.c``: it assembles the steady
discrete equations of Sec. II.A (Eq. BGK with the time derivative dropped, Eq. diffuse2 walls,
periodic ends, second-order upwind differences -- linear through the wall-face value in the cell
next to a wall, first order in the cell after it) as one matrix and solves it with LAPACK, with no
iteration, no lagging and no sweep order.  Unknowns: h[k, g] for every velocity k and gas cell g,
plus the scalar c that borders the system:

    (delta_c + v.D) h_k - delta_c M_k(h) + delta_c c = F v1_k      (every gas cell, velocity)
    sum_gas sum_k W_k h_k = 0                                       (mean density zero)

with M_k(h) = sum_j W_j psi(v_k)^T G^{-1} psi(v_j) h_j, psi = (1, v1, v2, |v|^2), G the quadrature
Gram matrix of psi: the projection of h onto the collision invariants, which for an exact quadrature
is rho + 2 u.v + tau (|v|^2 - 1) with the moments rho, u, tau of Sec. II.A.  Wall values h_w = alpha rho_w + (1 - alpha) h(mirror v), with
rho_w = sum_{v.n<0} |v.n| W h / sum_{v.n>0} (v.n) W at the gas cell owning the face; the plate beyond
the last row may move along x1 with speed U (Couette flow, Eq. diffuse1), adding alpha 2 U v1 to its
wall value (a source term of the system).  Rows may have unequal heights (x2 spacing of Sec. II.A):
each upwind derivative is then the derivative at the cell centre of the polynomial through the
points the stencil uses (the cell centre, the upstream centres, or the wall face), its weights found
by solving the small Vandermonde system of that polynomial.
"""
from __future__ import annotations

import numpy as np


def _solid(mask, px, py, i, j):
    ny, nx = mask.shape
    if i < 0 or i >= nx:
        if not px:
            return True
        i %= nx
    if j < 0 or j >= ny:
        if not py:
            return True
        j %= ny
    return bool(mask[j, i])


def derivative_weights(offsets):
    """Weights w with sum_m w_m p(t_m) = p'(0) for every polynomial p of degree len - 1 through the
    points t_m (t_0 = 0, the cell centre)."""
    t = np.asarray(offsets, dtype=np.float64)
    V = np.vander(t, len(t), increasing=True).T  # rows: 1, t, t^2 evaluated at the points
    rhs = np.zeros(len(t))
    if len(t) > 1:
        rhs[1] = 1.0
    return np.linalg.solve(V, rhs)


def collision_kernel(v1, v2, W, collision="projection"):
    """C[k, j] with M_k(h) = sum_j C[k, j] h_j.

    projection: C[k, j] = W_j psi(v_k)^T G^{-1} psi(v_j) (the W-orthogonal projection onto the
    collision invariants); literal: Eq. BGK as printed, rho + 2 u.v_k + tau (|v_k|^2 - 1) with
    rho = sum W h, u = sum W v h, tau = sum W (|v|^2 - 1) h, i.e.
    C[k, j] = W_j [1 + 2 v_k . v_j + (|v_k|^2 - 1)(|v_j|^2 - 1)]."""
    if collision == "literal":
        e = v1 * v1 + v2 * v2 - 1.0
        return (1.0 + 2.0 * (np.outer(v1, v1) + np.outer(v2, v2)) + np.outer(e, e)) * W[None, :]
    psi = np.stack([np.ones_like(v1), v1, v2, v1 * v1 + v2 * v2])  # [4][K]
    G = (psi * W[None, :]) @ psi.T
    return (psi.T @ np.linalg.inv(G) @ psi) * W[None, :]


def assemble(prob):
    """Dense bordered matrix B and right-hand side b; also the gas-cell index map."""
    mask = prob.mask
    ny, nx = mask.shape
    px, py = prob.periodic_x, prob.periodic_y
    v1, v2, W = prob.velocities()
    K = len(W)
    gas_cells = [(i, j) for j in range(ny) for i in range(nx) if not mask[j, i]]
    gid = {cell: g for g, cell in enumerate(gas_cells)}
    G = len(gas_cells)
    n = K * G
    idx = lambda k, g: k * G + g
    B = np.zeros((n + 1, n + 1))
    b = np.zeros(n + 1)
    dx = prob.dx
    rows = prob.row_heights()
    nv = prob.nv
    Ckern = collision_kernel(v1, v2, W, getattr(prob, "collision", "projection"))
    # wall normalisers per side: W (normal +x), E (-x), S (+y), N (-y)
    normal = {"W": (1.0, 0.0), "E": (-1.0, 0.0), "S": (0.0, 1.0), "N": (0.0, -1.0)}
    vn = {s: v1 * nxy[0] + v2 * nxy[1] for s, nxy in normal.items()}
    norm = {s: float(np.sum(np.where(vn[s] > 0, vn[s] * W, 0.0))) for s in normal}

    def mirror(k, side):
        a, bb = divmod(k, nv)
        if side in ("W", "E"):
            a = nv - 1 - a
        else:
            bb = nv - 1 - bb
        return a * nv + bb

    def add_wall(row, coef, owner_g, side, k):
        # coef multiplies h_w on the right-hand side -> -coef on the left
        inc = np.flatnonzero(vn[side] < 0)
        for j in inc:
            B[row, idx(j, owner_g)] -= coef * prob.alpha * (-vn[side][j]) * W[j] / norm[side]
        if prob.alpha < 1.0:
            B[row, idx(mirror(k, side), owner_g)] -= coef * (1.0 - prob.alpha)

    for g, (i, j) in enumerate(gas_cells):
        d = prob.delta[j, i]
        for k in range(K):
            row = idx(k, g)
            diag = d
            src = prob.force * v1[k]
            for axis in (0, 1):
                va = v1[k] if axis == 0 else v2[k]
                s = 1 if va > 0 else -1
                di, dj = (1, 0) if axis == 0 else (0, 1)
                side = ("W" if s > 0 else "E") if axis == 0 else ("S" if s > 0 else "N")
                i1, j1 = i - s * di, j - s * dj
                i2, j2 = i - 2 * s * di, j - 2 * s * dj
                # cell sizes along the axis at the cell and its two upstream neighbours
                size = (lambda jj: dx) if axis == 0 else (lambda jj: rows[jj % ny])
                h0, h1, h2 = size(j), size(j1), size(j2)
                # v_a dh/dx_a = |v_a| (dh/dt at t = 0), t the distance against the flow direction
                if _solid(mask, px, py, i1, j1):
                    # the polynomial through the wall face (t = -h0/2) and the cell centre
                    w = derivative_weights([0.0, -0.5 * h0])
                    diag += abs(va) * w[0]
                    add_wall(row, -abs(va) * w[1], g, side, k)
                    if side == "N" and not py and j == ny - 1 and prob.top_u != 0.0:
                        # the moving plate's wall value carries the drift 2 U v1 (Eq. diffuse1)
                        src += -abs(va) * w[1] * prob.alpha * 2.0 * prob.top_u * v1[k]
                elif _solid(mask, px, py, i2, j2):
                    # second cell from a wall: first-order upwind through the gas neighbour
                    w = derivative_weights([0.0, -0.5 * (h0 + h1)])
                    diag += abs(va) * w[0]
                    g1 = gid[(i1 % nx, j1 % ny)]
                    B[row, idx(k, g1)] += abs(va) * w[1]
                else:
                    t1 = -0.5 * (h0 + h1)
                    w = derivative_weights([0.0, t1, t1 - 0.5 * (h1 + h2)])
                    diag += abs(va) * w[0]
                    g1 = gid[(i1 % nx, j1 % ny)]
                    g2 = gid[(i2 % nx, j2 % ny)]
                    B[row, idx(k, g1)] += abs(va) * w[1]
                    B[row, idx(k, g2)] += abs(va) * w[2]
            B[row, idx(k, g)] += diag
            # collision: -delta M_k(h) at this cell
            for jv in range(K):
                B[row, idx(jv, g)] -= d * Ckern[k, jv]
            B[row, n] += d
            b[row] = src
    for g in range(G):
        for k in range(K):
            B[n, idx(k, g)] = W[k]
    return B, b, gas_cells


def solve(prob):
    """Direct solution: h [K][ny][nx] (0 in solid cells), c, Q, and the assembled system."""
    B, b, gas_cells = assemble(prob)
    ny, nx = prob.mask.shape
    K = prob.nv * prob.nv
    G = len(gas_cells)
    if np.all(prob.delta == 0.0):
        # free-molecular: the bordering column vanishes; solve the consistent system without c
        x_h, *_ = np.linalg.lstsq(B[:, :-1], b, rcond=None)
        x = np.append(x_h, 0.0)
    else:
        x = np.linalg.solve(B, b)
    h = np.zeros((K, ny, nx))
    for g, (i, j) in enumerate(gas_cells):
        h[:, j, i] = x[np.arange(K) * G + g]
    v1, v2, W = prob.velocities()
    u1 = np.tensordot(W * v1, h, axes=(0, 0))
    area = prob.dx * prob.row_heights()[:, None] * np.ones((1, nx))
    Q = float((u1 * area)[prob.mask == 0].sum() / (nx * prob.dx))
    return dict(h=h, c=float(x[-1]), Q=Q, B=B, b=b, x=x, gas_cells=gas_cells)


def adjoint_gradient(prob, sol=None):
    """dQ/d delta_c from the transposed bordered system B^T Lambda = [g; 0].

    dQ/d delta_c = -sum_k Lambda[k, c] (h_kc - M_kc(h) + c), the derivative of the rows of cell c.
    """
    if sol is None:
        sol = solve(prob)
    B, x, gas_cells = sol["B"], sol["x"], sol["gas_cells"]
    ny, nx = prob.mask.shape
    v1, v2, W = prob.velocities()
    K = len(W)
    G = len(gas_cells)
    n = K * G
    g = np.zeros(n + 1)
    rows = prob.row_heights()
    dA_over_L = np.array([prob.dx * rows[j] / (nx * prob.dx) for (i, j) in gas_cells])  # dA = dx dy_j
    for k in range(K):
        g[k * G:(k + 1) * G] = W[k] * v1[k] * dA_over_L
    lam = np.linalg.solve(B.T, g)
    Ckern = collision_kernel(v1, v2, W, getattr(prob, "collision", "projection"))
    grad = np.zeros((ny, nx))
    c = x[-1]
    for gi, (i, j) in enumerate(gas_cells):
        hc = x[np.arange(K) * G + gi]
        Mc = Ckern @ hc
        grad[j, i] = -np.dot(lam[np.arange(K) * G + gi], hc - Mc + c)
    return grad
