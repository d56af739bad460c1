"""Mobility oracle (FP64, dense Nystrom matrix + LU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's steps (Section 4, viscosity 1):
  1. rho_j = F_j/|Gamma_j| + T_j (x - x^c_j)^perp / W_j                (eq. rho)
  2. (K rho)_k(x) = n_{x,l} int T_{kml}(x,y) rho_m(y) ds_y,
     T_{ijk}(x,y) = -(1/pi) r_i r_j r_k / |r|^4, r = x - y             (stresslet, Section 4.1)
  3. L_i mu(x) = int_{Gamma_i} mu ds + (x - x^c_i)^perp int ((y - x^c_i)^perp, mu) ds
                                                                       (eq. ModRep2Stokes)
  4. solve (1/2 I + K + L) mu = -(1/2 I + K) rho
  5. u = S_Gamma(mu + rho) with the Stokeslet G_ij = (1/4pi)[-log|r| d_ij + r_i r_j/|r|^2];
     inside D_i, u = v_i + omega_i (x - x^c_i)^perp                      (eq. TotRepresentationStokes)

Unknowns are node-interleaved: entry 2a + c is component c of node a.
Nystrom 2x2 blocks with r = x_a - x_b and trapezoid weight w_b:
  K[a, b] = w_b * (-(1/pi) r r^T (r . n_a) / |r|^4)   for a != b
  K[a, a] = w_a * (-(kappa_a / (2 pi)) tau_a tau_a^T)  (the smooth diagonal limit)
  L[a, b] = w_b (I + p_a p_b^T), p = (x - x^c)^perp,   if body(a) == body(b)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import geometry

INV_PI = 1.0 / math.pi


def perp(geo: dict) -> tuple[np.ndarray, np.ndarray]:
    """(x - x^c_body)^perp = (-(x2 - c2), x1 - c1) at every node."""
    b = geo["body"]
    return -(geo["y"] - geo["yc"][b]), geo["x"] - geo["xc"][b]


def kernel_rows(geo: dict, rows: np.ndarray) -> np.ndarray:
    """Node rows `rows` of the discrete traction operator, shape [2*len(rows), 2M]."""
    rows = np.asarray(rows)
    M = geo["M"]
    rx = geo["x"][rows, None] - geo["x"][None, :]
    ry = geo["y"][rows, None] - geo["y"][None, :]
    r2 = rx * rx + ry * ry
    rn = rx * geo["nx"][rows, None] + ry * geo["ny"][rows, None]
    self_mask = rows[:, None] == np.arange(M)[None, :]
    r2 = np.where(self_mask, 1.0, r2)
    c = -INV_PI * rn / (r2 * r2)
    kxx, kxy, kyy = c * rx * rx, c * rx * ry, c * ry * ry
    # diagonal limit -(kappa/2pi) tau tau^T
    ia = np.nonzero(self_mask)
    kap = -geo["kappa"][rows] / (2.0 * math.pi)
    tx, ty = geo["tx"][rows], geo["ty"][rows]
    kxx[ia] = kap * tx * tx
    kxy[ia] = kap * tx * ty
    kyy[ia] = kap * ty * ty
    w = geo["w"][None, :]
    out = np.empty((2 * rows.size, 2 * M))
    out[0::2, 0::2] = kxx * w
    out[0::2, 1::2] = kxy * w
    out[1::2, 0::2] = kxy * w
    out[1::2, 1::2] = kyy * w
    return out


def completion_rows(geo: dict, rows: np.ndarray) -> np.ndarray:
    """Node rows of the discrete completion operator L, shape [2*len(rows), 2M]."""
    rows = np.asarray(rows)
    M = geo["M"]
    same = (geo["body"][rows, None] == geo["body"][None, :]).astype(np.float64)
    px, py = perp(geo)
    w = geo["w"][None, :]
    out = np.zeros((2 * rows.size, 2 * M))
    out[0::2, 0::2] = same * w * (1.0 + px[rows, None] * px[None, :])
    out[0::2, 1::2] = same * w * (px[rows, None] * py[None, :])
    out[1::2, 0::2] = same * w * (py[rows, None] * px[None, :])
    out[1::2, 1::2] = same * w * (1.0 + py[rows, None] * py[None, :])
    return out


def operator_matrix(geo: dict, block: int = 512) -> np.ndarray:
    """Dense 1/2 I + K + L, [2M, 2M], filled node-row block by block."""
    M = geo["M"]
    A = np.empty((2 * M, 2 * M))
    for s in range(0, M, block):
        rows = np.arange(s, min(M, s + block))
        blk = kernel_rows(geo, rows)
        blk[np.arange(2 * rows.size), 2 * rows[0] + np.arange(2 * rows.size)] += 0.5
        blk += completion_rows(geo, rows)
        A[2 * rows[0]:2 * rows[-1] + 2] = blk
    return A


def apply(geo: dict, v: np.ndarray, with_L: bool = True, block: int = 1024, workers: int = 1) -> np.ndarray:
    """(1/2 I + K [+ L]) v for an interleaved [2M] vector, row block by row block.

    workers > 1 computes the row blocks on that many threads (each block is
    independent; numpy releases the interpreter lock in its array loops).
    """
    M = geo["M"]
    out = np.empty(2 * M)

    def one(s):
        rows = np.arange(s, min(M, s + block))
        A = kernel_rows(geo, rows)
        if with_L:
            A += completion_rows(geo, rows)
        sl = slice(2 * rows[0], 2 * rows[-1] + 2)
        out[sl] = 0.5 * v[sl] + A @ v

    starts = range(0, M, block)
    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(one, starts))
    else:
        for s in starts:
            one(s)
    return out


def incident_density(geo: dict, FT: np.ndarray) -> np.ndarray:
    """rho_a = F_i/|Gamma_i| + T_i (x_a - x^c_i)^perp / W_i, interleaved [2M] (eq. rho)."""
    FT = np.asarray(FT, dtype=np.float64).reshape(-1, 3)
    b = geo["body"]
    px, py = perp(geo)
    rho = np.empty(2 * geo["M"])
    rho[0::2] = FT[b, 0] / geo["length"][b] + FT[b, 2] * px / geo["W"][b]
    rho[1::2] = FT[b, 1] / geo["length"][b] + FT[b, 2] * py / geo["W"][b]
    return rho


def rhs(geo: dict, rho: np.ndarray) -> np.ndarray:
    """b = -(1/2 I + K) rho (right-hand side of eq. ModRep2Stokes)."""
    return -apply(geo, rho, with_L=False)


def single_layer_at(geo: dict, density: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """Stokes single layer S_Gamma density at off-surface points, shape [len(px), 2]."""
    rx = np.asarray(px)[:, None] - geo["x"][None, :]
    ry = np.asarray(py)[:, None] - geo["y"][None, :]
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    f1 = geo["w"] * density[0::2]
    f2 = geo["w"] * density[1::2]
    s = 1.0 / (4.0 * math.pi)
    u1 = s * ((lg + rx * rx / r2) @ f1 + (rx * ry / r2) @ f2)
    u2 = s * ((rx * ry / r2) @ f1 + (lg + ry * ry / r2) @ f2)
    return np.stack([u1, u2], axis=1)


def rigid_motion(geo: dict, nu: np.ndarray) -> np.ndarray:
    """(v_x, v_y, omega) per body from u = S(nu) at z0, z0 + delta e1, z0 + delta e2.

    For a rigid field u = v + omega (x - z0)^perp these three points give v
    exactly and omega = [(u2(z1) - u2(z0)) - (u1(z2) - u1(z0))] / (2 delta).
    """
    pts = geometry.interior_points(geo)
    z0x, z0y, d = pts["z0x"], pts["z0y"], pts["delta"]
    u0 = single_layer_at(geo, nu, z0x, z0y)
    u1 = single_layer_at(geo, nu, z0x + d, z0y)
    u2 = single_layer_at(geo, nu, z0x, z0y + d)
    om = ((u1[:, 1] - u0[:, 1]) - (u2[:, 0] - u0[:, 0])) / (2.0 * d)
    return np.stack([u0[:, 0], u0[:, 1], om], axis=1)


def solve(g: dict, FT: np.ndarray) -> dict:
    """Full mobility solve: (F, T) [N, 3] -> (v_x, v_y, omega) [N, 3] (plus densities)."""
    geo = geometry.nodes(g)
    rho = incident_density(geo, FT)
    A = operator_matrix(geo)
    b = rhs(geo, rho)
    mu = sla.lu_solve(sla.lu_factor(A, overwrite_a=True, check_finite=False), b, check_finite=False)
    del A
    UW = rigid_motion(geo, mu + rho)
    return dict(UW=UW, mu=mu, rho=rho, nu=mu + rho, b=b, geo=geo)


def solve_gmres(g: dict, FT: np.ndarray, tol: float = 1e-13, restart: int = 200, workers: int = 1,
                block: int = 256, precond: bool = True) -> dict:
    """Mobility solve without the dense matrix, for systems too large to hold.

    The same discrete equation as `solve` (eq. ModRep2Stokes: rho, the right-hand
    side -(1/2 I + K) rho, the operator 1/2 I + K + L and the rigid-motion read
    out), with the LU step replaced by restarted GMRES (scipy) on the operator
    applied row block by row block, from x = 0.  With precond, GMRES runs with
    the block-Jacobi preconditioner (each body's own diagonal block of the
    operator, factored by LU); it changes the iteration count, not the
    solution.  The true residual b - A mu is recomputed after every GMRES run
    and, while ||b - A mu|| > tol ||b||, GMRES is run again on it and the
    correction added (FP64 iterative refinement).  The final true relative
    residual is returned.
    """
    from scipy.sparse.linalg import LinearOperator, gmres

    geo = geometry.nodes(g)
    rho = incident_density(geo, FT)
    n = 2 * geo["M"]
    bs = geo["body_start"]
    b = -apply(geo, rho, with_L=False, block=block, workers=workers)
    count = [0]

    def mv(v):
        count[0] += 1
        return apply(geo, np.asarray(v).reshape(-1), block=block, workers=workers)

    A = LinearOperator((n, n), matvec=mv, dtype=np.float64)
    Minv = None
    if precond:
        lus = []
        for i in range(geo["N"]):
            rows = np.arange(bs[i], bs[i + 1])
            blk = (kernel_rows(geo, rows) + completion_rows(geo, rows))[:, 2 * bs[i]:2 * bs[i + 1]]
            blk += 0.5 * np.eye(2 * rows.size)
            lus.append(sla.lu_factor(blk))

        def pv(v):
            v = np.asarray(v).reshape(-1)
            z = np.empty_like(v)
            for i, lu in enumerate(lus):
                sl = slice(2 * bs[i], 2 * bs[i + 1])
                z[sl] = sla.lu_solve(lu, v[sl])
            return z

        Minv = LinearOperator((n, n), matvec=pv, dtype=np.float64)
    mu = np.zeros(n)
    r = b.copy()
    bn = np.linalg.norm(b)
    rel = 1.0
    flags = []
    for _ in range(6):
        d, flag = gmres(A, r, rtol=0.1 * tol * bn / max(np.linalg.norm(r), 1e-300), atol=0.0, restart=restart,
                        maxiter=50, M=Minv)
        flags.append(int(flag))
        mu = mu + d
        r = b - apply(geo, mu, block=block, workers=workers)
        rel = float(np.linalg.norm(r) / bn)
        if rel <= tol:
            break
    UW = rigid_motion(geo, mu + rho)
    return dict(UW=UW, mu=mu, rho=rho, nu=mu + rho, b=b, geo=geo, rel_residual=rel, matvecs=count[0],
                flags=flags)


def motion_from_density(g: dict, nu: np.ndarray) -> np.ndarray:
    return rigid_motion(geometry.nodes(g), nu)


def mobility_matrix(g: dict) -> np.ndarray:
    """Mob[:, j] = (v, omega) stacked per body for the unit load e_j (log gauge)."""
    geo = geometry.nodes(g)
    A = operator_matrix(geo)
    lu = sla.lu_factor(A)
    N = geo["N"]
    Mob = np.empty((3 * N, 3 * N))
    for j in range(3 * N):
        FT = np.zeros(3 * N)
        FT[j] = 1.0
        rho = incident_density(geo, FT)
        mu = sla.lu_solve(lu, rhs(geo, rho))
        Mob[:, j] = rigid_motion(geo, mu + rho).reshape(-1)
    return Mob
