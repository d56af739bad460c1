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


def operator_matrix(geo: dict) -> np.ndarray:
    M = geo["M"]
    idx = np.arange(M)
    return 0.5 * np.eye(2 * M) + kernel_rows(geo, idx) + completion_rows(geo, idx)


def apply(geo: dict, v: np.ndarray, with_L: bool = True, block: int = 1024) -> np.ndarray:
    """(1/2 I + K [+ L]) v for an interleaved [2M] vector, row block by row block."""
    M = geo["M"]
    out = np.empty(2 * M)
    for s in range(0, M, block):
        rows = np.arange(s, min(M, s + block))
        A = kernel_rows(geo, rows)
        if with_L:
            A += completion_rows(geo, rows)
        sl = slice(2 * rows[0], 2 * rows[-1] + 2)
        out[sl] = 0.5 * v[sl] + A @ v
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
    mu = sla.lu_solve(sla.lu_factor(A), b)
    UW = rigid_motion(geo, mu + rho)
    return dict(UW=UW, mu=mu, rho=rho, nu=mu + rho, b=b, geo=geo)


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
