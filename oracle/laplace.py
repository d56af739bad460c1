"""Elastance oracle (FP64, dense Nystrom matrix + LU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's steps (Section 3):
  1. sigma_i = q_i / |Gamma_i| on Gamma_i                       (eq. sigma)
  2. K_ij sigma(x) = int_{Gamma_j} dG(x,y)/dn_x sigma(y) ds_y,   G = -(1/2pi) log|x-y|
     i.e. the normal derivative at the TARGET x (Section 3.4, operators K_ij, K_ii)
  3. L_i mu(x) = int_{Gamma_i} mu ds                              (eq. ModRep2)
  4. solve (1/2 I + K + L) mu = -(1/2 I + K) sigma               (eq. ModRep2)
  5. u = S_Gamma(mu + sigma); u is constant in each D_i and equals phi_i (eq. TotRepresentation)

Nystrom entries with r = x_a - x_b (target minus source) and trapezoid weight w_b:
  K[a, b] = w_b * (-(1/2pi) (r . n_a) / |r|^2)   for a != b
  K[a, a] = w_a * (-kappa_a / (4 pi))            (the smooth diagonal limit)
  L[a, b] = w_b  if body(a) == body(b) else 0
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import geometry

INV_2PI = 1.0 / (2.0 * math.pi)


def kernel_rows(geo: dict, rows: np.ndarray) -> np.ndarray:
    """Rows `rows` of the discrete K (weights included), shape [len(rows), M]."""
    rows = np.asarray(rows)
    rx = geo["x"][rows, None] - geo["x"][None, :]
    ry = geo["y"][rows, None] - geo["y"][None, :]
    r2 = rx * rx + ry * ry
    rn = rx * geo["nx"][rows, None] + ry * geo["ny"][rows, None]
    self_mask = rows[:, None] == np.arange(geo["M"])[None, :]
    r2 = np.where(self_mask, 1.0, r2)
    k = -INV_2PI * rn / r2
    k[self_mask] = -geo["kappa"][rows] / (4.0 * math.pi)
    return k * geo["w"][None, :]


def completion_rows(geo: dict, rows: np.ndarray) -> np.ndarray:
    """Rows of the discrete completion operator L (weights included)."""
    rows = np.asarray(rows)
    same = geo["body"][rows, None] == geo["body"][None, :]
    return np.where(same, geo["w"][None, :], 0.0)


def kernel_matrix(geo: dict) -> np.ndarray:
    return kernel_rows(geo, np.arange(geo["M"]))


def operator_matrix(geo: dict, block: int = 1024) -> np.ndarray:
    """Dense 1/2 I + K + L (unscaled unknowns).

    Filled row block by row block into one M x M array, so that the
    temporaries of the entry formulas stay block x M (M = 25,600 needs 5.2 GB
    for the matrix itself and no more than a few hundred MB besides).
    """
    M = geo["M"]
    A = np.empty((M, M))
    for s in range(0, M, block):
        rows = np.arange(s, min(M, s + block))
        blk = kernel_rows(geo, rows)
        blk[np.arange(rows.size), rows] += 0.5
        blk += completion_rows(geo, rows)
        A[rows] = blk
    return A


def apply(geo: dict, v: np.ndarray, with_L: bool = True, block: int = 2048) -> np.ndarray:
    """(1/2 I + K [+ L]) v, row block by row block (no full matrix held)."""
    M = geo["M"]
    out = np.empty(M)
    for s in range(0, M, block):
        rows = np.arange(s, min(M, s + block))
        A = kernel_rows(geo, rows)
        if with_L:
            A += completion_rows(geo, rows)
        out[rows] = 0.5 * v[rows] + A @ v
    return out


def incident_density(geo: dict, q: np.ndarray) -> np.ndarray:
    """sigma_a = q_i / |Gamma_i| for a on Gamma_i (eq. sigma)."""
    return np.asarray(q, dtype=np.float64)[geo["body"]] / geo["length"][geo["body"]]


def rhs(geo: dict, sigma: np.ndarray) -> np.ndarray:
    """b = -(1/2 I + K) sigma (right-hand side of eq. ModRep2)."""
    return -apply(geo, sigma, with_L=False)


def single_layer_at(geo: dict, density: np.ndarray, px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """S_Gamma density evaluated at off-surface points: sum_b w_b G(p, x_b) density_b."""
    rx = np.asarray(px)[:, None] - geo["x"][None, :]
    ry = np.asarray(py)[:, None] - geo["y"][None, :]
    G = -INV_2PI * 0.5 * np.log(rx * rx + ry * ry)
    return G @ (geo["w"] * density)


def solve(g: dict, q: np.ndarray) -> dict:
    """Full elastance solve: charges q [N] -> potentials phi [N] (plus densities)."""
    geo = geometry.nodes(g)
    sigma = incident_density(geo, q)
    A = operator_matrix(geo)
    b = rhs(geo, sigma)
    # LU with partial pivoting, factored in place (A is not used again)
    mu = sla.lu_solve(sla.lu_factor(A, overwrite_a=True, check_finite=False), b, check_finite=False)
    del A
    pts = geometry.interior_points(geo)
    phi = single_layer_at(geo, mu + sigma, pts["z0x"], pts["z0y"])
    return dict(phi=phi, mu=mu, sigma=sigma, nu=mu + sigma, b=b, geo=geo)


def potentials_from_density(g: dict, nu: np.ndarray) -> np.ndarray:
    """phi_i = S_Gamma(nu)(z_i) at each body's interior point z_i."""
    geo = geometry.nodes(g)
    pts = geometry.interior_points(geo)
    return single_layer_at(geo, nu, pts["z0x"], pts["z0y"])


def elastance_matrix(g: dict) -> np.ndarray:
    """P[:, j] = phi for q = e_j (free-space log gauge for non-neutral q)."""
    geo = geometry.nodes(g)
    A = operator_matrix(geo)
    lu = sla.lu_factor(A)
    pts = geometry.interior_points(geo)
    N = geo["N"]
    P = np.empty((N, N))
    for j in range(N):
        q = np.zeros(N)
        q[j] = 1.0
        sigma = incident_density(geo, q)
        mu = sla.lu_solve(lu, rhs(geo, sigma))
        P[:, j] = single_layer_at(geo, mu + sigma, pts["z0x"], pts["z0y"])
    return P
