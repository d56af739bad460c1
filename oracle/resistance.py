"""Resistance oracle (FP64, dense Nystrom matrix + LU): the other half of the
paper's mobility round trip (Section 6.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Prescribed rigid motions u = v_i + omega_i (x - x^c_i)^perp on the boundaries
Gamma_i give the forces F_i and torques T_i (about x^c_i) that the bodies
exert on the fluid (viscosity 1) and the velocity at infinity u_inf of the
bounded Stokes flow with these boundary values (so sum_i F_i = 0).  The paper
solves this problem by an integral equation that is not the inverse of its
mobility equations, and checks that the mobility solve driven by these forces
and torques returns the prescribed motions (velocities less u_inf).  This
module takes a classical exterior Dirichlet representation:

  u(x) = D[mu](x) + sum_i (G(x - z_i) F_i + R(x - z_i) T_i) + u_inf,
  D[mu](x) = (1/pi) int r r^T (r . n_y) / |r|^4 mu(y) ds_y,   r = x - y  (stresslet, source normal)
  G(r) = (1/4pi) (-log|r| I + r r^T / |r|^2)                            (Stokeslet)
  R(r) T = (T / 4pi) r^perp / |r|^2                                     (rotlet)

with z_i = x^c_i.  This D gives -c inside a curve for a constant density c,
0 outside and -c/2 on it, so the exterior boundary value is (D + 1/2 I) mu; it
annihilates the rigid motions of any one body, so the density is taken
orthogonal to them (int mu ds = 0, int (x - x^c)^perp . mu ds = 0 per body).
The double layer exerts no net force or torque and the rotlet no force; the
Stokeslet at x^c_i exerts the force F_i and no torque about x^c_i, the rotlet
the torque T_i.  Bounded flow: sum_i F_i = 0.  Square system of 2M + 3N + 2
equations in (mu, F, T, u_inf):

  (D + 1/2 I) mu + sum_i (G F_i + R T_i) + u_inf = v_{body} + omega_{body} p   (2M rows)
  int_{Gamma_i} mu ds = 0,  int_{Gamma_i} p . mu ds = 0                         (3N rows)
  sum_i F_i = 0                                                                 (2 rows)

p = (x - x^c)^perp.  Nystrom 2x2 blocks (trapezoid weight w_b):
  D[a, b] = w_b (1/pi) r r^T (r . n_b) / |r|^4     for a != b
  D[a, a] = w_a (-(kappa_a / 2pi)) tau_a tau_a^T   (the smooth diagonal limit)
Unknowns node-interleaved as in the mobility oracle.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import geometry

INV_PI = 1.0 / math.pi


def double_layer_matrix(geo: dict) -> np.ndarray:
    """Dense discrete D (2x2 blocks, weights included), shape [2M, 2M]."""
    M = geo["M"]
    rx = geo["x"][:, None] - geo["x"][None, :]
    ry = geo["y"][:, None] - geo["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    c = INV_PI * (rx * geo["nx"][None, :] + ry * geo["ny"][None, :]) / (r2 * r2)
    D = np.empty((2 * M, 2 * M))
    D[0::2, 0::2] = c * rx * rx
    D[0::2, 1::2] = c * rx * ry
    D[1::2, 0::2] = c * ry * rx
    D[1::2, 1::2] = c * ry * ry
    k = -geo["kappa"] / (2.0 * math.pi)
    tx, ty = geo["tx"], geo["ty"]
    a = np.arange(M)
    D[2 * a, 2 * a] = k * tx * tx
    D[2 * a, 2 * a + 1] = k * tx * ty
    D[2 * a + 1, 2 * a] = k * ty * tx
    D[2 * a + 1, 2 * a + 1] = k * ty * ty
    return D * np.repeat(geo["w"], 2)[None, :]


def _perp(geo: dict) -> tuple[np.ndarray, np.ndarray]:
    b = geo["body"]
    return -(geo["y"] - geo["yc"][b]), geo["x"] - geo["xc"][b]


def system_matrix(geo: dict) -> np.ndarray:
    """The (2M + 3N + 2)-square system of the module docstring."""
    M, N = geo["M"], geo["N"]
    n = 2 * M
    S = np.zeros((n + 3 * N + 2, n + 3 * N + 2))
    S[:n, :n] = double_layer_matrix(geo) + 0.5 * np.eye(n)
    # Stokeslet and rotlet at each body's centroid
    rx = geo["x"][:, None] - geo["xc"][None, :]
    ry = geo["y"][:, None] - geo["yc"][None, :]
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    s = 1.0 / (4.0 * math.pi)
    i = np.arange(N)
    S[0:n:2, n + 2 * i] = s * (lg + rx * rx / r2)
    S[0:n:2, n + 2 * i + 1] = s * (rx * ry / r2)
    S[1:n:2, n + 2 * i] = s * (rx * ry / r2)
    S[1:n:2, n + 2 * i + 1] = s * (lg + ry * ry / r2)
    S[0:n:2, n + 2 * N + i] = s * -ry / r2
    S[1:n:2, n + 2 * N + i] = s * rx / r2
    S[0:n:2, n + 3 * N] = 1.0
    S[1:n:2, n + 3 * N + 1] = 1.0
    # density orthogonal to each body's rigid motions
    a = np.arange(M)
    b = geo["body"]
    px, py = _perp(geo)
    S[n + 3 * b, 2 * a] = geo["w"]
    S[n + 3 * b + 1, 2 * a + 1] = geo["w"]
    S[n + 3 * b + 2, 2 * a] = geo["w"] * px
    S[n + 3 * b + 2, 2 * a + 1] = geo["w"] * py
    # no net force
    S[n + 3 * N, n + 2 * i] = 1.0
    S[n + 3 * N + 1, n + 2 * i + 1] = 1.0
    return S


def solve(g: dict, UW: np.ndarray) -> dict:
    """Rigid motions (v_x, v_y, omega) [N, 3] -> forces and torques (F_x, F_y, T) [N, 3]
    (net force zero) and the velocity at infinity."""
    geo = geometry.nodes(g)
    M, N = geo["M"], geo["N"]
    n = 2 * M
    UW = np.asarray(UW, dtype=np.float64).reshape(-1, 3)
    b = geo["body"]
    px, py = _perp(geo)
    rhs = np.zeros(n + 3 * N + 2)
    rhs[0:n:2] = UW[b, 0] + UW[b, 2] * px
    rhs[1:n:2] = UW[b, 1] + UW[b, 2] * py
    x = sla.lu_solve(sla.lu_factor(system_matrix(geo)), rhs)
    F = x[n:n + 2 * N].reshape(N, 2)
    T = x[n + 2 * N:n + 3 * N]
    return dict(FT=np.column_stack([F, T]), u_inf=x[n + 3 * N:n + 3 * N + 2].copy(), mu=x[:n], geo=geo)
