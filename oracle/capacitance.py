"""Capacitance oracle (FP64, dense Nystrom matrix + LU): the other half of the
paper's round trip (Section 6.1, "The elastance problem").

TEST INFRASTRUCTURE ONLY (see the package docstring).

Prescribed potentials phi_j on the conductors Gamma_j give the charges q_j and
the potential at infinity u_inf of the field that equals phi_j on Gamma_j and
stays bounded at infinity (so sum_j q_j = 0).  The paper solves this problem
with classical techniques (it cites Mikhlin) that differ from its elastance
equations, and checks that the elastance solve driven by these charges returns
phi_j - u_inf.  This module takes the classical exterior Dirichlet
representation for a multiply connected domain:

  u(x) = D[mu](x) + sum_i A_i log|x - z_i| + u_inf,
  D[mu](x) = (1/2pi) int mu(y) (y - x) . n_y / |x - y|^2 ds_y   (source normal, outward)

with z_i a point inside body i.  On the boundary the double layer jumps:
u_ext = (D - 1/2 I) mu + ...; (D - 1/2 I) annihilates a constant on any one
curve, so the density carries the constraints int_{Gamma_i} mu ds = 0, and
boundedness at infinity gives sum_i A_i = 0.  The unknowns (mu, A, u_inf) then
solve a square system of M + N + 1 equations:

  (D - 1/2 I) mu + sum_i A_i log|x_a - z_i| + u_inf = phi_{body(a)}   (M rows)
  int_{Gamma_i} mu ds = 0                                            (N rows)
  sum_i A_i = 0                                                      (1 row)

The double layer has zero flux through every curve and A_i log|x - z_i| has
flux 2 pi A_i through Gamma_i, while the field of a charge q is
-(q/2pi) log|x|: the charge on conductor i is q_i = -2 pi A_i.

Nystrom entries (trapezoid weight w_b, r = x_a - x_b):
  D[a, b] = w_b (1/2pi) (-r . n_b) / |r|^2      for a != b
  D[a, a] = w_a kappa_a / (4 pi)               (the smooth diagonal limit; on a
                                                circle of radius R the kernel
                                                is 1/(4 pi R) everywhere)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import geometry

INV_2PI = 1.0 / (2.0 * math.pi)


def double_layer_matrix(geo: dict) -> np.ndarray:
    """Dense discrete D (source normal, weights included), shape [M, M]."""
    M = geo["M"]
    rx = geo["x"][:, None] - geo["x"][None, :]
    ry = geo["y"][:, None] - geo["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    rn = -(rx * geo["nx"][None, :] + ry * geo["ny"][None, :])
    D = INV_2PI * rn / r2
    D[np.arange(M), np.arange(M)] = geo["kappa"] / (4.0 * math.pi)
    return D * geo["w"][None, :]


def system_matrix(geo: dict) -> np.ndarray:
    """The (M + N + 1)-square system of the module docstring."""
    M, N = geo["M"], geo["N"]
    pts = geometry.interior_points(geo)
    zx, zy = pts["z0x"], pts["z0y"]
    S = np.zeros((M + N + 1, M + N + 1))
    S[:M, :M] = double_layer_matrix(geo) - 0.5 * np.eye(M)
    S[:M, M:M + N] = np.log(np.hypot(geo["x"][:, None] - zx[None, :], geo["y"][:, None] - zy[None, :]))
    S[:M, M + N] = 1.0
    S[M + geo["body"], np.arange(M)] = geo["w"]  # int_{Gamma_i} mu ds = 0
    S[M + N, M:M + N] = 1.0  # sum_i A_i = 0
    return S


def solve(g: dict, phi: np.ndarray) -> dict:
    """Potentials phi [N] -> charges q [N] (sum zero) and the potential at infinity."""
    geo = geometry.nodes(g)
    M, N = geo["M"], geo["N"]
    b = np.zeros(M + N + 1)
    b[:M] = np.asarray(phi, dtype=np.float64)[geo["body"]]
    x = sla.lu_solve(sla.lu_factor(system_matrix(geo)), b)
    A = x[M:M + N]
    return dict(q=-2.0 * math.pi * A, u_inf=float(x[M + N]), mu=x[:M], A=A, geo=geo)

