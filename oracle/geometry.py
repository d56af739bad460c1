"""Nystrom geometry for the trapezoidal rule on smooth closed curves (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Given node positions x(theta_k) and the first and second theta-derivatives at
theta_k = 2 pi k / n_i on each positively oriented curve Gamma_i:
  speed      |x'| = sqrt(x1'^2 + x2'^2)
  weight     w = |x'| * 2 pi / n_i            (trapezoidal rule in arc length)
  tangent    tau = x' / |x'|
  normal     n = (tau_2, -tau_1)             (outward for a CCW curve)
  curvature  kappa = (x1' x2'' - x2' x1'') / |x'|^3   (1/R on a circle)
Per body (Section 4, definitions before the mobility BVP):
  length     |Gamma_i| = sum_{a in i} w_a
  centroid   x^c_i = (1/|Gamma_i|) sum w_a x_a   (arc-length centroid)
  W_i        sum w_a |x_a - x^c_i|^2            (eq. for rho, Section 4.2)
"""
from __future__ import annotations

import math

import numpy as np


def nodes(g: dict) -> dict:
    """Return the per-node and per-body quadrature data of a geometry record."""
    x = np.asarray(g["x"], dtype=np.float64)
    y = np.asarray(g["y"], dtype=np.float64)
    dx = np.asarray(g["dx"], dtype=np.float64)
    dy = np.asarray(g["dy"], dtype=np.float64)
    ddx = np.asarray(g["ddx"], dtype=np.float64)
    ddy = np.asarray(g["ddy"], dtype=np.float64)
    bs = np.asarray(g["body_start"], dtype=np.int64)
    N = bs.size - 1
    M = x.size
    counts = np.diff(bs)
    body = np.repeat(np.arange(N), counts)

    speed = np.sqrt(dx * dx + dy * dy)
    w = speed * (2.0 * math.pi) / counts[body]
    tx, ty = dx / speed, dy / speed
    nx, ny = ty, -tx
    kappa = (dx * ddy - dy * ddx) / speed**3

    length = np.zeros(N)
    np.add.at(length, body, w)
    xc = np.zeros(N)
    yc = np.zeros(N)
    np.add.at(xc, body, w * x)
    np.add.at(yc, body, w * y)
    xc /= length
    yc /= length
    W = np.zeros(N)
    np.add.at(W, body, w * ((x - xc[body]) ** 2 + (y - yc[body]) ** 2))
    return dict(M=M, N=N, x=x, y=y, w=w, tx=tx, ty=ty, nx=nx, ny=ny, kappa=kappa,
                body=body, body_start=bs, length=length, xc=xc, yc=yc, W=W)


def interior_points(geo: dict) -> dict:
    """Interior evaluation points per body.

    The field S(mu + sigma) is constant inside each conductor (Section 3, proof
    of the representation theorem), and S(mu + rho) is a rigid motion inside
    each body (Section 4, proof of the mobility theorem).  It is therefore read
    at interior points: z0 = the discrete centroid, and for the rotation rate
    z1 = z0 + delta e1, z2 = z0 + delta e2 with delta = 1/4 of the smallest
    node distance from z0 (a reading: the paper checks u on the boundary).
    """
    N = geo["N"]
    body = geo["body"]
    d = np.hypot(geo["x"] - geo["xc"][body], geo["y"] - geo["yc"][body])
    dmin = np.full(N, np.inf)
    np.minimum.at(dmin, body, d)
    return dict(z0x=geo["xc"].copy(), z0y=geo["yc"].copy(), delta=0.25 * dmin)
