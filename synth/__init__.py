"""Seeded synthetic inputs for the elastance and mobility solvers.

This module is shared by the tests, the benchmark and the FP64 oracle's test
harness.  It produces *inputs only*: smooth closed curves sampled at the
equispaced parameter values theta_k = 2*pi*k/n (positions and the first and
second derivatives with respect to theta), the body layout, and random loads
(charges, forces, torques).  It holds none of the solver's arithmetic: no
quadrature weights, normals, curvatures, kernels or operators are computed
here.

Geometry record (a plain dict of numpy arrays, float64 unless noted):
  x, y        node positions                                   [M]
  dx, dy      d(x, y)/d theta                                  [M]
  ddx, ddy    d^2(x, y)/d theta^2                              [M]
  body_start  int32, body i owns nodes [body_start[i], body_start[i+1])  [N+1]
All curves are positively (counter-clockwise) oriented, as the paper's
boundary-value problems assume (Section 2, smooth positively oriented
boundaries).

Workload shapes follow the paper's examples: discs (Section 6.1.1 two-disc
test), ellipses (Section 6.1.3 nanocomposite inclusions, Section 6.2), and
star/"splash"-like curves r(theta) = a(1 + eps cos k theta) (the smooth
perturbed circles of Section 6.1.2).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# single curves
# ---------------------------------------------------------------------------
def _theta(n: int) -> np.ndarray:
    return TWO_PI * np.arange(n, dtype=np.float64) / n


def disc(cx: float, cy: float, R: float, n: int) -> dict:
    """Circle of radius R centred at (cx, cy), CCW."""
    t = _theta(n)
    c, s = np.cos(t), np.sin(t)
    return dict(x=cx + R * c, y=cy + R * s, dx=-R * s, dy=R * c, ddx=-R * c, ddy=-R * s)


def ellipse(cx: float, cy: float, a: float, b: float, phi: float, n: int) -> dict:
    """Ellipse with semi-axes a (along angle phi) and b, centred at (cx, cy), CCW."""
    t = _theta(n)
    c, s = np.cos(t), np.sin(t)
    cp, sp = math.cos(phi), math.sin(phi)
    # local (a cos t, b sin t) rotated by phi
    lx, ly = a * c, b * s
    ldx, ldy = -a * s, b * c
    lddx, lddy = -a * c, -b * s
    rot = lambda u, v: (cp * u - sp * v, sp * u + cp * v)  # noqa: E731
    x, y = rot(lx, ly)
    dx, dy = rot(ldx, ldy)
    ddx, ddy = rot(lddx, lddy)
    return dict(x=cx + x, y=cy + y, dx=dx, dy=dy, ddx=ddx, ddy=ddy)


def star(cx: float, cy: float, a: float, eps: float, k: int, theta0: float, n: int) -> dict:
    """Star curve r(theta) = a (1 + eps cos(k (theta - theta0))), CCW, |eps| < 1."""
    t = _theta(n)
    ph = k * (t - theta0)
    r = a * (1.0 + eps * np.cos(ph))
    r1 = -a * eps * k * np.sin(ph)
    r2 = -a * eps * k * k * np.cos(ph)
    c, s = np.cos(t), np.sin(t)
    x = r * c
    y = r * s
    dx = r1 * c - r * s
    dy = r1 * s + r * c
    ddx = r2 * c - 2.0 * r1 * s - r * c
    ddy = r2 * s + 2.0 * r1 * c - r * s
    return dict(x=cx + x, y=cy + y, dx=dx, dy=dy, ddx=ddx, ddy=ddy)


def node_spacing(curve: dict) -> float:
    """Largest parameter-step arc length max_theta |x'(theta)| * 2 pi / n."""
    n = curve["x"].size
    return float(np.max(np.hypot(curve["dx"], curve["dy"])) * TWO_PI / n)


def assemble(curves: list[dict]) -> dict:
    """Concatenate curves (one body each) into a geometry record."""
    keys = ("x", "y", "dx", "dy", "ddx", "ddy")
    g = {k: np.ascontiguousarray(np.concatenate([c[k] for c in curves])) for k in keys}
    starts = np.zeros(len(curves) + 1, dtype=np.int32)
    starts[1:] = np.cumsum([c["x"].size for c in curves])
    g["body_start"] = starts
    return g


def bodies(g: dict) -> list[dict]:
    """Split a geometry record back into its curves."""
    bs = g["body_start"]
    out = []
    for i in range(bs.size - 1):
        sl = slice(int(bs[i]), int(bs[i + 1]))
        out.append({k: g[k][sl] for k in ("x", "y", "dx", "dy", "ddx", "ddy")})
    return out


def min_gap_ok(c1: dict, c2: dict, factor: float) -> bool:
    """True if every node of c1 is at least factor*max(h1, h2) from every node of c2."""
    h = max(node_spacing(c1), node_spacing(c2))
    d2 = (c1["x"][:, None] - c2["x"][None, :]) ** 2 + (c1["y"][:, None] - c2["y"][None, :]) ** 2
    return bool(np.sqrt(d2.min()) >= factor * h)


# ---------------------------------------------------------------------------
# loads
# ---------------------------------------------------------------------------
def charges(n_bodies: int, rng: np.random.Generator, neutral: bool = True) -> np.ndarray:
    """Charges q_i ~ N(0, 1); mean removed when neutral (the paper's sum q = 0 condition)."""
    q = rng.standard_normal(n_bodies)
    if neutral:
        q -= q.mean()
    return q


def forces_torques(n_bodies: int, rng: np.random.Generator, neutral: bool = True) -> np.ndarray:
    """Per-body (Fx, Fy, T) ~ N(0, 1), shape [N, 3]; net force removed when neutral."""
    ft = rng.standard_normal((n_bodies, 3))
    if neutral:
        ft[:, :2] -= ft[:, :2].mean(axis=0, keepdims=True)
    return ft


# ---------------------------------------------------------------------------
# placement helpers
# ---------------------------------------------------------------------------
class _Placer:
    """Random sequential addition with a uniform cell grid over body centres.

    A candidate body is accepted when its node-to-node distance to every
    already-placed body is at least gap_factor * max(h_i, h_j).
    """

    def __init__(self, cell: float, gap_factor: float):
        self.cell = cell
        self.gap = gap_factor
        self.grid: dict[tuple[int, int], list[int]] = {}
        self.curves: list[dict] = []
        self.centres: list[tuple[float, float]] = []
        self.radii: list[float] = []
        self.h: list[float] = []

    def _key(self, x, y):
        return (int(math.floor(x / self.cell)), int(math.floor(y / self.cell)))

    def try_add(self, curve: dict, cx: float, cy: float, rmax: float) -> bool:
        h = node_spacing(curve)
        kx, ky = self._key(cx, cy)
        reach = int(math.ceil((2 * rmax + self.gap * 2 * h) / self.cell)) + 1
        for ix in range(kx - reach, kx + reach + 1):
            for iy in range(ky - reach, ky + reach + 1):
                for j in self.grid.get((ix, iy), ()):
                    ox, oy = self.centres[j]
                    need = rmax + self.radii[j] + self.gap * max(h, self.h[j])
                    if (ox - cx) ** 2 + (oy - cy) ** 2 >= need * need:
                        continue
                    if not min_gap_ok(curve, self.curves[j], self.gap):
                        return False
        idx = len(self.curves)
        self.grid.setdefault((kx, ky), []).append(idx)
        self.curves.append(curve)
        self.centres.append((cx, cy))
        self.radii.append(rmax)
        self.h.append(h)
        return True


# ---------------------------------------------------------------------------
# the benchmark workloads
# ---------------------------------------------------------------------------
def four_discs(seed: int = 0, n: int = 128) -> dict:
    """4 discs, radii U[0.5, 1], centres on a jittered 2x2 grid (spacing 3), gap >= 0.5.

    Elastance workload of 512 nodes; charges N(0,1) with the mean removed.
    """
    rng = np.random.default_rng(seed)
    S = 3.0
    while True:
        radii = rng.uniform(0.5, 1.0, 4)
        cent = [(i * S + rng.uniform(-0.25, 0.25), j * S + rng.uniform(-0.25, 0.25))
                for i in range(2) for j in range(2)]
        ok = True
        for a in range(4):
            for b in range(a + 1, 4):
                d = math.hypot(cent[a][0] - cent[b][0], cent[a][1] - cent[b][1])
                if d - radii[a] - radii[b] < 0.5:
                    ok = False
        if ok:
            break
    g = assemble([disc(cx, cy, r, n) for (cx, cy), r in zip(cent, radii)])
    g["q"] = charges(4, rng)
    g["name"] = f"4 discs, n={n} per disc (M={4 * n})"
    return g


def star_grid(seed: int = 1000, n: int = 256, rows: int = 10, cols: int = 10,
              gap_factor: float = 5.0) -> dict:
    """rows x cols star curves r = a(1 + eps cos k(theta - theta0)) on a jittered grid.

    a ~ U[0.5, 1], eps ~ U[0, 0.3], k ~ U{3..6}, theta0 ~ U[0, 2 pi); grid spacing
    3.2 with jitter U[-0.15, 0.15]^2, redrawn until the node-to-node gap between
    neighbours is >= gap_factor node spacings.  Default: 100 stars x 256 nodes
    (M = 25,600), charges N(0,1) with the mean removed.
    """
    rng = np.random.default_rng(seed)
    S = 3.2
    placer = _Placer(cell=S, gap_factor=gap_factor)
    for i in range(rows):
        for j in range(cols):
            for _ in range(1000):
                a = rng.uniform(0.5, 1.0)
                eps = rng.uniform(0.0, 0.3)
                k = int(rng.integers(3, 7))
                th0 = rng.uniform(0.0, TWO_PI)
                cx = i * S + rng.uniform(-0.15, 0.15)
                cy = j * S + rng.uniform(-0.15, 0.15)
                c = star(cx, cy, a, eps, k, th0, n)
                if placer.try_add(c, cx, cy, a * (1 + eps)):
                    break
            else:
                raise RuntimeError("star placement failed")
    g = assemble(placer.curves)
    g["q"] = charges(len(placer.curves), rng)
    g["name"] = f"{rows * cols} stars, n={n} per star (M={rows * cols * n})"
    return g


def ellipse_suspension(seed: int = 2000, n_bodies: int = 400, n: int = 128,
                       area_fraction: float = 0.2, aspect: tuple[float, float] | None = None,
                       minor: tuple[float, float] = (0.3, 1.0), gap_factor: float = 5.0,
                       max_tries: int = 200000) -> dict:
    """Random sequential addition of ellipses (major semi-axis 1) in a square box.

    Minor semi-axis b ~ U[minor] (or 1/A with aspect ratio A ~ U[aspect]),
    orientation U[0, pi), box side sqrt(sum(pi b) / area_fraction), node gap
    >= gap_factor node spacings.  Default: 400 ellipses x 128 nodes (M = 51,200).
    Forces N(0,1)^2 with the mean removed, torques N(0,1).
    """
    rng = np.random.default_rng(seed)
    if aspect is not None:
        bs = 1.0 / rng.uniform(aspect[0], aspect[1], n_bodies)
    else:
        bs = rng.uniform(minor[0], minor[1], n_bodies)
    L = math.sqrt(np.sum(math.pi * bs) / area_fraction)
    placer = _Placer(cell=2.5, gap_factor=gap_factor)
    tries = 0
    for b in bs:
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError(f"ellipse placement failed after {max_tries} tries")
            cx, cy = rng.uniform(0, L, 2)
            phi = rng.uniform(0, math.pi)
            c = ellipse(cx, cy, 1.0, b, phi, n)
            if placer.try_add(c, cx, cy, 1.0):
                break
    g = assemble(placer.curves)
    g["FT"] = forces_torques(n_bodies, rng)
    g["name"] = f"{n_bodies} ellipses, n={n} per ellipse (M={n_bodies * n})"
    return g


def ellipse_lattice(seed: int = 5000, rows: int = 100, cols: int = 100, n: int = 64,
                    aspect: tuple[float, float] = (1.0, 3.0), gap_factor: float = 5.0) -> dict:
    """Ellipses (major semi-axis 1, aspect ratio U[aspect], random orientation) on
    a hexagonal lattice whose spacing 2 + gap_factor * (2 pi / n) keeps every
    node gap >= gap_factor node spacings for any orientations.  The default
    (100 x 100, 64 nodes: M = 640,000) has area fraction about 0.32; random
    sequential addition jams before 0.3 at this gap.  Forces N(0,1)^2 with the
    mean removed, torques N(0,1).
    """
    rng = np.random.default_rng(seed)
    h = TWO_PI / n  # largest node spacing of a major-semi-axis-1 ellipse
    d = 2.0 + gap_factor * h
    curves = []
    area = 0.0
    for i in range(rows):
        for j in range(cols):
            cx = j * d + (0.5 * d if i % 2 else 0.0)
            cy = i * d * math.sqrt(3.0) / 2.0
            b = 1.0 / rng.uniform(aspect[0], aspect[1])
            curves.append(ellipse(cx, cy, 1.0, b, rng.uniform(0.0, math.pi), n))
            area += math.pi * b
    g = assemble(curves)
    g["FT"] = forces_torques(rows * cols, rng)
    g["area_fraction"] = area / (cols * d * rows * d * math.sqrt(3.0) / 2.0)
    g["name"] = f"{rows * cols} ellipses on a hexagonal lattice, n={n} (M={rows * cols * n})"
    return g


def two_discs(d: float, n: int) -> dict:
    """Two unit discs centred at (-1 - d/2, 0) and (1 + d/2, 0) (Section 6.1.1 layout)."""
    return assemble([disc(-1.0 - d / 2, 0.0, 1.0, n), disc(1.0 + d / 2, 0.0, 1.0, n)])


def random_request(rng: np.random.Generator, max_bodies: int = 64,
                   nodes=(64, 128, 256), gap_factor: float = 5.0) -> dict:
    """One mixed request: 1..max_bodies ellipses or stars with per-body node counts.

    kind 0 = elastance (charges), 1 = mobility (forces and torques).
    """
    nb = int(rng.integers(1, max_bodies + 1))
    kind = int(rng.integers(0, 2))
    S = 3.2
    side = int(math.ceil(math.sqrt(nb)))
    placer = _Placer(cell=S, gap_factor=gap_factor)
    slots = rng.permutation(side * side)[:nb]
    for s in slots:
        i, j = divmod(int(s), side)
        for _ in range(1000):
            n = int(rng.choice(nodes))
            cx = i * S + rng.uniform(-0.15, 0.15)
            cy = j * S + rng.uniform(-0.15, 0.15)
            if rng.uniform() < 0.5:
                b = rng.uniform(0.3, 1.0)
                c = ellipse(cx, cy, 1.0, b, rng.uniform(0, math.pi), n)
                rmax = 1.0
            else:
                a = rng.uniform(0.5, 1.0)
                eps = rng.uniform(0.0, 0.3)
                c = star(cx, cy, a, eps, int(rng.integers(3, 7)), rng.uniform(0, TWO_PI), n)
                rmax = a * (1 + eps)
            if placer.try_add(c, cx, cy, rmax):
                break
        else:
            raise RuntimeError("request placement failed")
    g = assemble(placer.curves)
    g["kind"] = kind
    if kind == 0:
        g["q"] = charges(nb, rng)
    else:
        g["FT"] = forces_torques(nb, rng)
    return g


WORKLOADS = {
    "four_discs_M512": lambda: four_discs(seed=0),
    "stars100_M25600": lambda: star_grid(seed=1000),
    "ellipses400_M51200": lambda: ellipse_suspension(seed=2000),
    "ellipses10000_M640000": lambda: ellipse_lattice(seed=5000),
}
