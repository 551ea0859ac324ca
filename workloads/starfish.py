"""Starfish-curve workloads (Sec. 5 of Wala & Kloeckner, 'A Fast Algorithm with
Error Bounds for Quadrature by Expansion', uses starfish curves as its test
geometry; the shapes below follow the workload recipe of this library).

A curve is r(theta) = 1 + sum_k a_k cos(k theta + phi_k), scaled, rotated and
translated.  It is cut into panels equispaced in theta; each panel carries a
Gauss-Legendre rule at the *base* resolution (density unknowns) and at the
*upsampled* quadrature resolution (Sec. 2.2.1: density and geometry are
upsampled to the quadrature node count).  Everything here is exact evaluation
of the parametrisation plus seeded random numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Curve:
    cx: float = 0.0
    cy: float = 0.0
    scale: float = 1.0
    rot: float = 0.0
    # (k, a_k, phi_k) triples of r(theta) = 1 + sum a_k cos(k theta + phi_k)
    modes: tuple = field(default_factory=tuple)

    def radius(self, th):
        r = np.ones_like(th)
        dr = np.zeros_like(th)
        for k, a, phi in self.modes:
            r = r + a * np.cos(k * th + phi)
            dr = dr - a * k * np.sin(k * th + phi)
        return r, dr

    def point_and_tangent(self, th):
        r, dr = self.radius(th)
        c, s = np.cos(th + self.rot), np.sin(th + self.rot)
        x = self.cx + self.scale * r * c
        y = self.cy + self.scale * r * s
        dx = self.scale * (dr * c - r * s)
        dy = self.scale * (dr * s + r * c)
        return x, y, dx, dy


def _panel_nodes(curve: Curve, n_panels: int, ref: np.ndarray, refw: np.ndarray):
    dth = 2.0 * np.pi / n_panels
    th0 = dth * np.arange(n_panels)[:, None]
    th = th0 + (ref[None, :] + 1.0) * (0.5 * dth)
    x, y, dx, dy = curve.point_and_tangent(th)
    speed = np.hypot(dx, dy)
    nx, ny = dy / speed, -dx / speed          # outward for counter-clockwise curves
    w = refw[None, :] * speed * (0.5 * dth)
    return th, x, y, nx, ny, w


def discretize(curves, n_panels: int, nb: int = 16, nu: int = 64) -> dict:
    """Panels x Gauss-Legendre nodes for a list of curves.

    Returns a dict of contiguous arrays:
      base_xy, base_n  [P*nb, 2]  base nodes and unit outward normals
      base_theta, base_curve      curve parameter / curve index per base node
      up_xy, up_n      [P*nu, 2]  upsampled quadrature nodes and normals
      up_w             [P*nu]     quadrature weights (arc-length measure)
      up_base          [P*nu]     base node of the same panel nearest in the
                                  panel's reference coordinate
      panel_len        [P]        panel arc length (upsampled rule)
      ref_b, ref_u                reference Gauss-Legendre nodes in [-1, 1]
    """
    ref_b, w_b = np.polynomial.legendre.leggauss(nb)
    ref_u, w_u = np.polynomial.legendre.leggauss(nu)
    out = {k: [] for k in ("base_xy", "base_n", "base_theta", "base_curve",
                           "up_xy", "up_n", "up_w", "up_theta", "panel_len")}
    for ci, cv in enumerate(curves):
        th, x, y, nx, ny, _ = _panel_nodes(cv, n_panels, ref_b, w_b)
        out["base_xy"].append(np.stack([x.ravel(), y.ravel()], 1))
        out["base_n"].append(np.stack([nx.ravel(), ny.ravel()], 1))
        out["base_theta"].append(th.ravel())
        out["base_curve"].append(np.full(th.size, ci, np.int32))
        th, x, y, nx, ny, w = _panel_nodes(cv, n_panels, ref_u, w_u)
        out["up_xy"].append(np.stack([x.ravel(), y.ravel()], 1))
        out["up_n"].append(np.stack([nx.ravel(), ny.ravel()], 1))
        out["up_w"].append(w.ravel())
        out["up_theta"].append(th.ravel())
        out["panel_len"].append(w.sum(axis=1))
    g = {k: np.ascontiguousarray(np.concatenate(v)) for k, v in out.items()}
    npan = n_panels * len(curves)
    near = np.argmin(np.abs(ref_u[:, None] - ref_b[None, :]), axis=1)
    g["up_base"] = np.ascontiguousarray(
        (np.arange(npan)[:, None] * nb + near[None, :]).ravel().astype(np.int32))
    g.update(npanels=npan, nb=nb, nu=nu, ref_b=ref_b, ref_u=ref_u,
             n_curves=len(curves))
    return g


def _bbox(g):
    xy = g["up_xy"]
    return xy[:, 0].min(), xy[:, 0].max(), xy[:, 1].min(), xy[:, 1].max()


def _targets(g, rng, n_off: int, on_surface: str):
    parts_xy, parts_on = [], []
    if n_off:
        x0, x1, y0, y1 = _bbox(g)
        parts_xy.append(np.stack([rng.uniform(x0, x1, n_off), rng.uniform(y0, y1, n_off)], 1))
        parts_on.append(np.full(n_off, -1, np.int32))
    if on_surface == "base":
        parts_xy.append(g["base_xy"])
        parts_on.append(np.arange(len(g["base_xy"]), dtype=np.int32))
    elif on_surface == "up":
        parts_xy.append(g["up_xy"])
        parts_on.append(g["up_base"])
    g["tgt_xy"] = np.ascontiguousarray(np.concatenate(parts_xy))
    g["tgt_onsurf"] = np.ascontiguousarray(np.concatenate(parts_on).astype(np.int32))


def fourier_density(g, rng, n_modes: int = 10, scale: float = 1.0) -> np.ndarray:
    """Per-curve random Fourier series in theta with N(0, scale^2) coefficients."""
    nc = g["n_curves"]
    a = rng.normal(0.0, scale, (nc, n_modes))
    b = rng.normal(0.0, scale, (nc, n_modes))
    th, ci = g["base_theta"], g["base_curve"]
    k = np.arange(n_modes)
    mu = (a[ci] * np.cos(th[:, None] * k) + b[ci] * np.sin(th[:, None] * k)).sum(1)
    return np.ascontiguousarray(mu)


def starfish_c1(seed: int = 0) -> dict:
    """One starfish r = 1 + 0.25 cos 5 theta, 64 panels x 16 nodes (x4
    upsampled), density cos 3 theta + N(0, 0.1) noise, targets at the 1,024
    base nodes (on-surface, two-sided)."""
    rng = np.random.default_rng(seed)
    g = discretize([Curve(modes=((5, 0.25, 0.0),))], 64)
    g["density"] = np.ascontiguousarray(
        np.cos(3 * g["base_theta"]) + rng.normal(0.0, 0.1, g["base_theta"].size))
    _targets(g, rng, 0, "base")
    g.update(name="starfish-1x64x16-p5-10", p_qbx=5, p_fmm=10, n_max=32)
    return g


def starfish_grid(nx: int = 16, ny: int = 16, n_panels: int = 64, n_off: int = 1 << 20,
                  on_surface: str = "up", seed: int = 1, spacing: float = 3.0,
                  p_qbx: int = 8, p_fmm: int = 15) -> dict:
    """nx x ny grid of starfish (random rotation, scale U[0.5, 1], arm count in
    {3..8}, amplitude 0.25), random-Fourier density (10 modes, N(0,1)), n_off
    targets uniform in the bounding box plus on-surface targets."""
    rng = np.random.default_rng(seed)
    curves = []
    for j in range(ny):
        for i in range(nx):
            arms = int(rng.integers(3, 9))
            curves.append(Curve(cx=spacing * i, cy=spacing * j,
                                scale=float(rng.uniform(0.5, 1.0)),
                                rot=float(rng.uniform(0.0, 2 * np.pi)),
                                modes=((arms, 0.25, 0.0),)))
    g = discretize(curves, n_panels)
    g["density"] = fourier_density(g, rng)
    _targets(g, rng, n_off, on_surface)
    g.update(name=f"starfish-grid{nx}x{ny}x{n_panels}x16-p{p_qbx}-{p_fmm}",
             p_qbx=p_qbx, p_fmm=p_fmm, n_max=32)
    return g


def small_grid(nx: int = 2, ny: int = 2, n_panels: int = 16, n_off: int = 3000,
               seed: int = 7, p_qbx: int = 5, p_fmm: int = 10, on_surface: str = "base",
               spacing: float = 3.0) -> dict:
    """A few starfish with off-surface targets: small enough for brute force,
    large enough to have suspended centres, all list types and point targets."""
    g = starfish_grid(nx, ny, n_panels, n_off, on_surface, seed, spacing, p_qbx, p_fmm)
    g["name"] = f"starfish-grid{nx}x{ny}x{n_panels}-small"
    return g


def unit_circle(n_panels: int = 32, n_off: int = 0, seed: int = 3, off_radii=None) -> dict:
    """The unit circle (starfish with zero amplitude): closed forms exist for
    S and D of cos(k theta) densities.  Optional off-surface targets at given
    radii (angles uniform)."""
    rng = np.random.default_rng(seed)
    g = discretize([Curve()], n_panels)
    parts_xy = [g["base_xy"]]
    parts_on = [np.arange(len(g["base_xy"]), dtype=np.int32)]
    if off_radii is not None:
        for rad in off_radii:
            th = rng.uniform(0, 2 * np.pi, n_off)
            parts_xy.append(np.stack([rad * np.cos(th), rad * np.sin(th)], 1))
            parts_on.append(np.full(n_off, -1, np.int32))
    g["tgt_xy"] = np.ascontiguousarray(np.concatenate(parts_xy))
    g["tgt_onsurf"] = np.ascontiguousarray(np.concatenate(parts_on))
    g["density"] = np.ascontiguousarray(np.cos(3 * g["base_theta"]))
    g.update(name=f"unit-circle-{n_panels}", p_qbx=8, p_fmm=15, n_max=32)
    return g


def random_fourier_curves(n_curves: int, seed: int = 5, n_panels: int = 32, kmax: int = 8):
    """Star-shaped random curves r = 1 + sum_{k<=kmax} a_k cos(k theta + phi_k),
    a_k ~ U(0, 0.3/k): sum 0.3/k < 1 keeps them simple and star-shaped."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_curves):
        modes = tuple((k, float(rng.uniform(0, 0.3 / k)), float(rng.uniform(0, 2 * np.pi)))
                      for k in range(1, kmax + 1))
        out.append(Curve(modes=modes))
    return out


def order_training_curves(n_curves: int = 2000, seed: int = 5):
    """The curves of the order-selection training set: random star-shaped
    curves (random_fourier_curves, 32 panels each)."""
    return random_fourier_curves(n_curves, seed=seed)


def order_training_problem(curve: Curve, index: int) -> dict:
    """Curve `index` of the order-selection training set: 32 panels x 16
    nodes (x4 upsampled), a random-Fourier density seeded by its index, the
    base nodes as (on-surface, two-sided) targets."""
    g = discretize([curve], 32)
    g["density"] = fourier_density(g, np.random.default_rng(10_000 + index))
    g["tgt_xy"] = g["base_xy"]
    g["tgt_onsurf"] = np.arange(len(g["base_xy"]), dtype=np.int32)
    return g
