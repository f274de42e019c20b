"""Seeded synthetic workloads (grids, initial states, rotor and body geometry).

This module holds no arithmetic of the method: it only builds inputs. The
tests feed the same arrays to the CUDA library and to the CPU oracle, and the
benchmark uses the same builders. Shapes follow the paper's workloads:

* Taylor-Green vortex, periodic box [0, 2 pi)^3 (a smooth periodic field).
* Turbulent channel, Re_tau = 180, Sec. 4.1: tanh-stretched wall-normal axis
  y = tanh(b_g (eta / 1.5 pi - 1)) / tanh(b_g), b_g = 2, periodic x/z, no-slip
  walls, Poiseuille profile plus a seeded 5 % perturbation, constant body force.
* ALM rotor (Sec. 3.1, the NREL layout of Sec. 4.3 with a synthetic blade and
  polar): 3 blades x 50 actuator points, chord c(r) = 0.08 D (1 - 0.7 r/R),
  twist 15 deg (1 - r/R), tip-speed ratio 7, eps = 2 dx, inflow x-, outflow
  x+, periodic y, slip z.
* ALM rotor plus IBM tower and nacelle (Sec. 3.2, the NTNU layout of Sec. 4.4
  with synthetic cylinders): tower d = 0.08 D from the ground to the hub,
  nacelle d = 0.1 D, 0.3 D long, with flat caps.

The paper's own runs use airfoil tables, turbine geometry and measured data
that are not available here; these seeded inputs stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_NOSLIP, BC_SLIP, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3, 4
BC_NAMES = {"periodic": 0, "noslip": 1, "slip": 2, "inflow": 3, "outflow": 4}


@dataclass
class Rotor:
    n_blades: int
    r: np.ndarray
    chord: np.ndarray
    twist: np.ndarray
    width: np.ndarray
    hub: tuple
    omega: float
    azimuth0: float
    radius: float
    eps: float
    rho_inf: float = 1.0
    u_inf_ref: float = 1.0
    correction: bool = False
    tip_correction: bool = False


@dataclass
class Body:
    xyz: np.ndarray          # (n, 3)
    dS: np.ndarray           # (n,)
    eps: float
    vel: np.ndarray | None = None
    niter: int = 5
    tol: float = 0.0


@dataclass
class Workload:
    name: str
    n: tuple
    faces: list
    mach: float
    u_ref: float
    mu: float
    bc: list                  # [(lo, hi)] per axis, ints
    cfl: float = 0.5
    dt_fixed: float = 0.0
    inflow: tuple = (1.0, 0.0, 0.0, 0.0)   # rho, u, v, w
    body_force: tuple = (0.0, 0.0, 0.0)
    rho_ref: float = 1.0
    state0: np.ndarray | None = None       # (4, nz, ny, nx) float64
    rotors: list = field(default_factory=list)
    bodies: list = field(default_factory=list)
    steps: int = 20

    @property
    def cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


def uniform_faces(a: float, b: float, n: int) -> np.ndarray:
    return np.linspace(a, b, n + 1)


def cell_centres(faces: np.ndarray) -> np.ndarray:
    return 0.5 * (faces[1:] + faces[:-1])


def taylor_green_3d(n: int = 32, mach: float = 0.1, re: float = 1600.0, cfl: float = 0.5,
                    steps: int = 20) -> Workload:
    """Taylor-Green vortex: u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    rho = 1, on [0, 2 pi)^3, U_ref = 1, mu = 1 / Re."""
    L = 2.0 * math.pi
    f = [uniform_faces(0.0, L, n)] * 3
    xc = cell_centres(f[0])
    z, y, x = np.meshgrid(xc, xc, xc, indexing="ij")
    Q = np.zeros((4, n, n, n))
    Q[0] = 1.0
    Q[1] = np.sin(x) * np.cos(y) * np.cos(z)
    Q[2] = -np.cos(x) * np.sin(y) * np.cos(z)
    return Workload("taylor-green-%d^3" % n, (n, n, n), f, mach, 1.0, 1.0 / re,
                    [(0, 0)] * 3, cfl=cfl, state0=Q, steps=steps)


def tanh_faces(n: int, b_g: float = 2.0) -> np.ndarray:
    """Wall-normal faces of Sec. 4.1: y = tanh(b_g (eta/1.5pi - 1)) / tanh(b_g),
    eta uniform on [0, 3 pi]."""
    eta = np.linspace(0.0, 3.0 * math.pi, n + 1)
    y = np.tanh(b_g * (eta / (1.5 * math.pi) - 1.0)) / math.tanh(b_g)
    y[0], y[-1] = -1.0, 1.0
    return y


def channel(n=(128, 128, 128), re_tau: float = 180.0, re_b: float = 2800.0, mach: float = 0.1,
            b_g: float = 2.0, amp: float = 0.05, seed: int = 20260311, cfl: float = 0.5,
            steps: int = 500) -> Workload:
    """Turbulent channel: [0, 2 pi] x [-1, 1] x [0, pi], bulk velocity 1,
    mu = 1 / Re_b (half height), driving force u_tau^2 with u_tau = Re_tau mu."""
    nx, ny, nz = n
    fx = uniform_faces(0.0, 2.0 * math.pi, nx)
    fy = tanh_faces(ny, b_g)
    fz = uniform_faces(0.0, math.pi, nz)
    mu = 1.0 / re_b
    u_tau = re_tau * mu
    yc = cell_centres(fy)
    rng = np.random.default_rng(seed)
    r = rng.random((nz, ny, nx, 3))          # drawn x fastest, then y, z; component last
    Q = np.zeros((4, nz, ny, nx))
    Q[0] = 1.0
    U = 1.5 * (1.0 - yc ** 2)
    Q[1] = U[None, :, None] + amp * (2.0 * r[..., 0] - 1.0)
    Q[2] = amp * (2.0 * r[..., 1] - 1.0)
    Q[3] = amp * (2.0 * r[..., 2] - 1.0)
    return Workload("channel-Re_tau180-%dx%dx%d" % n, tuple(n), [fx, fy, fz], mach, 1.0, mu,
                    [(0, 0), (1, 1), (0, 0)], cfl=cfl, body_force=(u_tau ** 2, 0.0, 0.0),
                    state0=Q, steps=steps)


def rotor_3x50(D: float = 1.0, hub=(0.0, 0.0, 0.0), dx: float = 1.0 / 42.7, tsr: float = 7.0,
               u_inf: float = 1.0, n_pts: int = 50, n_blades: int = 3,
               eps_factor: float = 2.0) -> Rotor:
    """Synthetic rotor: points at r_i = (i + 1/2) R / N, width R / N (reading
    of 'evenly distributed'), c = 0.08 D (1 - 0.7 r/R), twist 15 deg (1 - r/R)."""
    R = 0.5 * D
    i = np.arange(n_pts)
    r = (i + 0.5) * R / n_pts
    chord = 0.08 * D * (1.0 - 0.7 * r / R)
    twist = math.radians(15.0) * (1.0 - r / R)
    width = np.full(n_pts, R / n_pts)
    omega = tsr * u_inf / R
    return Rotor(n_blades, r, chord, twist, width, tuple(hub), omega, 0.0, R,
                 eps_factor * dx, 1.0, u_inf)


def alm_rotor(n=(512, 192, 192), D: float = 1.0, mach: float = 0.1, re_d: float = 5000.0,
              cfl: float = 0.5, steps: int = 200, n_pts: int = 50) -> Workload:
    """Rotor without tower: [-3D, 9D] x [-2D, 2D]^2, inflow x-, outflow x+,
    periodic y, slip z; rotor at the origin, axis +x, uniform inflow 1."""
    nx, ny, nz = n
    f = [uniform_faces(-3 * D, 9 * D, nx), uniform_faces(-2 * D, 2 * D, ny),
         uniform_faces(-2 * D, 2 * D, nz)]
    dx = 12 * D / nx
    Q = np.zeros((4, nz, ny, nx))
    Q[0] = 1.0
    Q[1] = 1.0
    rot = rotor_3x50(D, (0.0, 0.0, 0.0), dx, n_pts=n_pts)
    return Workload("alm-rotor-%dx%dx%d" % n, tuple(n), f, mach, 1.0, D / re_d,
                    [(3, 4), (0, 0), (2, 2)], cfl=cfl, inflow=(1.0, 1.0, 0.0, 0.0), state0=Q,
                    rotors=[rot], steps=steps)


def cylinder_points(centre, axis: int, radius: float, z0: float, z1: float, spacing: float,
                    caps: bool) -> tuple:
    """Lagrangian points on a cylinder surface (rings along the axis), plus
    flat caps on concentric rings when asked. Returns (xyz, dS)."""
    pts, area = [], []
    n_th = max(8, int(round(2 * math.pi * radius / spacing)))
    n_ax = max(1, int(round((z1 - z0) / spacing)))
    dz = (z1 - z0) / n_ax
    dth = 2 * math.pi / n_th
    a1, a2 = [d for d in range(3) if d != axis]
    for k in range(n_ax):
        s = z0 + (k + 0.5) * dz
        for m in range(n_th):
            th = (m + 0.5) * dth
            p = [0.0, 0.0, 0.0]
            p[axis] = s
            p[a1] = centre[a1] + radius * math.cos(th)
            p[a2] = centre[a2] + radius * math.sin(th)
            pts.append(p)
            area.append(radius * dth * dz)
    if caps:
        n_r = max(1, int(round(radius / spacing)))
        dr = radius / n_r
        for s in (z0, z1):
            for ir in range(n_r):
                rr = (ir + 0.5) * dr
                nt = max(4, int(round(2 * math.pi * rr / spacing)))
                for m in range(nt):
                    th = (m + 0.5) * 2 * math.pi / nt
                    p = [0.0, 0.0, 0.0]
                    p[axis] = s
                    p[a1] = centre[a1] + rr * math.cos(th)
                    p[a2] = centre[a2] + rr * math.sin(th)
                    pts.append(p)
                    area.append(rr * dr * 2 * math.pi / nt)
    return np.array(pts, dtype=np.float64), np.array(area, dtype=np.float64)


def tower_and_nacelle(D: float, hub, dx: float, tower_spacing: float = 0.011,
                      nacelle_spacing: float = 0.0086, eps_factor: float = 2.0) -> list:
    """Tower: cylinder d = 0.08 D at (x = 0.16 D, y = hub y), z from the ground
    (z = 0) to the hub; nacelle: d = 0.1 D, x in [-0.05 D, 0.25 D] on the hub
    axis, flat caps."""
    hx, hy, hz = hub
    txyz, tdS = cylinder_points((hx + 0.16 * D, hy, 0.0), 2, 0.04 * D, 0.0, hz,
                                tower_spacing * D, caps=False)
    nxyz, ndS = cylinder_points((0.0, hy, hz), 0, 0.05 * D, hx - 0.05 * D, hx + 0.25 * D,
                                nacelle_spacing * D, caps=True)
    eps = eps_factor * dx
    return [Body(txyz, tdS, eps), Body(nxyz, ndS, eps)]


def alm_ibm_rotor(n=(384, 256, 256), D: float = 1.0, mach: float = 0.1, re_d: float = 5000.0,
                  cfl: float = 0.5, steps: int = 200, n_pts: int = 50) -> Workload:
    """Rotor plus IBM tower and nacelle: [-3D, 9D] x [-2D, 2D] x [0, 4D],
    hub (0, 0, 2D), inflow x-, outflow x+, periodic y, slip ground and top."""
    nx, ny, nz = n
    f = [uniform_faces(-3 * D, 9 * D, nx), uniform_faces(-2 * D, 2 * D, ny),
         uniform_faces(0.0, 4 * D, nz)]
    dx = 12 * D / nx
    hub = (0.0, 0.0, 2.0 * D)
    Q = np.zeros((4, nz, ny, nx))
    Q[0] = 1.0
    Q[1] = 1.0
    rot = rotor_3x50(D, hub, dx, n_pts=n_pts)
    bodies = tower_and_nacelle(D, hub, dx)
    return Workload("alm-ibm-rotor-%dx%dx%d" % n, tuple(n), f, mach, 1.0, D / re_d,
                    [(3, 4), (0, 0), (2, 2)], cfl=cfl, inflow=(1.0, 1.0, 0.0, 0.0), state0=Q,
                    rotors=[rot], bodies=bodies, steps=steps)


def perturbed(w: Workload, amp: float, seed: int) -> np.ndarray:
    """A copy of the initial state with seeded uniform noise of amplitude amp on
    the momentum components (density untouched)."""
    rng = np.random.default_rng(seed)
    Q = w.state0.copy()
    Q[1:] += amp * (2.0 * rng.random(Q[1:].shape) - 1.0)
    return Q
