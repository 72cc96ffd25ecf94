"""Seeded synthetic inputs shaped like the paper's runs.

This module holds geometry and parameter presets only: it places bidisperse
spheres (1:1 by number, a_max = 1.4 a_min, Sec. 2) in a periodic box at a
requested volume or area fraction (Sec. 3.1 for phi_3, Sec. 4.1 for the
monolayer phi) and lists the lattice sizes and physical parameters of each
workload.  It contains none of the lattice-Boltzmann or particle arithmetic,
so both the CUDA path and the CPU oracle can take their inputs from here.

Placement: random positions with the radii shrunk to a dilute packing, then
the radii grown to full size in a few stages, each stage minimising the
harmonic overlap energy sum max(0, a_i + a_j + gap - d_ij)^2 with L-BFGS, and a
final pass of pairwise pushes until every gap is at least ``min_gap`` (a
soft-sphere relaxation; random sequential addition alone jams near
phi ~ 0.38 in 3D, and plain pushes converge slowly near phi ~ 0.58).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

try:  # neighbour search and minimiser of the relaxation
    from scipy.spatial import cKDTree
    from scipy.optimize import minimize
except Exception:  # pragma: no cover - scipy is present on both machines
    cKDTree = None
    minimize = None


def bidisperse_radii(n: int, a_min: float, ratio: float = 1.4) -> np.ndarray:
    """n radii, half a_min and half ratio * a_min (small ones first)."""
    r = np.full(n, float(a_min))
    r[n // 2:] = a_min * ratio
    return r


def n_for_phi3(phi3: float, box, a_min: float, a_max: float) -> int:
    """Particle count for phi_3 = 2 N pi (a_max^3 + a_min^3) / (3 V)."""
    V = box[0] * box[1] * box[2]
    n = 3.0 * phi3 * V / (2.0 * math.pi * (a_max ** 3 + a_min ** 3))
    return 2 * int(round(n / 2))


def n_for_phi2(phi: float, box, a_min: float, a_max: float) -> int:
    """Particle count for the monolayer phi = N pi (a_max^2 + a_min^2) / (2 Lx Ly)."""
    n = phi * 2.0 * box[0] * box[1] / (math.pi * (a_max ** 2 + a_min ** 2))
    return 2 * int(round(n / 2))


def _wrap(d, L):
    return d - L * np.round(d / L)


def _relax(x, r, L, quasi2d, min_gap, max_iter):
    """Push overlapping pairs apart until every gap >= min_gap; True on success."""
    n = r.size
    reach = 2.0 * r.max() + min_gap
    for _ in range(max_iter):
        x %= L
        if cKDTree is not None:
            tree = cKDTree(x, boxsize=L * (1 + 1e-12))
            pairs = tree.query_pairs(reach, output_type="ndarray")
        else:
            ii, jj = np.triu_indices(n, 1)
            d = _wrap(x[jj] - x[ii], L)
            keep = (d * d).sum(1) < reach * reach
            pairs = np.stack([ii[keep], jj[keep]], 1)
        if len(pairs) == 0:
            return True
        i, j = pairs[:, 0], pairs[:, 1]
        d = _wrap(x[j] - x[i], L)
        dist = np.sqrt((d * d).sum(1))
        ov = r[i] + r[j] + min_gap - dist
        bad = ov > 0
        if not bad.any():
            return True
        i, j, d, dist, ov = i[bad], j[bad], d[bad], dist[bad], ov[bad]
        nvec = d / np.maximum(dist, 1e-12)[:, None]
        push = 0.5 * (ov[:, None] + 1e-3) * nvec
        dx = np.zeros_like(x)
        np.add.at(dx, i, -push)
        np.add.at(dx, j, push)
        if quasi2d:
            dx[:, 2] = 0.0
        x += dx
    return False


def _minimise(x, r, L, quasi2d, gap, iters=2000):
    """L-BFGS on the harmonic overlap energy (periodic box); returns new x."""
    n = r.size
    reach = 2.0 * r.max() + gap
    dim = 2 if quasi2d else 3
    z0 = x[:, 2].copy()

    def unpack(v):
        y = x.copy()
        y[:, :dim] = v.reshape(n, dim)
        if quasi2d:
            y[:, 2] = z0
        return y

    def energy(v):
        y = unpack(v) % L
        tree = cKDTree(y, boxsize=L * (1 + 1e-12))
        pairs = tree.query_pairs(reach, output_type="ndarray")
        g = np.zeros_like(y)
        if len(pairs) == 0:
            return 0.0, g[:, :dim].ravel()
        i, j = pairs[:, 0], pairs[:, 1]
        d = _wrap(y[j] - y[i], L)
        dist = np.sqrt((d * d).sum(1))
        ov = r[i] + r[j] + gap - dist
        m = ov > 0
        if not m.any():
            return 0.0, g[:, :dim].ravel()
        i, j, d, dist, ov = i[m], j[m], d[m], dist[m], ov[m]
        nv = d / np.maximum(dist, 1e-12)[:, None]
        # dE/dx_j = -2 ov n, dE/dx_i = +2 ov n
        f = 2.0 * ov[:, None] * nv
        np.add.at(g, i, f)
        np.add.at(g, j, -f)
        return float((ov * ov).sum()), g[:, :dim].ravel()

    res = minimize(energy, x[:, :dim].ravel(), jac=True, method="L-BFGS-B",
                   options=dict(maxiter=iters, ftol=1e-16, gtol=1e-12))
    return unpack(res.x) % L


def place_spheres(box, radii, seed: int, quasi2d: bool = False, min_gap: float = 0.05,
                  max_iter: int = 400) -> np.ndarray:
    """Non-overlapping centres (gap >= min_gap) in a periodic box.

    Radii are grown from a dilute packing to their final size in a few
    stages, minimising the overlap energy after each, then the remaining
    small overlaps are pushed apart, so dense packings (phi_3 ~ 0.58) form
    in seconds."""
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=np.float64)
    r = np.asarray(radii, dtype=np.float64)
    n = r.size
    x = rng.random((n, 3)) * L
    if quasi2d:
        x[:, 2] = L[2] / 2.0
    if n < 2:
        return x
    dim = 2 if quasi2d else 3
    if quasi2d:
        phi = np.pi * (r ** 2).sum() / (L[0] * L[1])
    else:
        phi = 4.0 / 3.0 * np.pi * (r ** 3).sum() / L.prod()
    scale = min(1.0, (0.25 / max(phi, 1e-9)) ** (1.0 / dim))
    if not _relax(x, r * scale, L, quasi2d, min_gap * scale, max_iter):
        raise RuntimeError("sphere placement did not converge")
    # the minimiser aims at a wider gap so that its residual overlaps are
    # far below min_gap; the pushes then close what is left
    target = 1.5 * min_gap + 0.02
    for s in np.linspace(scale, 1.0, 5)[1:]:
        x = _minimise(x, r * s, L, quasi2d, target * s)
    if not _relax(x, r, L, quasi2d, min_gap, 20 * max_iter):
        raise RuntimeError("sphere placement did not converge")
    x %= L
    if quasi2d:
        x[:, 2] = L[2] / 2.0
    return x


@dataclass
class Workload:
    """One synthetic box: lattice, particles, physical parameters, shear."""
    name: str
    nx: int
    ny: int
    nz: int
    radius: np.ndarray
    pos: np.ndarray
    params: dict = field(default_factory=dict)
    shear: dict = field(default_factory=dict)
    precision: str = "fp32"
    steps: int = 100

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return int(self.radius.size)


def _mass(a, rho_p=1.0):
    return rho_p * 4.0 / 3.0 * math.pi * a ** 3


def config_small(seed: int = 1001, n: int = 20, box=(32, 32, 32), radius: float = 4.5,
                 precision: str = "fp64") -> Workload:
    """32^3, tau = 1, 20 spheres of radius 4.5, Lees-Edwards rate 1e-4, mu = 1."""
    r = np.full(n, radius)
    pos = place_spheres(box, r, seed, min_gap=0.3)
    m0 = _mass(radius)
    params = dict(tau=1.0, rho0=1.0, rho_p=1.0, mu=1.0, kn=0.36 * m0, kt_ratio=0.2,
                  F0=0.0, debye=0.02 * radius, lub_delta=0.01 * radius, lub_cut=0.5,
                  a_map_ratio=0.95, quasi2d=False, nbins=36)
    return Workload("d3q19-32^3-20spheres-a4.5-LE1e-4", *box, r, pos, params,
                    dict(kind=0, rate=1e-4), precision, 200)


def config_dst(seed: int = 1002, phi3: float = 0.50, L: int = 96, rate: float = 1e-4,
               precision: str = "fp32") -> Workload:
    """96^3 bulk simple shear: bidisperse radii 4 / 5.6, kn = 1e3, kt = 0.5 kn, mu = 1."""
    a_min, a_max = 4.0, 5.6
    box = (L, L, L)
    n = n_for_phi3(phi3, box, a_min, a_max)
    r = bidisperse_radii(n, a_min)
    pos = place_spheres(box, r, seed, min_gap=0.05)
    kn = 1.0e3
    params = dict(tau=1.0, rho0=1.0, rho_p=1.0, mu=1.0, kn=kn, kt_ratio=0.5,
                  F0=2e-4 * kn, debye=0.02 * a_min, lub_delta=0.01 * a_min, lub_cut=0.5,
                  a_map_ratio=0.95, quasi2d=False, nbins=36)
    return Workload(f"dst-{L}^3-phi{phi3:.2f}-N{n}", *box, r, pos, params,
                    dict(kind=0, rate=rate), precision, 100000)


def config_monolayer(seed: int = 1003, phi: float = 0.70, Lx: int = 512, Ly: int = 512,
                     Lz: int = 12, gamma0: float = 1.0, theta: float = 0.0,
                     precision: str = "fp16") -> Workload:
    """Quasi-2D oscillatory shear: radii scaled to a_max = Lz / 4 (monolayer)."""
    a_max = Lz / 4.0
    a_min = a_max / 1.4
    box = (Lx, Ly, Lz)
    n = n_for_phi2(phi, box, a_min, a_max)
    r = bidisperse_radii(n, a_min)
    pos = place_spheres(box, r, seed, quasi2d=True, min_gap=0.05)
    m0 = 0.5 * (_mass(a_min) + _mass(a_max))
    kn = 0.36 * m0                      # dt = 0.6 tau_c
    tau_c = math.sqrt(m0 / kn)
    omega = 1e-3 / tau_c                # omega tau_c = 1e-3
    params = dict(tau=1.0, rho0=1.0, rho_p=1.0, mu=1.0, kn=kn, kt_ratio=0.2,
                  F0=2e-4 * kn, debye=0.02 * a_min, lub_delta=0.01 * a_min, lub_cut=0.5,
                  a_map_ratio=0.95, quasi2d=True, nbins=36)
    return Workload(f"monolayer-{Lx}x{Ly}x{Lz}-phi{phi:.2f}-N{n}", *box, r, pos, params,
                    dict(kind=1, gamma0=gamma0, omega=omega, theta=theta), precision, 1000)


def batch_sweep(seed: int = 1004, nbox: int = 64, lo: int = 48, hi: int = 96):
    """Independent cubes of seeded edge U{lo..hi}, phi_3 ~ U(0.45, 0.58), mixed shear."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbox):
        L = int(rng.integers(lo, hi + 1))
        phi3 = float(rng.uniform(0.45, 0.58))
        if b % 2 == 0:
            sh = dict(kind=0, rate=float(10 ** rng.uniform(-5, -3)))
        else:
            sh = dict(kind=1, gamma0=float(rng.choice([0.1, 1.0])), omega=6e-4,
                      theta=float(rng.choice([0.0, math.pi / 2])))
        w = config_dst(seed=seed * 100 + b, phi3=phi3, L=L, precision="bf16")
        w.shear = sh
        w.name = f"box{b}-{L}^3-phi{phi3:.3f}"
        out.append(w)
    return out


def bumpy_wall(nx: int, nz: int, y: float, radius: float, gap: float = 0.5) -> np.ndarray:
    """Centres of one wall layer: spheres of the given radius on a square
    lattice in the periodic x-z plane at height y, spaced as evenly as the
    box allows with at least ``gap`` between neighbours."""
    s = 2.0 * radius + gap
    mx, mz = max(1, int(nx // s)), max(1, int(nz // s))
    xs = (np.arange(mx) + 0.5) * nx / mx
    zs = (np.arange(mz) + 0.5) * nz / mz
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    return np.stack([X.ravel(), np.full(X.size, float(y)), Z.ravel()], axis=1)


def config_walls(seed: int = 1006, L: int = 48, a_wall: float = 3.0, phi3: float = 0.30,
                 wall_speed: float = 0.02, precision: str = "fp64") -> Workload:
    """Shear driven by bumpy walls made of particles (the paper's driver,
    Sec. 3): a bottom and a top layer of wall spheres moving at -U/2 and +U/2
    in x with a bidisperse suspension between them.  The box stays periodic
    in y through a Lees-Edwards plane whose image velocity is U, so the image
    of the top wall below the bottom wall moves with the bottom wall and the
    thin layer across the plane is not sheared.  Returns the workload with
    ``driven`` (1 for wall spheres) and their velocities in ``params``."""
    yb, yt = a_wall + 1.0, L - a_wall - 2.0
    bottom = bumpy_wall(L, L, yb, a_wall)
    top = bumpy_wall(L, L, yt, a_wall)
    a_min, gap = 3.0, 0.5
    # centres of the suspension lie in a band that keeps every sphere clear of
    # both walls; they are placed in a periodic box of the band's height (its
    # gaps across the periodic y boundary are only stricter) and lifted
    band = (yt - a_wall) - (yb + a_wall) - 2 * (1.4 * a_min + gap)
    n = n_for_phi3(phi3, (L, band + 2 * 1.4 * a_min, L), a_min, 1.4 * a_min) if phi3 > 0 else 0
    r = bidisperse_radii(n, a_min) if n else np.zeros(0)
    body = place_spheres((L, band, L), r, seed, min_gap=0.1) if n else np.zeros((0, 3))
    body[:, 1] += yb + a_wall + 1.4 * a_min + gap
    pos = np.concatenate([bottom, top, body])
    rad = np.concatenate([np.full(len(bottom) + len(top), a_wall), r])
    vel = np.zeros((len(pos), 3))
    vel[:len(bottom), 0] = -0.5 * wall_speed
    vel[len(bottom):len(bottom) + len(top), 0] = 0.5 * wall_speed
    driven = np.zeros(len(pos), dtype=np.int32)
    driven[:len(bottom) + len(top)] = 1
    kn = 1.0e3
    params = dict(tau=1.0, rho0=1.0, rho_p=1.0, mu=1.0, kn=kn, kt_ratio=0.5,
                  F0=2e-4 * kn, debye=0.02 * a_min, lub_delta=0.01 * a_min, lub_cut=0.5,
                  a_map_ratio=0.95, quasi2d=False, nbins=36, vel=vel, driven=driven)
    return Workload(f"walls-{L}^3-phi{phi3:.2f}-N{n}+{len(bottom) + len(top)}", L, L, L, rad, pos,
                    params, dict(kind=0, rate=wall_speed / L), precision, 2000)


def random_populations(nx, ny, nz, seed: int, amplitude: float = 0.02, weights=None):
    """Positive perturbed populations (19, nz, ny, nx) around a rest state.

    ``weights`` are the 19 lattice weights in the caller's velocity order;
    the perturbation is multiplicative so every population stays positive."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=np.float64).reshape(19, 1, 1, 1)
    return w * (1.0 + amplitude * rng.standard_normal((19, nz, ny, nx)))
