"""The seeded input builders: the structure of the paper's workloads
(bidisperse 1:1 by number with a_max = 1.4 a_min, Sec. 2; phi_3 from N,
Sec. 3.1; gaps between every pair; bumpy walls of Sec. 3) holds for what
they return.  Pure geometry, no method arithmetic."""
import math

import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I


def _min_gap(pos, rad, L):
    d = pos[:, None, :] - pos[None, :, :]
    d -= np.asarray(L) * np.round(d / np.asarray(L))
    dist = np.sqrt((d * d).sum(-1))
    gap = dist - rad[:, None] - rad[None, :]
    np.fill_diagonal(gap, np.inf)
    return gap.min()


def test_bidisperse_radii_and_volume_fraction():
    r = I.bidisperse_radii(10, 3.0)
    assert sorted(set(r.tolist())) == [3.0, pytest.approx(4.2)] and (r == 3.0).sum() == 5
    box = (96, 96, 96)
    n = I.n_for_phi3(0.50, box, 4.0, 5.6)
    assert n % 2 == 0
    # phi_3 = 2 N pi (a_max^3 + a_min^3) / (3 V) with N / 2 spheres of each size
    phi = (n / 2) * 4.0 / 3.0 * math.pi * (4.0 ** 3 + 5.6 ** 3) / 96 ** 3
    assert phi == pytest.approx(0.50, abs=0.002)


def test_placement_keeps_every_gap_and_is_seeded():
    box = (40, 40, 40)
    n = I.n_for_phi3(0.45, box, 3.0, 4.2)
    r = I.bidisperse_radii(n, 3.0)
    a = I.place_spheres(box, r, seed=7, min_gap=0.05)
    b = I.place_spheres(box, r, seed=7, min_gap=0.05)
    assert np.array_equal(a, b)
    assert ((a >= 0) & (a < np.asarray(box))).all()
    assert _min_gap(a, r, box) >= 0.05 - 1e-9


def test_bumpy_walls_geometry():
    L, aw, U = 32, 3.0, 0.02
    w = I.config_walls(L=L, a_wall=aw, phi3=0.2, wall_speed=U)
    drv = w.params["driven"].astype(bool)
    vel = w.params["vel"]
    pos, rad = w.pos, w.radius
    assert (pos >= 0).all() and (pos < L).all()
    assert _min_gap(pos, rad, (L, L, L)) >= 0.1 - 1e-9
    ys = pos[drv, 1]
    bottom, top = ys < L / 2, ys > L / 2
    assert bottom.sum() == top.sum() > 0 and set(np.unique(ys)) == {aw + 1.0, L - aw - 2.0}
    assert (rad[drv] == aw).all()
    # walls move at -U/2 (bottom) and +U/2 (top) along x; the suspension starts at rest
    assert np.allclose(vel[drv][bottom], [-U / 2, 0, 0]) and np.allclose(vel[drv][top], [U / 2, 0, 0])
    assert not vel[~drv].any()
    # every suspended sphere lies strictly between the walls' inner surfaces
    susp = pos[~drv, 1]
    assert (susp - rad[~drv] > aw + 1.0 + aw).all() and (susp + rad[~drv] < L - aw - 2.0 - aw).all()
    # Lees-Edwards rate U / L: the image of the top wall co-moves with the bottom wall
    assert w.shear == {"kind": 0, "rate": U / L}
    assert U / 2 - L * w.shear["rate"] == pytest.approx(-U / 2)
    # walls only
    w0 = I.config_walls(L=L, a_wall=aw, phi3=0.0)
    assert w0.params["driven"].all()
