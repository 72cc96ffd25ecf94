"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 storage <= 1e-12 relative on populations after 100 steps,
FP32 <= 2e-5; particle centres <= 1e-9 (FP64) over 50 steps; stresses of FP64
runs <= 1e-9 relative.  Population errors are max |gpu - oracle| over the
nodes that are fluid on both sides, divided by max |oracle| there.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S
from parity_helpers import dilate as _dilate, fp32_particle_pop_err as _fp32_particle_pop_err
from parity_helpers import fp32_particle_comparison as _fp32_particle_comparison

pytestmark = pytest.mark.gpu

C_LAT, W_LAT, _ = O.lattice()


def _both(nx, ny, nz, radius=(), pos=(), precision="fp64", **kw):
    g = S.Suspension(nx, ny, nz, radius, pos, precision=precision, **kw)
    o = O.Oracle(nx, ny, nz, radius, pos, **kw)
    return g, o


def _step(g, o, n, **sh):
    g.step(n, S.make_shear(**sh))
    o.step(n, O.shear(**sh))


def _pop_err(g, o):
    fo, fg = o.populations(), g.populations()
    fl = (o.owner() < 0) & (g.owner() < 0)
    return np.abs(fg[:, fl] - fo[:, fl]).max() / np.abs(fo[:, fl]).max()


def _assert_hist_equal(hg, ho):
    """FP64 angular histograms (Eq. 19-23) bin by bin: contact counts exactly,
    the summed normal and counter-clockwise tangential forces to 1e-9 of the
    largest bin."""
    assert (hg[:, 0] == ho[:, 0]).all()
    for col in (1, 2):
        scale = max(np.abs(ho[:, col]).max(), 1e-300)
        assert np.abs(hg[:, col] - ho[:, col]).max() <= 1e-9 * scale, col


def _params(w, **over):
    kw = dict(w.params)
    kw.update(over)
    return kw


# ------------------------------------------------------------------ fluid only
@pytest.mark.parametrize("shape", [(37, 21, 13), (32, 16, 8), (4, 4, 4)])
def test_fluid_lees_edwards_fp64(shape):
    nx, ny, nz = shape
    f0 = I.random_populations(nx, ny, nz, seed=11, amplitude=0.03, weights=W_LAT)
    g, o = _both(nx, ny, nz, tau=0.8)
    g.set_populations(f0)
    o.set_populations(f0)
    _step(g, o, 100, kind=0, rate=3.7e-3)
    assert _pop_err(g, o) < 1e-12
    tg, dg = g.time()
    assert tg == 100 and abs(dg - o.delta) < 1e-12


def test_fluid_oscillatory_fp64():
    nx, ny, nz = 24, 18, 10
    f0 = I.random_populations(nx, ny, nz, seed=12, amplitude=0.03, weights=W_LAT)
    g, o = _both(nx, ny, nz, tau=1.0)
    g.set_populations(f0)
    o.set_populations(f0)
    sh = dict(kind=1, gamma0=0.5, omega=2 * math.pi / 50, theta=math.pi / 2)
    _step(g, o, 60, **sh)
    # amplitude reduction: a second protocol continues the offset
    sh2 = dict(kind=1, gamma0=0.05, omega=2 * math.pi / 50, theta=math.pi / 2)
    _step(g, o, 40, **sh2)
    assert _pop_err(g, o) < 1e-12
    assert abs(g.time()[1] - o.delta) < 1e-11


def test_fluid_fp32():
    nx, ny, nz = 40, 24, 12
    f0 = I.random_populations(nx, ny, nz, seed=13, amplitude=0.03, weights=W_LAT)
    g, o = _both(nx, ny, nz, precision="fp32", tau=0.9)
    g.set_populations(f0)
    o.set_populations(f0)
    _step(g, o, 100, kind=0, rate=2.3e-3)
    assert _pop_err(g, o) < 2e-5


def test_viscous_stress_fp64():
    nx, ny, nz = 16, 20, 8
    f0 = I.random_populations(nx, ny, nz, seed=14, amplitude=0.02, weights=W_LAT)
    g, o = _both(nx, ny, nz, tau=0.7)
    g.set_populations(f0)
    o.set_populations(f0)
    _step(g, o, 30, kind=0, rate=1e-3)
    sg, _ = g.stress(S.VISCOUS)
    so, _ = o.stress(O.VISCOUS)
    assert np.abs(sg - so).max() <= 1e-10 * np.abs(so).max()


# ------------------------------------------------------------ with particles
def test_held_particles_fp64():
    w = I.config_small()
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, **_params(w, move_particles=False))
    assert (g.owner() == o.owner()).all()
    _step(g, o, 100, kind=0, rate=1e-3)
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12
    Fg, Tg = g.hydro()
    Fo, To = o.hydro()
    scale = np.abs(Fo).max()
    # the oracle holds the link sums of the last step, the library those for the next
    o.step(1, O.shear(kind=0, rate=1e-3))
    Fo, To = o.hydro()
    assert np.abs(Fg - Fo).max() <= 1e-10 * max(scale, np.abs(Fo).max())
    assert np.abs(Tg - To).max() <= 1e-10 * np.abs(To).max()


def test_moving_particles_fp64_trajectories():
    w = I.config_small()
    vel = np.random.default_rng(21).normal(0, 2e-3, (w.n, 3))
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, vel=vel, **_params(w))
    _step(g, o, 50, kind=0, rate=2e-3)
    Rg, Ug, Wg = g.particles()
    Ro, Uo, Wo = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    assert np.abs(Ug - Uo).max() < 1e-9
    assert np.abs(Wg - Wo).max() < 1e-9
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12


def test_dense_contacts_lubrication_repulsion_fp64():
    """Bidisperse 40^3 at phi_3 ~ 0.35 with kn = 1e3, kt = 0.5 kn, F0 > 0:
    contacts, tangential history, Coulomb slip, lubrication and double-layer
    forces are all active; 50 steps of trajectories and every stress kind."""
    a_min = 4.0
    box = (40, 40, 40)
    n = I.n_for_phi3(0.35, box, a_min, 1.4 * a_min)
    r = I.bidisperse_radii(n, a_min)
    pos = I.place_spheres(box, r, seed=31, min_gap=0.02)
    vel = np.random.default_rng(32).normal(0, 5e-3, (n, 3))
    kw = dict(tau=1.0, kn=1e3, kt_ratio=0.5, mu=1.0, F0=0.2, debye=0.08, lub_delta=0.04,
              lub_cut=0.5, a_map_ratio=0.95, nbins=36)
    g, o = _both(*box, r, pos, vel=vel, **kw)
    _step(g, o, 50, kind=0, rate=1e-3)
    Rg, Ug, _ = g.particles()
    Ro, Uo, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12
    for kind in (S.VISCOUS, S.CONTACT, S.REPULSIVE, S.LUBRICATION, S.TOTAL, S.ANGULAR):
        sg, hg = g.stress(kind)
        so, ho = o.stress(kind)
        assert np.abs(sg - so).max() <= 1e-9 * max(np.abs(so).max(), 1e-300), kind
    _assert_hist_equal(hg, ho)
    assert hg[:, 0].sum() > 0, "the run should have contacts"
    assert np.abs(hg[:, 2]).max() > 0, "the run should have tangential contact forces"
    assert np.abs(g.stress(S.LUBRICATION)[0]).max() > 0, "the run should have lubricated pairs"


def test_cell_list_and_two_particles_per_warp_fp64():
    """More than 4096 particles in one box: candidates come from the
    counting-sort cell list, and (FP64 keeps the particle kernel at two
    resident blocks per SM) each warp steps two particles per sub-step.
    Monodisperse a = 2.5 at phi_3 ~ 0.33 in 96^3, sheared."""
    box = (96, 96, 96)
    n = 4500
    r = np.full(n, 2.5)
    pos = I.place_spheres(box, r, seed=51, min_gap=0.05)
    vel = np.random.default_rng(52).normal(0, 2e-3, (n, 3))
    kw = dict(tau=1.0, kn=1e3, kt_ratio=0.5, mu=1.0, F0=0.2, debye=0.05, lub_delta=0.025,
              lub_cut=0.5, a_map_ratio=0.95, nbins=36)
    g, o = _both(*box, r, pos, vel=vel, **kw)
    _step(g, o, 6, kind=0, rate=1e-3)
    assert o.error() == 0
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12
    for kind in (S.CONTACT, S.TOTAL):
        sg, hg = g.stress(kind)
        so, ho = o.stress(kind)
        assert np.abs(sg - so).max() <= 1e-9 * max(np.abs(so).max(), 1e-300), kind
    _assert_hist_equal(hg, ho)


@pytest.mark.parametrize("case", ["rest", "comoving", "relative", "moving_le"])
def test_touching_spheres_fp64(case):
    """Mapped spheres closer than one spacing (Appendix A (i)): links between
    the two solids carry the equilibrium of the surfaces' mean velocity.  A
    held pair at rest and a held pair moving with its uniform fluid feel no
    force (to round-off, on both sides); a held pair in relative motion, and
    a free pair in relative motion crossing the Lees-Edwards plane under
    shear, match the oracle's forces, torques, centres and populations."""
    d = np.array([0.6, 0.48, 0.64])
    R0 = np.array([8.3, 9.1, 8.7])
    sh = dict(kind=0, rate=0.0)
    held = case != "moving_le"
    if case == "moving_le":
        R0 = np.array([8.3, 21.5, 8.7])        # the pair straddles y = L_y
        sh = dict(kind=0, rate=2e-3)
    if case in ("relative", "moving_le"):
        vel = [[0.02, -0.01, 0.005], [-0.015, 0.01, 0.02]]
    else:
        U = [0.03, -0.02, 0.012] if case == "comoving" else [0.0, 0.0, 0.0]
        vel = [U, U]
    pos = [R0, (R0 + 8.0 * d) % 24.0]
    g, o = _both(24, 24, 24, [4.0, 4.0], pos, vel=vel, move_particles=not held, kn=1e3,
                 lub_cut=0.5, dem_substeps=4)
    if case == "comoving":
        feq = O.equilibrium(1.0, np.array(vel[0]))
        f0 = np.broadcast_to(feq[:, None], (19, 24 ** 3)).copy()
        g.set_populations(f0)
        o.set_populations(f0)
    assert (g.owner() == o.owner()).all()
    _step(g, o, 5, **sh)
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12
    Rg, Ug, _ = g.particles()
    Ro, Uo, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9 and np.abs(Ug - Uo).max() < 1e-9
    # the library holds the link sums that the next step applies, the oracle
    # those of the step it took last: one more oracle step lines them up
    Fg, Tg = g.hydro()
    o.step(1, O.shear(**sh))
    Fo, To = o.hydro()
    if case in ("relative", "moving_le"):
        scale = np.abs(Fo).max()
        assert scale > 1e-4
        assert np.abs(Fg - Fo).max() <= 1e-10 * scale
        assert np.abs(Tg - To).max() <= 1e-10 * np.abs(To).max()
    else:
        assert np.abs(Fg).max() < 1e-13 and np.abs(Tg).max() < 1e-12
        assert np.abs(Fo).max() < 1e-13


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_ladd_operator(precision, tol):
    """Ladd's linear operator (tau = 0.8, tau_bulk = 1.3) through the C ABI
    against the oracle: random populations under oscillatory Lees-Edwards
    shear, then moving spheres; populations, viscous stress and centres."""
    nx, ny, nz = 24, 18, 10
    kw = dict(tau=0.8, collision="ladd", tau_bulk=1.3)
    f0 = I.random_populations(nx, ny, nz, seed=61, amplitude=0.03, weights=W_LAT)
    g, o = _both(nx, ny, nz, precision=precision, **kw)
    g.set_populations(f0)
    o.set_populations(f0)
    _step(g, o, 60, kind=1, gamma0=0.05, omega=2 * math.pi / 200, theta=0.3)
    assert _pop_err(g, o) < tol
    sg, _ = g.stress(S.VISCOUS)
    so, _ = o.stress(S.VISCOUS)
    assert np.abs(sg - so).max() <= (1e-9 if precision == "fp64" else 1e-4) * np.abs(so).max()
    w = I.config_small()
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, precision=precision, **_params(w, **kw))
    if precision == "fp64":
        _step(g, o, 40, kind=0, rate=2e-3)
        assert _pop_err(g, o) < tol
    else:
        _fp32_particle_pop_err(g, o, 40, w.radius, tol, kind=0, rate=2e-3)
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < (1e-9 if precision == "fp64" else 1e-4)


def test_drag_on_periodic_sphere_arrays_hasimoto():
    """Hasimoto's series over box sizes (FP64): a held sphere of radius 4.5
    in periodic boxes of 24, 32, 48 and 64, fluid driven by a body force and
    run to steady state (drag = body force on the fluid); the hydrodynamic
    radius read from the drag through the series, calibrated in the largest
    box, predicts the boxes of 32 and 48 within 1 % (24, where a / L = 0.19,
    within 2 %), and is the mapped radius within 3 %.  The force scales as L^-3 so that the superficial
    velocity, hence the Reynolds number (~0.015), is the same in every box."""
    from test_oracle_pins import hasimoto_radius, _hasimoto_K
    a, tau = 4.5, 1.0
    eta = (tau - 0.5) / 3.0
    radii = {}
    for L in (24, 32, 48, 64):
        g = 1e-6 * (24.0 / L) ** 3
        s = S.Suspension(L, L, L, np.array([a]), np.array([[L / 2, L / 2, L / 2]]), precision="fp64",
                         tau=tau, move_particles=False, body_force=(g, 0.0, 0.0), F0=0.0, lub_cut=0.0)
        c = 4.0 * math.pi / 3.0 * a ** 3 / L ** 3
        t_mean = L ** 3 * _hasimoto_K(c) / (6.0 * math.pi * eta * a)   # decay time of the mean flow
        s.step(int(10 * t_mean), S.make_shear(kind=0, rate=0.0))
        F, _ = s.hydro()
        f = s.populations().reshape(19, -1)
        fluid = (s.owner() < 0).ravel()
        U = (np.asarray(C_LAT, dtype=float)[:, 0] @ f)[fluid].sum() / L ** 3
        print(f"L={L}: drag / body force on the fluid - 1 = {F[0, 0] / (g * fluid.sum()) - 1:.2e}")
        assert F[0, 0] == pytest.approx(g * fluid.sum(), rel=3e-3)
        radii[L] = hasimoto_radius(L, eta, U, F[0, 0])
        s.close()
    for L in (32, 48):
        assert radii[L] == pytest.approx(radii[64], rel=0.01), radii
    assert radii[24] == pytest.approx(radii[64], rel=0.02), radii
    assert radii[64] == pytest.approx(0.95 * a, rel=0.03)


def test_torque_on_a_spinning_sphere_fp64():
    """Rotlet: a held sphere of radius 4.5 spinning in periodic boxes of 48
    and 64 feels T = -8 pi eta0 a_h^3 Omega about its axis, a_h the mapped
    radius within 3 % and the same in both boxes within 0.5 %."""
    a, tau, Om = 4.5, 1.0, 1e-4
    eta = (tau - 0.5) / 3.0
    radii = []
    for L in (48, 64):
        s = S.Suspension(L, L, L, np.array([a]), np.array([[L / 2, L / 2, L / 2]]), precision="fp64",
                         tau=tau, omega=np.array([[0.0, 0.0, Om]]), move_particles=False, F0=0.0,
                         lub_cut=0.0)
        s.step(int(10 / (eta * (2 * math.pi / L) ** 2)), S.make_shear(kind=0, rate=0.0))
        F, T = s.hydro()
        assert T[0, 2] < 0 and np.abs(T[0, :2]).max() < 1e-9 * abs(T[0, 2])
        radii.append((-T[0, 2] / (8 * math.pi * eta * Om)) ** (1 / 3))
        s.close()
    assert radii[1] == pytest.approx(0.95 * a, rel=0.03)
    assert radii[0] == pytest.approx(radii[1], rel=0.005)


def test_moduli_fp64():
    """Storage and loss moduli (Eq. 17, 18) through the C ABI against the
    oracle: moving spheres under oscillatory shear, one period measured after
    a warm-up period; the Newtonian limit of a particle-free box; no moduli
    without an oscillatory protocol."""
    w = I.config_small()
    P, g0, th = 100, 0.05, 0.4
    sh = dict(kind=1, gamma0=g0, omega=2 * math.pi / P, theta=th)
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, **_params(w))
    _step(g, o, P, **sh)
    g.stress_reset()
    o.stress_reset()
    _step(g, o, P, **sh)
    gg, go = g.moduli(), o.moduli(g0)
    scale = max(abs(go[0]), abs(go[1]))
    assert scale > 0
    assert abs(gg[0] - go[0]) <= 1e-9 * scale and abs(gg[1] - go[1]) <= 1e-9 * scale
    # particle-free: G'' = eta0 omega, G' = 0
    f = S.Suspension(4, 8, 4, precision="fp64", tau=1.0)
    P2 = 2000
    sh2 = S.make_shear(kind=1, gamma0=g0, omega=2 * math.pi / P2, theta=0.0)
    f.step(P2, sh2)
    f.stress_reset()
    f.step(2 * P2, sh2)
    gp, gpp = f.moduli()
    eta0 = 0.5 / 3.0
    assert gpp == pytest.approx(eta0 * 2 * math.pi / P2, rel=1e-5)
    assert abs(gp) < 1e-6 * gpp
    c = S.Suspension(8, 8, 8, precision="fp64", tau=1.0)
    c.step(2, S.make_shear(kind=0, rate=1e-3))
    with pytest.raises(S.SuspError) as e:
        c.moduli()
    assert e.value.status == S.SUSP_ESTATE


def test_quasi2d_oscillatory_fp64():
    """Monolayer at the paper's resolution (radii 5 / 7, L_z = 4 a_max, Sec. 4.1)."""
    box = (64, 64, 28)
    a_min, a_max = 5.0, 7.0
    n = I.n_for_phi2(0.5, box, a_min, a_max)
    r = I.bidisperse_radii(n, a_min)
    pos = I.place_spheres(box, r, seed=41, quasi2d=True, min_gap=0.05)
    m0 = 0.5 * 4 / 3 * math.pi * (a_min ** 3 + a_max ** 3)
    kw = dict(tau=1.0, kn=0.36 * m0, kt_ratio=0.2, mu=1.0, F0=2e-4 * 0.36 * m0,
              debye=0.02 * a_min, lub_delta=0.01 * a_min, lub_cut=0.5, quasi2d=True)
    g, o = _both(*box, r, pos, **kw)
    sh = dict(kind=1, gamma0=0.1, omega=2 * math.pi / 400, theta=0.0)
    _step(g, o, 60, **sh)
    assert o.error() == 0
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    assert np.abs(Rg[:, 2] - box[2] / 2).max() == 0.0
    assert _pop_err(g, o) < 1e-12
    for kind in (S.VISCOUS, S.ANGULAR, S.TOTAL):
        sg, _ = g.stress(kind)
        so, _ = o.stress(kind)
        assert np.abs(sg - so).max() <= 1e-9 * max(np.abs(so).max(), 1e-300), kind


def test_moving_particles_fp32():
    w = I.config_small(precision="fp32")
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **_params(w))
    _fp32_particle_pop_err(g, o, 100, w.radius, 2e-5, kind=0, rate=1e-3)
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-4



@pytest.mark.parametrize("precision,pop_tol,r_tol,u_tol,s_tol",
                         [("fp64", 1e-12, 1e-9, 1e-10, 1e-9), ("fp32", 2e-5, 1e-4, 1e-5, 2e-2)])
def test_bumpy_walls(precision, pop_tol, r_tol, u_tol, s_tol):
    """Shear driven by two layers of wall spheres (driven: they keep their
    velocity and spin) moving at -U/2 and +U/2, with a Lees-Edwards rate U / L
    so the image of the top wall co-moves with the bottom wall (Sec. 3).
    Driven spheres take part in contacts, lubrication and bounce-back; their
    velocities must come back unchanged and their centres advanced by U t."""
    w = I.config_walls(L=32, a_wall=3.0, phi3=0.2, wall_speed=0.02, precision=precision)
    kw = _params(w)
    drv = kw["driven"].astype(bool)
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, precision=precision, **kw)
    if precision == "fp64":
        _step(g, o, 60, **w.shear)
        assert (g.owner() == o.owner()).all()
        assert _pop_err(g, o) < pop_tol
    else:
        _fp32_particle_pop_err(g, o, 60, w.radius, pop_tol, **w.shear)
    assert o.error() == 0
    Rg, Ug, Wg = g.particles()
    Ro, Uo, Wo = o.particles()
    assert np.array_equal(Ug[drv], kw["vel"][drv]) and not Wg[drv].any()
    assert np.abs(Rg - Ro).max() < r_tol
    assert np.abs(Ug - Uo).max() < u_tol
    for kind in (S.VISCOUS, S.CONTACT, S.LUBRICATION, S.TOTAL):
        sg, _ = g.stress(kind)
        so, _ = o.stress(kind)
        assert np.abs(sg - so).max() <= s_tol * max(np.abs(so).max(), 1e-300), kind


def _pair_case(name):
    """Two heavy spheres (rho_p = 1e6) in the pinned two-body settings:
    crossing the Lees-Edwards plane, touching through its image, repelling
    at a gap (Eq. 13), colliding with a dashpot over 200 sub-steps."""
    heavy = dict(rho_p=1e6, tau=1.0, kt_ratio=0.5)
    if name == "le_crossing":
        return (24, [[6.0, 23.0, 6.0], [18.0, 1.0, 18.0]], dict(vel=[[0.0, 0.04, 0.0], [0.0, -0.04, 0.0]],
                **heavy), dict(kind=0, rate=1e-3), 40)
    if name == "le_image_contact":
        return (24, [[12.0, 21.05, 12.0], [8.0, 2.95, 12.0]], dict(kn=100.0, mu=0.0, eta_n=0.0, F0=0.0,
                lub_cut=0.0, **heavy), dict(kind=0, rate=2e-3), 72)
    if name == "double_layer":
        d = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0) * 6.5
        return (24, [[12.0, 12.0, 12.0], list(12.0 + d)], dict(kn=100.0, F0=0.3, debye=0.2, lub_cut=0.0,
                **heavy), dict(kind=0, rate=0.0), 20)
    m = 1e6 * 4.0 / 3.0 * math.pi * 27.0
    return (32, [[12.75, 16.0, 16.0], [19.25, 16.0, 16.0]], dict(vel=[[0.01, 0, 0], [-0.01, 0, 0]], kn=1e9,
            mu=0.0, eta_n=0.3 * math.sqrt(2e9 / m) * m, F0=0.0, lub_cut=0.0, dem_substeps=200, **heavy),
            dict(kind=0, rate=0.0), 60)


@pytest.mark.parametrize("name", ["le_crossing", "le_image_contact", "double_layer", "dashpot"])
def test_two_body_cases_fp64(name):
    L, pos, kw, sh, T = _pair_case(name)
    g, o = _both(L, L, L, [3.0, 3.0], pos, **kw)
    _step(g, o, T, **sh)
    assert o.error() == 0
    Rg, Ug, _ = g.particles()
    Ro, Uo, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max() + 1e-15
    assert (g.owner() == o.owner()).all()
    assert _pop_err(g, o) < 1e-12
    for kind in (S.CONTACT, S.REPULSIVE, S.TOTAL):
        sg, _ = g.stress(kind)
        so, _ = o.stress(kind)
        assert np.abs(sg - so).max() <= 1e-9 * max(np.abs(so).max(), 1e-300), kind

# ---------------------------------------------------------------- edge cases
def test_no_particles_and_minimum_box():
    g = S.Suspension(4, 4, 4, precision="fp32")
    g.step(3, S.make_shear(kind=0, rate=1e-2))
    f = g.populations()
    assert np.isfinite(f).all()
    s, h = g.stress(S.TOTAL)
    assert np.isfinite(s).all() and h.sum() == 0


def test_overlapping_mapped_spheres_are_rejected():
    with pytest.raises(S.SuspError) as e:
        S.Suspension(24, 24, 24, [4.0, 4.0], [[12, 12, 12], [12, 12, 17.0]], precision="fp32")
    assert e.value.status == S.SUSP_EOVERLAP


# -------------------------------------------------------- full-size workload
def test_full_size_dense_shear_fp32():
    """The benchmark workload (96^3, phi_3 = 0.50, N = 882, FP32) in the
    benchmark's launch configuration (tuned), against the oracle on the whole
    box for 40 steps: populations at every step before any node-map flip
    within the FP32 tolerance (flips need the two sides' centres to differ
    by a node's distance from a surface, and every one is checked to lie
    there), centres within 1e-5."""
    w = I.config_dst(phi3=0.50)
    kw = _params(w)
    g, o = _both(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **kw)
    g.tune()
    c = _fp32_particle_comparison(g, o, 40, w.radius, **w.shear)
    print(c)
    c.check(2e-5)
    assert o.error() == 0
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-5