"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: lattice
identities, closed forms, conservation laws, an independent brute-force
stream-collide on a tiny lattice, limits of the lubrication functions,
frame indifference, Onsager reciprocity and the protocol of Eq. 16.
"""
import math

import numpy as np
import pytest

import oracle as O


C, W, OPP = O.lattice()
CF = C.astype(np.float64)


# ---------------------------------------------------------------- lattice
def test_d3q19_weights_and_isotropy():
    """Appendix A: C^q = 1/3, 1/18, 1/36; c_s^2 = 1/3; 4th-order isotropy."""
    assert len({tuple(c) for c in C}) == 19
    assert math.isclose(W.sum(), 1.0, abs_tol=1e-15)
    assert W[0] == pytest.approx(1 / 3)
    assert sorted(set(np.round(W, 12))) == sorted({round(1 / 3, 12), round(1 / 18, 12),
                                                   round(1 / 36, 12)})
    np.testing.assert_allclose(W @ CF, 0, atol=1e-16)
    second = np.einsum("q,qa,qb->ab", W, CF, CF)
    np.testing.assert_allclose(second, np.eye(3) / 3, atol=1e-15)
    fourth = np.einsum("q,qa,qb,qc,qd->abcd", W, CF, CF, CF, CF)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(fourth, iso, atol=1e-15)
    for q in range(19):
        np.testing.assert_array_equal(C[OPP[q]], -C[q])


def test_equilibrium_moments():
    """Eq. 4 moments of n^eq: rho, j and rho c_s^2 delta + j j / rho."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho = 0.8 + 0.4 * rng.random()
        j = 0.05 * rng.standard_normal(3)
        f = O.equilibrium(rho, j)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(f @ CF, j, atol=1e-15)
        pi = np.einsum("q,qa,qb->ab", f, CF, CF)
        np.testing.assert_allclose(pi, rho / 3 * np.eye(3) + np.outer(j, j) / rho, atol=1e-14)


# --------------------------------------------------------- fluid, periodic
def _numpy_bgk_periodic(f, tau, steps):
    """Independent brute force: np.roll streaming + BGK, all periodic."""
    f = f.copy()
    for _ in range(steps):
        g = np.empty_like(f)
        for q in range(19):
            # pull: n_q(r) = n*_q(r - c_q); axes of f are (q, z, y, x)
            g[q] = np.roll(f[q], shift=(C[q][2], C[q][1], C[q][0]), axis=(0, 1, 2))
        rho = g.sum(0)
        j = np.einsum("qa,qzyx->azyx", CF, g)
        jc = np.einsum("qa,azyx->qzyx", CF, j)
        jj = (j * j).sum(0)
        feq = W[:, None, None, None] * (rho + 3 * jc + 4.5 * jc ** 2 / rho - 1.5 * jj / rho)
        f = g - (g - feq) / tau
    return f


def test_stream_collide_matches_brute_force_periodic():
    """With zero shear the Lees-Edwards planes reduce to plain periodicity."""
    nx, ny, nz = 6, 5, 4
    rng = np.random.default_rng(2)
    f0 = W[:, None, None, None] * (1 + 0.05 * rng.standard_normal((19, nz, ny, nx)))
    s = O.Oracle(nx, ny, nz, tau=0.7)
    s.set_populations(f0)
    s.step(3, O.shear(0, rate=0.0))
    np.testing.assert_allclose(s.populations(), _numpy_bgk_periodic(f0, 0.7, 3),
                               rtol=0, atol=1e-15)


def test_mass_momentum_conserved_periodic():
    nx, ny, nz = 8, 8, 8
    rng = np.random.default_rng(3)
    f0 = W[:, None, None, None] * (1 + 0.05 * rng.standard_normal((19, nz, ny, nx)))
    s = O.Oracle(nx, ny, nz, tau=0.6)
    s.set_populations(f0)
    s.step(20)
    f = s.populations()
    assert abs(f.sum() - f0.sum()) < 1e-13 * f0.sum()
    np.testing.assert_allclose(np.einsum("qa,qzyx->a", CF, f),
                               np.einsum("qa,qzyx->a", CF, f0), atol=1e-13)


def test_lees_edwards_conserves_mass():
    """Interpolation weights sum to one and the Galilean correction is mass
    neutral over a plane, so total mass is exact with a fractional offset."""
    nx, ny, nz = 10, 8, 4
    rng = np.random.default_rng(4)
    f0 = W[:, None, None, None] * (1 + 0.05 * rng.standard_normal((19, nz, ny, nx)))
    s = O.Oracle(nx, ny, nz, tau=0.9)
    s.set_populations(f0)
    s.step(37, O.shear(0, rate=3.7e-3))
    assert 0 < s.delta < nx and abs(s.delta - (37 * 3.7e-3 * ny) % nx) < 1e-12
    assert abs(s.populations().sum() - f0.sum()) < 1e-12 * f0.sum()


def _couette_state(nx, ny, nz, tau, rate, rho0=1.0):
    """Linear profile u_x = rate (y - y0) plus its first-order non-equilibrium
    part -tau C^q 3 rho c_x c_y rate, stored post-collision."""
    y0 = (ny - 1) / 2
    f = np.zeros((19, nz, ny, nx))
    neq = -tau * W * 3 * rho0 * C[:, 0] * C[:, 1] * rate
    for y in range(ny):
        feq = O.equilibrium(rho0, [rho0 * rate * (y - y0), 0, 0])
        f[:, :, y, :] = (feq + (1 - 1 / tau) * neq)[:, None, None]
    return f


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_fixed_point_and_viscous_stress(tau):
    """P3: under Lees-Edwards shear the linear profile's rho and j are kept to
    round-off for every cell, across the shifted planes, and the viscous
    stress equals eta0 * rate with eta0 = rho0 (tau - 1/2) / 3."""
    nx, ny, nz, rate = 8, 16, 4, 2e-3
    f0 = _couette_state(nx, ny, nz, tau, rate)
    s = O.Oracle(nx, ny, nz, tau=tau)
    s.set_populations(f0)
    s.step(60, O.shear(0, rate=rate))
    f = s.populations()
    np.testing.assert_allclose(f.sum(0), f0.sum(0), rtol=0, atol=1e-13)
    np.testing.assert_allclose(np.einsum("qa,qzyx->azyx", CF, f),
                               np.einsum("qa,qzyx->azyx", CF, f0), rtol=0, atol=1e-13)
    sig, _ = s.stress(O.VISCOUS)
    eta0 = (tau - 0.5) / 3
    assert sig[0, 1] == pytest.approx(eta0 * rate, rel=1e-12)
    assert sig[1, 0] == pytest.approx(eta0 * rate, rel=1e-12)


@pytest.mark.parametrize("tau,tau_bulk", [(0.8, 1.3), (1.2, 0.6)])
def test_couette_shear_stress_under_ladd_operator(tau, tau_bulk):
    """Ladd's operator (reading R-BGK): the Couette shear stress is set by the
    shear eigenvalue alone, eta0 rate with eta0 = rho0 (tau - 1/2) / 3,
    whatever the bulk relaxation time; mass and momentum stay those of the
    linear profile."""
    nx, ny, nz, rate = 8, 16, 4, 2e-3
    f0 = _couette_state(nx, ny, nz, tau, rate)
    s = O.Oracle(nx, ny, nz, tau=tau, collision="ladd", tau_bulk=tau_bulk)
    s.set_populations(f0)
    s.step(60, O.shear(0, rate=rate))
    f = s.populations()
    np.testing.assert_allclose(f.sum(0), f0.sum(0), rtol=0, atol=1e-13)
    np.testing.assert_allclose(np.einsum("qa,qzyx->azyx", CF, f),
                               np.einsum("qa,qzyx->azyx", CF, f0), rtol=0, atol=1e-13)
    sig, _ = s.stress(O.VISCOUS)
    assert sig[0, 1] == pytest.approx((tau - 0.5) / 3 * rate, rel=1e-12)


def test_couette_develops_from_rest():
    """Started at rest, the Lees-Edwards boundary drives the linear profile
    (diffusive time Ly^2 / nu); slope -> rate, sign pinned by the image
    velocity convention."""
    nx, ny, nz, rate = 4, 12, 4, 1e-3
    s = O.Oracle(nx, ny, nz, tau=1.0)
    s.step(6000, O.shear(0, rate=rate))
    f = s.populations()
    ux = (np.einsum("q,qzyx->zyx", CF[:, 0], f) / f.sum(0)).mean(axis=(0, 2))
    slope = np.polyfit(np.arange(ny), ux, 1)[0]
    assert slope == pytest.approx(rate, rel=1e-3)
    assert np.abs(ux - np.polyval(np.polyfit(np.arange(ny), ux, 1), np.arange(ny))).max() < 1e-3 * rate * ny


# ----------------------------------------------------------- bounce-back
def test_rest_state_with_held_sphere_is_exact():
    """A sphere at rest in fluid at rest: bounce-back of the rest state is the
    rest state (Eq. 7 with u_b = 0); no force, populations unchanged."""
    s = O.Oracle(16, 16, 16, radius=[4.0], pos=[[8.2, 7.9, 8.1]], move_particles=False)
    s.step(5)
    own = s.owner()
    f = s.populations()
    fluid = own < 0
    np.testing.assert_allclose(f[:, fluid], np.broadcast_to(W[:, None], f[:, fluid].shape),
                               atol=1e-16)
    F, T = s.hydro()
    np.testing.assert_allclose(F, 0, atol=1e-14)
    np.testing.assert_allclose(T, 0, atol=1e-14)
    assert (~fluid).sum() == pytest.approx(4 / 3 * math.pi * (0.95 * 4) ** 3, rel=0.15)


def _cross_links(own):
    """Links between solid nodes of two different particles, from the node
    map alone (periodic box, no shear): for every node r owned by j and every
    direction p whose source s = r - c_p is owned by i != j, one link of
    particle i with c_q = -c_p pointing from r into i's solid.  Returns a list
    of (i, j, q)."""
    out = []
    for p in range(1, 19):
        src = np.roll(own, shift=tuple(int(v) for v in C[p][::-1]), axis=(0, 1, 2))
        hit = (own >= 0) & (src >= 0) & (src != own)
        for idx in zip(*np.nonzero(hit)):
            out.append((int(src[idx]), int(own[idx]), int(OPP[p])))
    return out


def _touching_pair(vel=None):
    """Two held spheres, a = 4 (mapped 3.8), centres 8.0 apart along a skew
    direction: the mapped spheres are 0.4 apart, so solid nodes of the two
    touch along the gap."""
    d = np.array([0.6, 0.48, 0.64])
    R0 = np.array([8.3, 9.1, 8.7])
    pos = [R0, R0 + 8.0 * d]
    return O.Oracle(24, 24, 24, radius=[4.0, 4.0], pos=pos, vel=vel, move_particles=False)


def test_touching_spheres_at_rest_feel_no_force():
    """Appendix A (i): mapped spheres closer than one spacing have solid nodes
    that are each other's link neighbours.  Two such spheres held in fluid at
    rest must feel no force or torque (hydrostatic balance: a uniform
    pressure exerts no net force on a closed body), and the fluid must stay
    at rest.  The test first shows that the pair has links between the two
    solids, and that without them each sphere would feel the rest pressure of
    its fluid links alone, -sum 2 C^q rho0 c_q over the missing links."""
    s = _touching_pair()
    own = s.owner()[...].transpose(0, 1, 2)
    links = _cross_links(own)
    assert len(links) >= 4
    for i in (0, 1):
        miss = sum(2 * W[q] * CF[q] for (a, _, q) in links if a == i)
        assert np.linalg.norm(miss) > 1e-3          # a dropped link would show
    s.step(5)
    F, T = s.hydro()
    np.testing.assert_allclose(F, 0, atol=1e-13)
    np.testing.assert_allclose(T, 0, atol=1e-13)
    f = s.populations()
    fluid = s.owner() < 0
    np.testing.assert_allclose(f[:, fluid], np.broadcast_to(W[:, None], f[:, fluid].shape),
                               atol=1e-16)


def test_touching_spheres_moving_together_feel_no_force():
    """The same pair held at one velocity U in fluid moving uniformly with U:
    the uniform equilibrium n^eq(rho0, rho0 U) is a fixed point of Eq. 7 with
    u_b = U, so every fluid link carries C^q rho0 [2 + 9 (U.c)^2 - 3 U^2] c_q.
    Those terms sum to zero over a closed link set, so the pair feels no force
    or torque only if a link between the two solids carries the same value,
    i.e. stands for fluid in equilibrium moving with the surfaces.  Counting
    such a link as fluid at rest instead (2 C^q rho0) leaves each sphere with
    a force of order rho0 U^2, computed here to show the test would see it."""
    U = np.array([0.03, -0.02, 0.012])
    s = _touching_pair(vel=[U, U])
    nx = 24
    feq = O.equilibrium(1.0, U)
    s.set_populations(np.broadcast_to(feq[:, None], (19, nx ** 3)).copy())
    links = _cross_links(s.owner())
    for i in (0, 1):
        resid = sum(W[q] * (9 * (U @ CF[q]) ** 2 - 3 * U @ U) * CF[q]
                    for (a, _, q) in links if a == i)
        assert np.linalg.norm(resid) > 1e-6         # the rest reading would show
    s.step(5)
    F, T = s.hydro()
    np.testing.assert_allclose(F, 0, atol=1e-13)
    np.testing.assert_allclose(T, 0, atol=1e-13)
    f = s.populations()
    fluid = s.owner() < 0
    np.testing.assert_allclose(f[:, fluid], np.broadcast_to(feq[:, None], f[:, fluid].shape),
                               atol=1e-15)


def test_touching_spheres_in_relative_motion_conserve_momentum():
    """A link between two solids exchanges momentum between the two spheres
    only (no fluid takes part), so the pair's link forces must cancel exactly
    whatever their velocities: the sum over both spheres of the links between
    them is zero.  Checked as total momentum of fluid + held spheres: the held
    spheres' surfaces inject momentum -sum F^h per step, which must equal the
    fluid's momentum change; with the pair's internal links unbalanced the
    two would differ."""
    Ua = np.array([0.02, -0.01, 0.005])
    Ub = np.array([-0.015, 0.01, 0.02])
    s = _touching_pair(vel=[Ua, Ub])
    fluid = s.owner() < 0

    def jfluid():
        f = s.populations()
        return np.einsum("qa,qn->a", CF, f[:, fluid])

    j0 = jfluid()
    for _ in range(4):
        s.step(1)
        F, _ = s.hydro()
        j1 = jfluid()
        np.testing.assert_allclose(j1 - j0, -F.sum(0), rtol=0, atol=1e-13)
        j0 = j1
    """Eq. 7/8 sign: a sphere held at velocity U in fluid at rest receives a
    force against U and gives the fluid momentum along U; a sphere held at
    spin Omega receives a torque against Omega."""
    U = np.array([[0.01, -0.004, 0.002]])
    s = O.Oracle(20, 20, 20, radius=[4.0], pos=[[10.0, 10.0, 10.0]], vel=U,
                 move_particles=False)
    s.step(20)
    F, _ = s.hydro()
    assert (F[0] @ U[0]) < 0
    f = s.populations()
    fluid = s.owner() < 0
    jf = np.einsum("qa,qn->a", CF, f[:, fluid])
    assert jf @ U[0] > 0
    Om = np.array([[0.0, 0.0, 0.003]])
    s2 = O.Oracle(20, 20, 20, radius=[4.0], pos=[[10.0, 10.0, 10.0]], omega=Om,
                  move_particles=False)
    s2.step(20)
    _, T = s2.hydro()
    assert T[0, 2] < 0 and abs(T[0, 0]) < 1e-3 * abs(T[0, 2])


def test_momentum_conserved_with_moving_particles():
    """P1: fluid + particle momentum + pending covering impulses is constant
    to round-off while spheres move, cover and uncover nodes and touch."""
    rad = [3.0, 3.0, 3.5]
    pos = [[6.0, 8.0, 8.0], [12.4, 8.5, 8.3], [9.0, 14.0, 4.0]]
    vel = [[0.02, 0.0, 0.0], [-0.02, 0.003, 0.0], [0.0, -0.01, 0.01]]
    s = O.Oracle(20, 18, 16, radius=rad, pos=pos, vel=vel, kn=50.0, F0=0.05, debye=0.2,
                 lub_cut=0.5, lub_delta=0.03)
    m = np.array([4 / 3 * math.pi * a ** 3 for a in rad])

    def total():
        f = s.populations()
        fluid = s.owner() < 0
        jf = np.einsum("qa,qn->a", CF, f[:, fluid])
        _, U, _ = s.particles()
        Fp, _ = s.pending()
        return jf + (m[:, None] * U).sum(0) + Fp.sum(0)

    p0 = total()
    nsteps = 0
    for _ in range(6):
        s.step(10)
        nsteps += 10
        np.testing.assert_allclose(total(), p0, rtol=0, atol=1e-12)
    assert s.error() == 0


def test_sphere_crossing_the_lees_edwards_plane():
    """A sphere that leaves through y = L_y re-enters at y = 0 shifted by
    -Delta(t+1) in x with its x velocity lowered by U_LE (and the reverse
    through y = 0): the image box above moves with +U_LE and is offset by
    +Delta.  Heavy spheres (rho_p = 1e6) so the fluid's force changes their
    velocity by ~1e-9 per step; Delta(t) = t L_y rate under a constant rate."""
    L, rate = 24, 1e-3
    ule = L * rate
    o = O.Oracle(L, L, L, [3.0, 3.0], [[6.0, L - 1.0, 6.0], [18.0, 1.0, 18.0]],
                 vel=[[0.0, 0.04, 0.0], [0.0, -0.04, 0.0]], rho_p=1e6, tau=1.0)
    sh = O.shear(kind=0, rate=rate)
    crossed = set()
    for t in range(40):
        R0, U0, _ = o.particles()
        o.step(1, sh)
        R1, U1, _ = o.particles()
        d1 = o.delta
        assert d1 == pytest.approx((t + 1) * ule, rel=1e-12)
        for i in range(2):
            if abs(R1[i, 1] - R0[i, 1]) < L / 2:
                continue
            s = 1 if R1[i, 1] < R0[i, 1] else -1       # +1: out through the top
            dx = R1[i, 0] - (R0[i, 0] + U0[i, 0] - s * d1)
            dx -= L * np.round(dx / L)
            assert abs(dx) < 1e-7, (t, i)
            assert U1[i, 0] - (U0[i, 0] - s * ule) == pytest.approx(0.0, abs=1e-7)
            crossed.add(s)
    assert crossed == {1, -1} and o.error() == 0


def test_contact_across_the_lees_edwards_plane():
    """Two heavy spheres at rest on either side of the y boundary touch only
    through the image box above, offset by +Delta(t): as Delta grows the
    image of B slides over A, and each step's contact virial (sampled at the
    step start, Eq. 12) is the closed form -(kn delta / d) r r / V with
    r = R_A - (R_B + (Delta(t), L_y, 0)), no tangential force (mu = 0) and no
    dashpot; zero before the image reaches A."""
    L, rate, kn = 24, 2e-3, 100.0
    o = O.Oracle(L, L, L, [3.0, 3.0], [[12.0, L - 2.95, 12.0], [8.0, 2.95, 12.0]], rho_p=1e6,
                 tau=1.0, kn=kn, kt_ratio=0.5, mu=0.0, eta_n=0.0, F0=0.0, lub_cut=0.0)
    sh = O.shear(kind=0, rate=rate)
    touching = 0
    for t in range(72):
        R, _, _ = o.particles()
        r = R[0] - (R[1] + np.array([o.delta, L, 0.0]))
        d = np.linalg.norm(r)
        o.stress_reset()
        o.step(1, sh)
        sc, _ = o.stress(O.CONTACT)
        if d < 6.0:
            touching += 1
            expect = -(kn * (6.0 - d) / d) * np.outer(r, r) / L ** 3
            np.testing.assert_allclose(sc, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())
        else:
            assert not sc.any(), t
    assert touching == 11 and o.error() == 0


def test_quasi2d_monolayer_stays_in_its_plane():
    """Quasi-2D constraint of the monolayer (Sec. 4.1): whatever velocities
    and spins the spheres start with, after the first step U_z = 0 and
    Omega_x = Omega_y = 0 exactly and the centres keep their z, while the
    in-plane motion and the contacts go on (48 x 48 x 20, phi = 0.70,
    a_max = L_z / 4)."""
    from paper_1904_02929_gb300 import inputs as I
    w = I.config_monolayer(Lx=48, Ly=48, Lz=20, phi=0.70, precision="fp64")
    kw = dict(w.params)
    rng = np.random.default_rng(5)
    kw["vel"] = rng.normal(0, 3e-3, (w.n, 3))
    kw["omega"] = rng.normal(0, 1e-3, (w.n, 3))
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    z0 = o.particles()[0][:, 2].copy()
    o.step(30, O.shear(kind=0, rate=1e-3))
    R, U, W = o.particles()
    assert o.error() == 0
    assert not U[:, 2].any() and not W[:, :2].any() and np.array_equal(R[:, 2], z0)
    assert np.abs(U[:, :2]).max() > 1e-3 and np.abs(W[:, 2]).max() > 1e-4
    assert o.stress(O.CONTACT)[1][:, 0].sum() > 0


# ---------------------------------------------------------------- contacts
def test_normal_contact_closed_form():
    """Linear spring + dashpot: F = (kn delta_n + eta_n v_n), repulsive,
    equal and opposite, no torque for a central approach."""
    kn, eta = 200.0, 7.0
    d = np.array([7.9, 0.0, 0.0])
    u = np.array([0.01, 0.0, 0.0])             # a approaching b
    t, Fa, Ta, Tb, fn, Ft, ht = O.contact(4.0, 4.0, d, u, [0, 0, 0], [0, 0, 0], kn, 0.2 * kn,
                                          eta, 1.0, 1.0, [0, 0, 0])
    assert t
    assert fn == pytest.approx(kn * 0.1 + eta * 0.01, rel=1e-13)
    np.testing.assert_allclose(Fa, [-fn, 0, 0], atol=1e-14)
    np.testing.assert_allclose(Ta, 0, atol=1e-15)
    np.testing.assert_allclose(Ft, 0, atol=1e-15)
    t, *_ = O.contact(4.0, 4.0, [8.01, 0, 0], u, [0, 0, 0], [0, 0, 0], kn, kn, eta, 1.0, 1.0,
                      [0.3, 0.1, 0.0])
    assert not t


def test_tangential_spring_and_coulomb_slip():
    """Stick: F_t = -kt * integral of v_t; slip once |F_t| reaches mu |F_n|,
    then |F_t| = mu |F_n| exactly with the spring reset to the slip length;
    torque a n x F_t on both spheres (Eq. 11t)."""
    kn, kt, mu = 100.0, 20.0, 0.5
    ra, rb = 4.0, 5.0
    d = np.array([0.0, 8.95, 0.0])              # overlap 0.05, n = +y
    vt = np.array([0.004, 0.0, 0.0])
    ht = np.zeros(3)
    fn_expected = kn * 0.05
    slipped = False
    for k in range(1, 200):
        t, Fa, Ta, Tb, fn, Ft, ht = O.contact(ra, rb, d, vt, [0, 0, 0], [0, 0, 0], kn, kt, 0.0,
                                              mu, 0.5, ht)
        assert fn == pytest.approx(fn_expected, rel=1e-13)
        trial = kt * 0.004 * 0.5 * k
        if trial < mu * fn:
            assert Ft[0] == pytest.approx(-trial, rel=1e-12)
        else:
            slipped = True
            assert np.linalg.norm(Ft) == pytest.approx(mu * fn, rel=1e-13)
            np.testing.assert_allclose(ht, -Ft / kt, rtol=1e-14)
        assert np.linalg.norm(Ft) <= mu * abs(fn) * (1 + 1e-12)
        n = d / np.linalg.norm(d)
        np.testing.assert_allclose(Ta, ra * np.cross(n, Ft), atol=1e-14)
        np.testing.assert_allclose(Tb, rb * np.cross(n, Ft), atol=1e-14)
    assert slipped


def test_tangential_spring_is_projected_onto_the_tangent_plane():
    """When the line of centres turns, the stored spring loses its normal
    part before v_t dt is added (reading R-tangential): with no tangential
    motion the spring comes back as its tangent-plane projection and the
    tangential force is -kt times it, perpendicular to n."""
    d = np.array([0.0, 7.9, 0.0])                # n = +y
    h0 = np.array([0.01, 0.02, -0.005])          # carries a normal (y) part
    t, Fa, Ta, Tb, fn, Ft, ht = O.contact(4.0, 4.0, d, [0, 0, 0], [0, 0, 0], [0, 0, 0], 100.0, 20.0,
                                          0.0, 10.0, 1.0, h0)
    assert t
    np.testing.assert_allclose(ht, [0.01, 0.0, -0.005], rtol=0, atol=1e-17)
    np.testing.assert_allclose(Ft, -20.0 * np.array([0.01, 0.0, -0.005]), rtol=1e-14)
    assert abs(np.dot(Ft, d)) < 1e-15


def test_contact_rolling_without_slip_has_no_tangential_force():
    """Relative surface velocity includes the spins: equal and opposite rolling
    (U_ab = 0, a Omega_a + b Omega_b = 0) loads no tangential spring."""
    d = np.array([7.95, 0.0, 0.0])
    wa = np.array([0.0, 0.0, 0.01])
    wb = -wa * 4.0 / 4.0
    t, Fa, Ta, Tb, fn, Ft, ht = O.contact(4.0, 4.0, d, [0, 0, 0], wa, wb, 100.0, 20.0, 0.0,
                                          1.0, 1.0, [0, 0, 0])
    assert t
    np.testing.assert_allclose(Ft, 0, atol=1e-16)


@pytest.mark.parametrize("h", [0.05, 0.5, 1.9, 2.1])
def test_double_layer_repulsion_virial(h):
    """Eq. 13: two heavy spheres at surface gap h (along a diagonal of the
    x-y plane) repel with F0 exp(-h / lambda) along the line of centres, cut
    off at h = 10 lambda; the step's double-layer virial (Eq. 14) is
    -(F / d) r r / V with r = R_a - R_b."""
    L, F0, lam = 24, 0.3, 0.2
    d = 6.0 + h
    dvec = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0) * d
    pa = np.array([12.0, 12.0, 12.0])
    o = O.Oracle(L, L, L, [3.0, 3.0], [pa, pa + dvec], rho_p=1e6, tau=1.0, kn=100.0, F0=F0,
                 debye=lam, lub_cut=0.0)
    o.step(1, O.shear(kind=0, rate=0.0))
    sr, _ = o.stress(O.REPULSIVE)
    f = F0 * math.exp(-h / lam) if h < 10 * lam else 0.0
    expect = -(f / d) * np.outer(dvec, dvec) / L ** 3
    np.testing.assert_allclose(sr, expect, rtol=1e-12, atol=1e-22)
    assert o.error() == 0


def _restitution(kn, substeps):
    """Head-on collision of two heavy equal spheres (a = 3, relative speed
    0.02, no dashpot, friction, lubrication or repulsion): the ratio of the
    relative speeds after and before."""
    o = O.Oracle(32, 32, 32, [3.0, 3.0], [[12.75, 16.0, 16.0], [19.25, 16.0, 16.0]],
                 vel=[[0.01, 0, 0], [-0.01, 0, 0]], rho_p=1e6, tau=1.0, kn=kn, kt_ratio=0.5,
                 mu=0.0, eta_n=0.0, F0=0.0, lub_cut=0.0, dem_substeps=substeps)
    _, U0, _ = o.particles()
    o.step(60, O.shear(kind=0, rate=0.0))
    _, U, _ = o.particles()
    return -(U[0, 0] - U[1, 0]) / (U0[0, 0] - U0[1, 0]), o.nsub, o.error()


def test_elastic_collision_and_the_substep_rule():
    """Eq. 1 integrated semi-implicitly over the automatic sub-steps: an
    elastic head-on collision (contact frequency sqrt(2 kn / m)) returns the
    approach speed to within the first-order error of the contact's entry and
    exit, the error shrinks as the sub-steps are refined, and one sub-step per
    lattice step at the same stiffness pumps energy into the pair (what the
    automatic count prevents)."""
    e_auto, ns, err = _restitution(1e9, 0)
    m = 1e6 * 4.0 / 3.0 * math.pi * 27.0
    assert ns == math.ceil(math.sqrt(2e9 / m)) and err == 0
    assert 0.85 < e_auto < 1.15
    errs = [abs(_restitution(1e9, k)[0] - 1.0) for k in (5, 10, 20, 50)]
    assert errs == sorted(errs, reverse=True) and errs[-1] < 5e-3
    assert _restitution(1e9, 1)[0] > 2.0


@pytest.mark.parametrize("zeta", [0.1, 0.3])
def test_spring_dashpot_restitution_closed_form(zeta):
    """Normal contact as a linear spring plus a dashpot on the approach speed
    (Eq. 11, reading R-normal): a head-on collision of equal spheres (reduced
    mass m / 2) leaves with the textbook restitution exp(-gamma pi / omega),
    gamma = eta_n / m, omega^2 = 2 kn / m - gamma^2, here at damping ratios
    0.1 and 0.3 with 200 sub-steps per lattice step."""
    m = 1e6 * 4.0 / 3.0 * math.pi * 27.0
    kn = 1e9
    w0 = math.sqrt(2.0 * kn / m)
    g = zeta * w0
    eta_n = g * m
    e_th = math.exp(-g * math.pi / math.sqrt(w0 * w0 - g * g))
    o = O.Oracle(32, 32, 32, [3.0, 3.0], [[12.75, 16.0, 16.0], [19.25, 16.0, 16.0]],
                 vel=[[0.01, 0, 0], [-0.01, 0, 0]], rho_p=1e6, tau=1.0, kn=kn, kt_ratio=0.5,
                 mu=0.0, eta_n=eta_n, F0=0.0, lub_cut=0.0, dem_substeps=200)
    _, U0, _ = o.particles()
    o.step(60, O.shear(kind=0, rate=0.0))
    _, U, _ = o.particles()
    e = -(U[0, 0] - U[1, 0]) / (U0[0, 0] - U0[1, 0])
    assert e == pytest.approx(e_th, rel=5e-3) and o.error() == 0


# ------------------------------------------------------------- lubrication
ETA0 = 1.0 / 6.0


def test_lubrication_reynolds_limit_equal_spheres():
    """P7: for equal spheres the squeeze force is (3/2) pi eta a^2 U / h at
    leading order; with delta = 0 and the cutoff term subtracted the oracle
    gives (3/2) pi eta a^2 U (1/h - 1/h_c) exactly."""
    a, h, hc, U = 4.0, 1e-3, 2.0, 0.01
    d = np.array([0.0, 0.0, 2 * a + h])
    Fa, Ta, Tb = O.lubrication(a, a, d, [0, 0, U], [0, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    expect = 1.5 * math.pi * ETA0 * a * a * U * (1 / h - 1 / hc)
    assert -Fa[2] == pytest.approx(expect, rel=1e-12)
    np.testing.assert_allclose(Fa[:2], 0, atol=1e-16)


@pytest.mark.parametrize("ra,rb", [(3.0, 4.2), (4.2, 3.0), (2.0, 5.0)])
def test_lubrication_reynolds_limit_unequal_spheres(ra, rb):
    """Reynolds' squeeze force between unequal spheres, 6 pi eta (a b / (a +
    b))^2 U / h, minus its value at the cutoff, exactly with delta = 0: the
    leading X^A term 2 beta^2 / (1 + beta)^3 / xi with beta = a_b / a_a and
    xi = 2 h / (a_a + a_b) (reading R-lub); beta the other way round is off
    by ~30 %."""
    h, hc, U = 1e-3, 2.0, 0.01
    d = np.array([0.0, 0.0, ra + rb + h])
    Fa, _, _ = O.lubrication(ra, rb, d, [0, 0, U], [0, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    red = ra * rb / (ra + rb)
    assert -Fa[2] == pytest.approx(6 * math.pi * ETA0 * red ** 2 * U * (1 / h - 1 / hc), rel=1e-11)


def test_lubrication_tangential_log_term():
    """Relative sliding at a small gap: the leading shear resistance is
    logarithmic, 6 pi eta a_a Y^A U_t ln(1/xi) with Jeffrey and Onishi's
    Y^A = 4 beta (2 + beta + 2 beta^2) / (15 (1 + beta)^3) (1/6 for equal
    spheres, i.e. pi eta a U_t ln(1/xi)), here minus its value at the
    cutoff: pi eta a U ln(h_c / h) for equal spheres; and the force does not
    depend on which sphere is called a."""
    h, hc, U = 1e-3, 0.5, 0.01
    a = 4.0
    Fa, _, _ = O.lubrication(a, a, [0, 0, 2 * a + h], [U, 0, 0], [0, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    assert -Fa[0] == pytest.approx(math.pi * ETA0 * a * U * math.log(hc / h), rel=1e-11)
    assert Fa[1] == 0.0 and Fa[2] == 0.0
    ra, rb = 3.0, 4.2
    b = rb / ra
    ya = 4 * b * (2 + b + 2 * b * b) / (15 * (1 + b) ** 3)
    F1, _, _ = O.lubrication(ra, rb, [0, 0, ra + rb + h], [U, 0, 0], [0, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    F2, _, _ = O.lubrication(rb, ra, [0, 0, ra + rb + h], [U, 0, 0], [0, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    assert -F1[0] == pytest.approx(6 * math.pi * ETA0 * ra * ya * U * math.log(hc / h), rel=1e-11)
    assert F2[0] == pytest.approx(F1[0], rel=1e-12)


@pytest.mark.parametrize("ra,rb", [(4.0, 4.0), (3.0, 4.2)])
def test_lubrication_rotation_log_terms(ra, rb):
    """Sphere a spinning about a tangential axis next to sphere b at rest:
    the torques are the logarithmic leading terms of Jeffrey and Onishi,
    T_a = -8 pi eta a_a^3 Y^C_11 Omega, T_b = -8 pi eta a_a^3 Y^C_12 Omega,
    Y^C_11 = 2 beta / (5 (1 + beta)) ln(1/xi), Y^C_12 = beta^2 / (10 (1 + beta))
    ln(1/xi), each minus its value at the cutoff."""
    h, hc, w = 1e-3, 0.5, 0.001
    _, Ta, Tb = O.lubrication(ra, rb, [0, 0, ra + rb + h], [0, 0, 0], [w, 0, 0], [0, 0, 0], ETA0, 0.0, hc)
    b = rb / ra
    unit = 8 * math.pi * ETA0 * ra ** 3 * w * math.log(hc / h)
    assert -Ta[0] == pytest.approx(2 * b / (5 * (1 + b)) * unit, rel=1e-11)
    assert -Tb[0] == pytest.approx(b * b / (10 * (1 + b)) * unit, rel=1e-11)
    assert Ta[1] == Ta[2] == Tb[1] == Tb[2] == 0.0


def test_lubrication_vanishes_at_cutoff_and_beyond():
    a, b = 4.0, 5.6
    for h in (0.5, 0.5000001, 0.7):
        d = np.array([a + b + h, 0.0, 0.0])
        Fa, Ta, Tb = O.lubrication(a, b, d, [0.01, 0.02, -0.01], [0.001, 0, 0.002],
                                   [0, 0.003, 0], ETA0, 0.04, 0.5)
        assert np.abs(Fa).max() < 1e-14 and np.abs(Ta).max() < 1e-13


@pytest.mark.parametrize("ra,rb", [(4.0, 4.0), (4.0, 5.6), (5.6, 4.0)])
def test_lubrication_frame_indifference(ra, rb):
    """A touching pair rotating rigidly has no relative surface motion: the
    leading-order tangential force and both torques vanish.  This holds only
    with beta = a_b / a_a in the printed Y^A, Y^B, Y^C functions."""
    d = np.array([ra + rb, 0.0, 0.0]) * 1.00001
    Om = np.array([0.0, 0.002, 0.005])
    uab = np.cross(Om, -d)                       # U_a - U_b = Om x (R_a - R_b)
    Fa, Ta, Tb = O.lubrication(ra, rb, d, uab, Om, Om, ETA0, 0.0, 0.5)
    scale = ETA0 * 6 * math.pi * ra * np.linalg.norm(uab)
    assert np.abs(Fa).max() < 1e-3 * scale
    assert np.abs(Ta).max() < 1e-3 * scale * ra
    assert np.abs(Tb).max() < 1e-3 * scale * rb


def _resistance_matrix(ra, rb, d):
    """12 x 12 map (U_a, U_b, W_a, W_b) -> (F_a, F_b, T_a, T_b) probed column by column."""
    M = np.zeros((12, 12))
    for k in range(12):
        e = np.zeros(12)
        e[k] = 1.0
        Ua, Ub, Wa, Wb = e[0:3], e[3:6], e[6:9], e[9:12]
        Fa, Ta, Tb = O.lubrication(ra, rb, d, Ua - Ub, Wa, Wb, ETA0, 0.04, 0.5)
        M[:, k] = np.concatenate([Fa, -Fa, Ta, Tb])
    return M


@pytest.mark.parametrize("ra,rb", [(4.0, 4.0), (4.0, 5.6)])
def test_lubrication_reciprocity_and_dissipation(ra, rb):
    """Lorentz reciprocity (A_ab = A_ba^T and its B, C analogues, Appendix A):
    the resistance matrix is symmetric, and it is negative semidefinite."""
    d = np.array([0.3, -0.2, 1.0])
    d = d / np.linalg.norm(d) * (ra + rb + 0.1)
    M = _resistance_matrix(ra, rb, d)
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.max() < 1e-10 * np.abs(ev).max()


# --------------------------------------------------------------- protocol
def test_oscillatory_protocol_eq16():
    """P9: gamma(2 pi k / omega) = 0, dgamma/dt = omega gamma0 sin(omega t + Theta),
    and the summed per-step increments return the offset to zero after a cycle."""
    period = 1000
    om = 2 * math.pi / period
    for theta in (0.0, math.pi / 2, 1.1):
        sh = O.shear(1, gamma0=0.7, omega=om, theta=theta)
        for k in range(3):
            assert abs(O.gamma(sh, k * period)) < 1e-12
        for t in (13.0, 250.5, 777.0):
            eps = 1e-4
            num = (O.gamma(sh, t + eps) - O.gamma(sh, t - eps)) / (2 * eps)
            assert num == pytest.approx(om * 0.7 * math.sin(om * t + theta), rel=1e-6, abs=1e-12)
        ly = 24.0
        tot = sum(O.le_increment(sh, t, ly) for t in range(period))
        assert abs(tot) < 1e-12
    s = O.Oracle(8, 24, 4, tau=1.0)
    s.step(period, O.shear(1, gamma0=0.7, omega=om, theta=math.pi / 2))
    d = s.delta
    assert min(d, 8 - d) < 1e-9


# -------------------------------------------------------- angular stress
def test_angular_stress_eq26_matches_virial_normal_part():
    """P8: monodisperse disks, contacts at bin centres with |r| = 2a: Eq. 26's
    normal part equals the pairwise virial of Eq. 12 per unit area (with the
    opposite sign convention: Eq. 26 counts compression positive)."""
    nb, a, N, area = 36, 3.0, 50, 4000.0
    rng = np.random.default_rng(5)
    dth = math.pi / nb
    hist = np.zeros((nb, 3))
    vir = np.zeros((2, 2))
    ncont = 0
    for b in range(nb):
        for _ in range(int(rng.integers(0, 4))):
            th = (b + 0.5) * dth
            F = float(rng.uniform(0.1, 2.0))
            n = np.array([math.cos(th), math.sin(th)])
            hist[b] += [1, F, 0.0]
            vir += np.outer(2 * a * n, F * n)      # r_alpha F_beta, r = 2a n, F = F n
            ncont += 1
    phi = N * math.pi * a * a / area
    Z = 2 * ncont / N
    sig = O.angular_stress(hist, phi, Z, a, True)
    np.testing.assert_allclose(sig[:2, :2], vir / area, rtol=1e-12)
    rho = hist[:, 0] / (ncont * dth)
    assert (rho * dth).sum() == pytest.approx(1.0, rel=1e-14)       # Eq. 23


def test_angular_stress_eq27_as_printed_is_twice_the_virial():
    """Eq. 27 is implemented as printed.  With rho normalised over [0, pi)
    (Eq. 23) its prefactor 3 phi_3 Z <F> / (2 pi a^2) gives twice the pairwise
    virial of coplanar monodisperse contacts, while Eq. a18 / a19 (prefactor
    3/4, rho normalised over [0, 2 pi) by Eq. a14) gives the virial itself."""
    nb, a, N, V = 24, 4.5, 40, 30000.0
    rng = np.random.default_rng(6)
    dth = math.pi / nb
    hist = np.zeros((nb, 3))
    vir = np.zeros((2, 2))
    nc = 0
    for b in range(nb):
        for _ in range(int(rng.integers(0, 4))):
            th = (b + 0.5) * dth
            F = float(rng.uniform(0.1, 2.0))
            n = np.array([math.cos(th), math.sin(th)])
            hist[b] += [1, F, 0.0]
            vir += np.outer(2 * a * n, F * n)
            nc += 1
    phi3 = N * 4 / 3 * math.pi * a ** 3 / V
    Z = 2 * nc / N
    sig = O.angular_stress(hist, phi3, Z, a, False)
    np.testing.assert_allclose(sig[:2, :2], 2 * vir / V, rtol=1e-12)


def test_angular_stress_eq26_matches_full_virial_with_tangential_forces():
    """P8 with friction: monodisperse disks, contacts at bin centres with
    |r| = 2a carrying normal AND tangential forces.  The third histogram
    column holds the tangential force counted positive when it turns the
    spheres counter-clockwise (Sec. 3.2, Eq. 22): the force on the sphere at
    the tip of r = R_a - R_b is then F_n n - xi t, since its torque about the
    centre, (-a n) x (F_n n - xi t), is +a xi along z.  Eq. 26 as printed,
    [zeta_N n_alpha - zeta_T t_alpha] n_beta (force index first, Appendix C),
    must then equal the full virial (1/A) sum F_alpha r_beta, compression
    positive, including its antisymmetric part.  A flipped sign of the
    tangential term, a transposed index order or a dropped column fails."""
    nb, a, N, area = 36, 2.5, 60, 5000.0
    rng = np.random.default_rng(11)
    dth = math.pi / nb
    hist = np.zeros((nb, 3))
    vir = np.zeros((2, 2))
    ncont = 0
    for b in range(nb):
        for _ in range(int(rng.integers(0, 4))):
            th = (b + 0.5) * dth
            Fn = float(rng.uniform(0.1, 2.0))
            xi = float(rng.uniform(-1.0, 1.0)) * Fn
            n = np.array([math.cos(th), math.sin(th)])
            t = np.array([-math.sin(th), math.cos(th)])
            Fa = Fn * n - xi * t
            torque = np.cross(np.append(-a * n, 0.0), np.append(Fa, 0.0))[2]
            assert torque == pytest.approx(a * xi, abs=1e-14)   # CCW for xi > 0
            hist[b] += [1, Fn, xi]
            vir += np.outer(Fa, 2 * a * n)          # F_alpha r_beta
            ncont += 1
    assert np.abs(vir - vir.T).max() > 1e-3 * np.abs(vir).max()   # asymmetric on purpose
    phi = N * math.pi * a * a / area
    Z = 2 * ncont / N
    sig = O.angular_stress(hist, phi, Z, a, True)
    np.testing.assert_allclose(sig[:2, :2], vir / area, rtol=1e-12, atol=1e-15)


def test_histogram_of_a_single_contact():
    """A single overlapping pair, fluid held at rest: one histogram count in
    the bin of the contact angle, the normal force of the spring law, and the
    contact virial -r F / V of Eq. 12."""
    th = 0.3
    r = 8.9
    pa = np.array([20.0, 20.0, 20.0])
    pb = pa - r * np.array([math.cos(th), math.sin(th), 0.0])   # r_ab = R_a - R_b at angle th
    kn = 300.0
    s = O.Oracle(40, 40, 40, radius=[4.5, 4.5], pos=[pa, pb], kn=kn, eta_n=0.0, lub_cut=0.0,
                 dem_substeps=1)
    s.step(1)
    _, hist = s.stress(O.CONTACT)
    b = int(th / (math.pi / 36))
    assert hist[b, 0] == 1 and hist[:, 0].sum() == 1
    assert hist[b, 1] == pytest.approx(kn * 0.1, rel=1e-9)
    sig, _ = s.stress(O.CONTACT)
    n = np.array([math.cos(th), math.sin(th), 0.0])
    expect = -np.outer(r * n, kn * 0.1 * n) / 40 ** 3
    np.testing.assert_allclose(sig, expect, rtol=1e-8, atol=1e-18)


@pytest.mark.parametrize("th,tip_first", [(math.pi / 2, True), (math.pi / 2, False), (0.9, True),
                                           (2.4, False)])
def test_histogram_tangential_column_is_counter_clockwise(th, tip_first):
    """Sec. 3.2, Eq. 22: the tangential column of the histogram is the
    tangential contact force counted positive when it turns the spheres
    counter-clockwise.  One overlapping pair in the x-y plane, the sphere at
    the tip of the contact direction n = (cos th, sin th) sliding along the
    tangent t: the first sub-step loads the tangential spring by the sliding
    displacement, so the force on the tip sphere is -k_t v dt along the
    sliding direction.  The expected value is that force's torque about the
    tip sphere's centre (contact point at -a n) divided by a.  The sphere
    index order must not matter (a contact counts once, in the bin of the
    folded angle); the force on the wrong sphere or a flipped tangent fails."""
    a, r, kn, kt_ratio, vt = 4.5, 8.9, 300.0, 0.2, 0.012
    n = np.array([math.cos(th), math.sin(th), 0.0])
    t = np.array([-math.sin(th), math.cos(th), 0.0])
    tip = np.array([20.0, 20.0, 20.0])
    base = tip - r * n
    vtip = vt * t
    pos, vel = ([tip, base], [vtip, np.zeros(3)]) if tip_first else ([base, tip], [np.zeros(3), vtip])
    s = O.Oracle(40, 40, 40, radius=[a, a], pos=pos, vel=vel, kn=kn, kt_ratio=kt_ratio,
                 eta_n=0.0, lub_cut=0.0, mu=1.0, dem_substeps=1)
    s.step(1)
    _, hist = s.stress(O.CONTACT)
    F_tip = -kt_ratio * kn * vtip * 1.0                  # spring loaded over dt = 1
    expect = np.cross(-a * n, F_tip)[2] / a
    b = int((th % math.pi) / (math.pi / 36))
    assert hist[b, 0] == 1 and hist[:, 0].sum() == 1
    assert hist[b, 1] == pytest.approx(kn * (2 * a - r), rel=1e-9)
    assert hist[b, 2] == pytest.approx(expect, rel=1e-9)
    assert abs(expect) == pytest.approx(kt_ratio * kn * vt, rel=1e-12)


# ------------------------------------------------------- moduli (Eq. 17, 18)
@pytest.mark.parametrize("theta", [0.0, math.pi / 2, 0.7])
def test_moduli_of_a_newtonian_fluid(theta):
    """A particle-free Lees-Edwards box is a Newtonian fluid: its volume-mean
    shear stress is eta0 * gamma_dot(t) at every step (the mean velocity
    gradient is the plane's velocity jump over L_y), so Eq. 17, 18 give
    G'' = eta0 omega and G' = 0 over whole periods, for any phase Theta.
    A phase taken at t instead of t + 1/2, a swapped cos / sin or a lost
    factor 2 fails this."""
    P = 2000
    om, g0, tau = 2 * math.pi / P, 0.05, 1.0
    o = O.Oracle(4, 8, 4, tau=tau)
    sh = O.shear(kind=1, gamma0=g0, omega=om, theta=theta)
    o.step(P, sh)                       # one period to settle
    o.stress_reset()
    o.step(2 * P, sh)                   # two periods measured
    gp, gpp = o.moduli(g0)
    eta0 = (tau - 0.5) / 3.0
    assert gpp == pytest.approx(eta0 * om, rel=1e-5)
    assert abs(gp) < 1e-6 * eta0 * om


# ------------------------------------------------- derived observables (host)
def test_stress_anisotropy_and_scalings():
    """Delta lambda / P (Sec. 3.3) from the eigenvalues: a diagonal tensor
    gives its extreme entries, any rotation of it the same numbers; the
    reduced rate and the dimensionless moduli are the printed ratios."""
    from paper_1904_02929_gb300 import observables as X
    d = np.diag([-1.0, -2.5, -4.0])
    dl, p, r = X.stress_anisotropy(d)
    assert dl == pytest.approx(3.0) and p == pytest.approx(2.5) and r == pytest.approx(1.2)
    q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    dl2, p2, _ = X.stress_anisotropy(q @ d @ q.T)
    assert dl2 == pytest.approx(dl, rel=1e-12) and p2 == pytest.approx(p, rel=1e-12)
    # simple shear stress sigma_xy = s, no normal stress: eigenvalues +s, 0, -s
    s = 0.3
    dl3, p3, _ = X.stress_anisotropy([[0, s, 0], [s, 0, 0], [0, 0, 0]])
    assert dl3 == pytest.approx(2 * s) and p3 == pytest.approx(0.0, abs=1e-15)
    # monolayer form: only the x-y block counts, whatever sigma_zz is
    d2 = np.diag([-1.0, -3.0, -40.0])
    dl4, p4, r4 = X.stress_anisotropy_2d(d2)
    assert dl4 == pytest.approx(2.0) and p4 == pytest.approx(2.0) and r4 == pytest.approx(1.0)
    c, sn = math.cos(0.7), math.sin(0.7)
    rz = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1.0]])
    dl5, p5, _ = X.stress_anisotropy_2d(rz @ d2 @ rz.T)
    assert dl5 == pytest.approx(dl4, rel=1e-12) and p5 == pytest.approx(p4, rel=1e-12)
    dl6, p6, _ = X.stress_anisotropy_2d([[0, s, 0], [s, 0, 0], [0, 0, -9.0]])
    assert dl6 == pytest.approx(2 * s) and p6 == pytest.approx(0.0, abs=1e-15)
    # averaging window of Sec. 3.1 (gamma = 5 .. 11) and the walls' nominal rate
    assert X.strain_window(1e-4) == (50000, 110000)
    assert X.strain_window(3e-4) == (16667, 36666)
    with pytest.raises(ValueError):
        X.strain_window(0.0)
    assert X.wall_shear_rate(0.02, 4.0, 43.0) == pytest.approx(0.02 / 39.0)
    eta0 = X.solvent_viscosity(1.0)
    assert eta0 == pytest.approx(1.0 / 6.0)
    assert X.reduced_shear_rate(1e-4, eta0, 4.0, 0.2) == pytest.approx(6 * math.pi * eta0 * 16 * 1e-4 / 0.2)
    assert X.relative_viscosity(eta0 * 1e-3, 1e-3, eta0) == pytest.approx(1.0)
    gps, gpps, es = X.dimensionless_moduli(2.0, 3.0, 1e3, 6e-4, 1.0 / 0.6)
    assert (gps, gpps) == (2e-3, 3e-3) and es == pytest.approx(3e-3 / 1e-3)


# ----------------------------------------- Ladd's linear collision operator
def _mode_decay(collision, tau, tau_bulk, shear_wave, L=32, T=320, eps=1e-3):
    """Decay rate and frequency of one Fourier mode of a periodic 32 x 4 x 4
    box: a density (sound) wave along x, or a transverse velocity wave
    u_x(y) (shear); no Lees-Edwards offset (rate 0)."""
    from scipy.optimize import curve_fit
    C, W, _ = O.lattice()
    C, W = np.asarray(C, dtype=float), np.asarray(W)
    nx, ny, nz = (L, 4, 4) if not shear_wave else (4, L, 4)
    o = O.Oracle(nx, ny, nz, tau=tau, collision=collision, tau_bulk=tau_bulk)
    k = 2 * np.pi / L
    f = np.zeros((19, nz, ny, nx))
    if shear_wave:
        y = np.arange(ny)
        for yy in range(ny):
            feq = O.equilibrium(1.0, np.array([eps * np.sin(k * yy), 0.0, 0.0]))
            f[:, :, yy, :] = np.asarray(feq)[:, None, None]
    else:
        x = np.arange(nx)
        rho = 1 + eps * np.cos(k * x)
        f[:] = W[:, None, None, None] * rho[None, None, None, :]
    o.set_populations(f.reshape(19, -1))
    sh = O.shear(kind=0, rate=0.0)
    amp = []
    for t in range(T):
        fp = o.populations().reshape(19, nz, ny, nx)
        if shear_wave:
            ux = np.tensordot(C[:, 0], fp, axes=1).mean(axis=(0, 2))
            amp.append(2.0 / ny * np.sum(ux * np.sin(k * np.arange(ny))))
        else:
            r = fp.sum(0).mean(axis=(0, 1))
            amp.append(2.0 / nx * np.sum((r - 1) * np.cos(k * np.arange(nx))))
        o.step(1, sh)
    t, a = np.arange(T, dtype=float), np.array(amp)
    if shear_wave:
        g = -np.polyfit(t, np.log(a), 1)[0]
        return g, 0.0, k
    fn = lambda t, A, B, G, w: np.exp(-G * t) * (A * np.cos(w * t) + B * np.sin(w * t))
    p, _ = curve_fit(fn, t, a, p0=[eps, 0.0, 0.005, k / np.sqrt(3.0)])
    return p[2], p[3], k


@pytest.mark.parametrize("collision,tau,tau_bulk", [("bgk", 0.8, 0.8), ("ladd", 0.8, 1.5), ("ladd", 0.7, 0.6)])
def test_sound_damping_fixes_the_bulk_eigenvalue(collision, tau, tau_bulk):
    """A standing sound wave oscillates at c_s k and decays at
    k^2 (4 nu / 3 + nu_v) / 2 with nu = (tau - 1/2) / 3 and the bulk
    viscosity nu_v = 2 (tau_v - 1/2) / 9 (BGK: tau_v = tau, so nu_v = 2 nu / 3);
    Ladd's operator moves only the bulk part with tau_bulk."""
    g, w, k = _mode_decay(collision, tau, tau_bulk, shear_wave=False)
    nu = (tau - 0.5) / 3.0
    nuv = 2.0 * ((tau if collision == "bgk" else tau_bulk) - 0.5) / 9.0
    assert g == pytest.approx(0.5 * k * k * (4.0 * nu / 3.0 + nuv), rel=1e-2)
    assert w == pytest.approx(k / math.sqrt(3.0), rel=1e-2)


@pytest.mark.parametrize("tau_bulk", [0.6, 1.5])
def test_shear_wave_decay_fixes_the_shear_eigenvalue(tau_bulk):
    """A transverse wave u_x(y) decays at nu k^2 whatever the bulk eigenvalue."""
    g, _, k = _mode_decay("ladd", 0.8, tau_bulk, shear_wave=True)
    assert g == pytest.approx((0.8 - 0.5) / 3.0 * k * k, rel=1e-2)


def test_ladd_at_tau_one_is_the_equilibrium_like_bgk():
    """At tau = tau_bulk = 1 every non-conserved mode is removed by both
    operators: the populations after a step are n^eq of the pulled moments,
    the same (to rounding) for a sheared box with held spheres."""
    from paper_1904_02929_gb300 import inputs as I
    w = I.config_small(n=6)
    kw = dict(w.params)
    kw["move_particles"] = False
    a = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, collision="bgk", **kw)
    b = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, collision="ladd", tau_bulk=1.0, **kw)
    sh = O.shear(kind=0, rate=2e-3)
    a.step(5, sh)
    b.step(5, sh)
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() < 1e-14


# ------------------------------------------- drag on a periodic sphere array
def _hasimoto_K(c):
    """Drag correction of a simple cubic array of spheres at volume fraction
    c (Hasimoto's series with Sangani and Acrivos' higher terms):
    F = 6 pi eta a U / K(c)."""
    return (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2 + 3.9799 * c ** (8 / 3)
            - 3.0734 * c ** (10 / 3))


def hasimoto_radius(L, eta, U, F):
    """Radius of the sphere whose Hasimoto drag at superficial velocity U in
    a cubic array of period L is F."""
    from scipy.optimize import brentq
    f = lambda r: 6.0 * math.pi * eta * r * U / _hasimoto_K(4.0 * math.pi / 3.0 * r ** 3 / L ** 3) - F
    return brentq(f, 0.05 * L, 0.45 * L)


def test_drag_on_a_periodic_sphere_array_against_hasimoto():
    """A held sphere (a = 3.4, mapped radius 3.23) in a periodic 16^3 box,
    the fluid driven by a uniform body force g, run to steady state: the drag
    balances the body force on the fluid nodes (momentum), and read through
    Hasimoto's series at the measured superficial velocity U it belongs to a
    sphere of the mapped radius within 3 % (the bounce-back links cross the
    mapped sphere at their midpoints).  A lost factor in the momentum
    exchange (Eq. 6), the bounce-back term (Eq. 7) or the viscosity fails
    this."""
    L, a, tau, g = 16, 3.4, 1.0, 1e-6
    o = O.Oracle(L, L, L, np.array([a]), np.array([[L / 2, L / 2, L / 2]]), tau=tau,
                 move_particles=False, body_force=(g, 0.0, 0.0), F0=0.0, lub_cut=0.0)
    eta = (tau - 0.5) / 3.0
    o.step(2400, O.shear(kind=0, rate=0.0))     # about 12 decay times of the mean flow
    F, _ = o.hydro()
    C, _, _ = O.lattice()
    f = o.populations().reshape(19, -1)
    fluid = (o.owner() < 0).ravel()
    U = (np.asarray(C, dtype=float)[:, 0] @ f)[fluid].sum() / L ** 3
    assert F[0, 0] == pytest.approx(g * fluid.sum(), rel=1e-4)
    assert hasimoto_radius(L, eta, U, F[0, 0]) == pytest.approx(0.95 * a, rel=0.03)
    assert abs(F[0, 1]) < 1e-6 * F[0, 0] and abs(F[0, 2]) < 1e-6 * F[0, 0]


def test_torque_on_a_spinning_sphere():
    """A held sphere spinning at Omega in a periodic 20^3 box: at steady
    state the fluid exerts T = -8 pi eta0 a_h^3 Omega (the rotlet; periodic
    images change it at O(a^3 / L^3)) with a_h the mapped radius within 3 %,
    about the spin axis only, and no net force."""
    L, a, tau, Om = 20, 3.4, 1.0, 1e-4
    eta = (tau - 0.5) / 3.0
    o = O.Oracle(L, L, L, np.array([a]), np.array([[L / 2, L / 2, L / 2]]), tau=tau,
                 omega=np.array([[0.0, 0.0, Om]]), move_particles=False, F0=0.0, lub_cut=0.0)
    o.step(int(10 / (eta * (2 * math.pi / L) ** 2)), O.shear(kind=0, rate=0.0))
    F, T = o.hydro()
    assert T[0, 2] < 0
    a_h = (-T[0, 2] / (8 * math.pi * eta * Om)) ** (1 / 3)
    assert a_h == pytest.approx(0.95 * a, rel=0.03)
    assert np.abs(T[0, :2]).max() < 1e-9 * abs(T[0, 2]) and np.abs(F[0]).max() < 1e-9 * abs(T[0, 2])


def test_einstein_viscosity_of_a_held_sphere():
    """The particle stresslet of the momentum exchange (Eq. 9, 10, reading
    R-sigma_h) carries the symmetric stress of a rigid sphere in shear: one
    held sphere (a_map = 0.95 x 3.4) in a 24^3 Lees-Edwards box raises the
    viscous shear stress by Einstein's 2.5 phi (phi of the mapped radius)
    plus the few per cent of its hydrodynamic radius and the periodic
    images.  The fluid nodes alone average to the imposed eta0 rate (inside
    a rigid sphere the strain rate vanishes), so a missing, halved or
    sign-flipped stresslet falls outside the band."""
    L, a, rate, tau = 24, 3.4, 1e-3, 1.0
    eta0 = (tau - 0.5) / 3.0
    o = O.Oracle(L, L, L, [a], [[L / 2, L / 2, L / 2]], tau=tau, move_particles=False,
                 a_map_ratio=0.95)
    # start from the Couette profile the Lees-Edwards planes impose
    f = np.zeros((19, L, L, L))
    for y in range(L):
        feq = np.asarray(O.equilibrium(1.0, np.array([rate * (y + 0.5 - L / 2), 0.0, 0.0])))
        f[:, :, y, :] = feq[:, None, None]
    o.set_populations(f.reshape(19, -1))
    sh = O.shear(kind=0, rate=rate)
    o.step(150, sh)
    o.stress_reset()
    o.step(100, sh)
    sv, _ = o.stress(O.VISCOUS)
    excess = sv[0, 1] / (eta0 * rate) - 1.0
    phi = 4.0 / 3.0 * math.pi * (0.95 * a) ** 3 / L ** 3
    assert 1.0 < excess / (2.5 * phi) < 1.15
    assert o.error() == 0


# ------------------------------------------ lubrication stresslet (G, H blocks)
@pytest.mark.parametrize("ra,rb,h", [(4.0, 5.6, 0.08), (5.6, 4.0, 0.01), (5.0, 5.0, 0.05), (3.0, 7.0, 0.02)])
def test_lubrication_stresslet_vanishes_for_rigid_rotation(ra, rb, h):
    """A pair turning as one rigid body (U_a - U_b = Omega x (R_a - R_b),
    Omega_a = Omega_b = Omega) deforms no gap, so its near-field stresslet
    must vanish: the printed functions satisfy Y^H_aa + Y^H_ab =
    (a_a + a_b) Y^G_aa exactly when each sphere's beta is partner / own
    radius (the reading the lubrication forces use), leaving only the
    h / (a_a + a_b + h) remainder of the finite gap.  The printed beta =
    a_i / a_j breaks this for unequal spheres."""
    rng = np.random.default_rng(int(100 * ra + 10 * rb))
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    d = (ra + rb + h) * n
    om = rng.normal(size=3) * 1e-3
    uab = np.cross(om, -d)
    S = O.lubrication_stresslet(ra, rb, d, uab, om, om, 1 / 6, 0.04, 0.5)
    SG = O.lubrication_stresslet(ra, rb, d, uab, np.zeros(3), np.zeros(3), 1 / 6, 0.04, 0.5)
    assert np.abs(S).max() / np.abs(SG).max() == pytest.approx(h / (ra + rb + h), rel=1e-9)


def test_lubrication_stresslet_squeeze_and_shape():
    """Equal spheres approaching along n: S = -2 X^G (n n - I/3)(n . U) with
    X^G = eta0 4 pi a^2 (3/8) [1/(xi + delta) - 1/(xi_c + delta)] (the
    correction form of the forces); any motion gives a symmetric traceless
    stresslet; none beyond the cut-off, and it goes to zero at the cut-off."""
    a, eta0, dlt, hc, h = 5.0, 1 / 6, 0.04, 0.5, 0.1
    n = np.array([0.6, 0.8, 0.0])
    u = 2e-3
    Sq = O.lubrication_stresslet(a, a, (2 * a + h) * n, u * n, np.zeros(3), np.zeros(3), eta0, dlt, hc)
    sc = 2.0 / (2 * a)
    XG = eta0 * 4 * math.pi * a * a * 3.0 / 8.0 * (1 / (sc * h + sc * dlt) - 1 / (sc * hc + sc * dlt))
    assert np.allclose(Sq, -2 * XG * (np.outer(n, n) - np.eye(3) / 3) * u, rtol=1e-12, atol=0)
    rng = np.random.default_rng(9)
    S = O.lubrication_stresslet(4.0, 5.6, (9.7) * n, rng.normal(size=3) * 1e-3, rng.normal(size=3) * 1e-3,
                                rng.normal(size=3) * 1e-3, eta0, dlt, hc)
    assert np.abs(S - S.T).max() < 1e-15 and abs(np.trace(S)) < 1e-15
    far = O.lubrication_stresslet(a, a, (2 * a + hc + 1e-9) * n, u * n, np.zeros(3), np.zeros(3), eta0, dlt, hc)
    assert np.abs(far).max() == 0.0
    near_cut = O.lubrication_stresslet(a, a, (2 * a + hc - 1e-9) * n, u * n, np.zeros(3), np.zeros(3), eta0,
                                       dlt, hc)
    assert np.abs(near_cut).max() < 1e-7 * np.abs(Sq).max()     # linear in the distance to h_c


def test_total_stress_is_the_sum_of_its_kinds():
    """Eq. 15 with the lubrication stresslets: the total is viscous +
    contact + double layer + lubrication for a sheared dense box."""
    from paper_1904_02929_gb300 import inputs as I
    w = I.config_small(n=20)
    kw = dict(w.params)
    kw.update(F0=0.2, debye=0.2, lub_cut=0.5, lub_delta=0.04)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, vel=np.random.default_rng(4).normal(0, 1e-3, (w.n, 3)), **kw)
    o.step(6, O.shear(kind=0, rate=2e-3))
    parts = [o.stress(k)[0] for k in (O.VISCOUS, O.CONTACT, O.REPULSIVE, O.LUBRICATION)]
    total, _ = o.stress(O.TOTAL)
    assert np.allclose(total, sum(parts), rtol=1e-12, atol=1e-18)
    lub = parts[3]
    assert np.abs(lub - lub.T).max() <= 1e-12 * max(np.abs(lub).max(), 1e-300)
    assert abs(np.trace(lub)) <= 1e-10 * max(np.abs(lub).max(), 1e-300)


# ----------------------------------------------- bumpy walls (driven spheres)
def _couette_profile(o, w):
    C, _, _ = O.lattice()
    C = np.asarray(C, dtype=float)
    f = o.populations().reshape(19, w.nz, w.ny, w.nx)
    own = o.owner().reshape(w.nz, w.ny, w.nx)
    rho = f.sum(0)
    ux = np.where(own < 0, np.tensordot(C[:, 0], f, axes=1) / rho, np.nan)
    return np.nanmean(ux, axis=(0, 2))


def test_bumpy_walls_move_as_prescribed_and_drive_the_suspension():
    """Wall spheres (driven) keep their velocity whatever the contacts and
    lubrication forces on them, so their centres advance exactly by U t; the
    suspension between them is set in motion, and the fluid's mean velocity
    rises monotonically from -U/2 at the bottom wall to +U/2 at the top one
    (Sec. 3: shear applied by moving bumpy walls made of particles)."""
    from paper_1904_02929_gb300 import inputs as I
    w = I.config_walls(L=32, a_wall=3.0, phi3=0.2, wall_speed=0.02)
    kw = dict(w.params)
    drv = kw["driven"].astype(bool)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    R0, U0, W0 = o.particles()
    T = 200
    o.step(T, O.shear(**w.shear))
    assert o.error() == 0
    R, U, W = o.particles()
    assert np.array_equal(U[drv], U0[drv]) and np.array_equal(W[drv], W0[drv])
    d = R[drv] - R0[drv]
    d[:, 0] -= U0[drv, 0] * T
    d[:, 0] -= w.nx * np.round(d[:, 0] / w.nx)
    assert np.abs(d).max() < 1e-10
    assert np.abs(U[~drv]).max() > 1e-4            # the suspension is driven
    prof = _couette_profile(o, w)
    assert np.all(np.diff(prof) > -1e-9)
    assert prof[0] == pytest.approx(-0.01, rel=0.02) and prof[-1] == pytest.approx(0.01, rel=0.02)
