"""Batched stepping: boxes of different sizes, particle counts, sub-step counts
and protocols, stepped in lockstep by one launch sequence, give the same
results as the same boxes stepped alone, and as the FP64 oracle.

Per-node and per-particle arithmetic does not depend on which block or warp
does it, so populations and trajectories agree to the last bits the summation
order of the link-force and viscous-stress reductions allows (<= 1e-13
relative).  Boxes join and leave a running batch (continuous batching) without
changing their results.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu


def _mix(precision):
    """Four boxes: dense moving particles (many sub-steps), the small config,
    a held-particle box, and a particle-free box with an odd shape."""
    out = []
    a_min = 4.0
    box = (40, 40, 40)
    n = I.n_for_phi3(0.35, box, a_min, 1.4 * a_min)
    r = I.bidisperse_radii(n, a_min)
    pos = I.place_spheres(box, r, seed=31, min_gap=0.02)
    vel = np.random.default_rng(32).normal(0, 5e-3, (n, 3))
    kw = dict(tau=1.0, kn=1e3, kt_ratio=0.5, mu=1.0, F0=0.2, debye=0.08, lub_delta=0.04,
              lub_cut=0.5, nbins=36, precision=precision)
    out.append((box, r, pos, dict(kw, vel=vel), dict(kind=0, rate=1e-3)))
    w = I.config_small()
    kw = dict(w.params)
    kw["precision"] = precision
    out.append(((w.nx, w.ny, w.nz), w.radius, w.pos, kw,
                dict(kind=1, gamma0=0.05, omega=2 * math.pi / 400, theta=0.3)))
    # held particles under a negative rate (the offset wraps to just below L_x);
    # the rate is small enough that no held sphere meets another's sheared image
    # in the steps run here (at -2e-3 one does at step 17, in the oracle too)
    out.append(((w.nx, w.ny, w.nz), w.radius, w.pos, dict(kw, move_particles=False),
                dict(kind=0, rate=-5e-4)))
    out.append(((37, 21, 13), (), (), dict(tau=0.8, precision=precision), dict(kind=0, rate=3e-3)))
    return out


def _make(spec):
    box, r, pos, kw, sh = spec
    return S.Suspension(*box, r, pos, **kw), S.make_shear(**sh)


def _assert_same(a, b, tol):
    fa, fb = a.populations(), b.populations()
    fl = (a.owner() < 0) & (b.owner() < 0)
    assert (a.owner() == b.owner()).all()
    assert np.abs(fa[:, fl] - fb[:, fl]).max() <= tol * np.abs(fb[:, fl]).max()
    if a.n:
        for xa, xb in zip(a.particles(), b.particles()):
            assert np.abs(xa - xb).max() <= tol * max(1.0, np.abs(xb).max())
    ta, da = a.time()
    tb, db = b.time()
    assert ta == tb and abs(da - db) <= 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
def test_batch_equals_alone(precision, tol):
    specs = _mix(precision)
    alone = [_make(s) for s in specs]
    mixed = [_make(s) for s in specs]
    batch = S.Batch(len(specs))
    for (box, sh) in mixed:
        batch.attach(box, sh)
    assert len(batch) == len(specs)
    steps = 30
    batch.step(steps)
    for (box, sh) in alone:
        box.step(steps, sh)
    for (a, _), (m, _) in zip(alone, mixed):
        _assert_same(m, a, tol)
    # the time-averaged stresses too
    for (a, _), (m, _) in zip(alone, mixed):
        sa, _ = a.stress(S.TOTAL)
        sm, _ = m.stress(S.TOTAL)
        assert np.abs(sa - sm).max() <= 1e-6 * max(np.abs(sa).max(), 1e-300)


def test_batched_box_against_oracle():
    w = I.config_small()
    kw = dict(w.params)
    sh = dict(kind=0, rate=2e-3)
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp64", **kw)
    other = S.Suspension(24, 16, 12, precision="fp64", tau=0.7)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    batch = S.Batch(2)
    batch.attach(other, S.make_shear(kind=0, rate=5e-3))
    batch.attach(g, S.make_shear(**sh))
    batch.step(40)
    o.step(40, O.shear(**sh))
    Rg, _, _ = g.particles()
    Ro, _, _ = o.particles()
    assert np.abs(Rg - Ro).max() < 1e-9
    fo, fg = o.populations(), g.populations()
    fl = (o.owner() < 0) & (g.owner() < 0)
    assert np.abs(fg[:, fl] - fo[:, fl]).max() <= 1e-12 * np.abs(fo[:, fl]).max()


def test_continuous_batching_join_and_leave():
    """A box that joins a running batch, leaves it and continues alone ends
    where a box stepped alone all along does; the others are undisturbed."""
    specs = _mix("fp64")
    ref = [_make(s) for s in specs]
    run = [_make(s) for s in specs]
    batch = S.Batch(3)
    batch.attach(run[0][0], run[0][1])
    batch.attach(run[3][0], run[3][1])
    batch.step(5)
    batch.attach(run[1][0], run[1][1])        # joins at t = 0 while the others are at t = 5
    batch.step(10)
    batch.detach(run[0][0])                   # leaves at t = 15
    run[0][0].step(5, run[0][1])
    batch.step(5)
    run[2][0].step(20, run[2][1])             # never batched
    for (box, sh), steps in zip(ref, (20, 15, 20, 20)):
        box.step(steps, sh)
    for (a, _), (r, _) in zip(run, ref):
        _assert_same(a, r, 1e-13)


def test_batch_state_errors():
    a = S.Suspension(16, 16, 16, precision="fp32")
    b = S.Suspension(16, 16, 16, precision="fp64")
    batch = S.Batch(1)
    with pytest.raises(S.SuspError) as e:
        batch.attach(a)                       # no protocol set yet
    assert e.value.status == S.SUSP_ESTATE
    batch.attach(a, S.make_shear(kind=0, rate=1e-3))
    with pytest.raises(S.SuspError) as e:
        a.step(1, S.make_shear(kind=0, rate=1e-3))
    assert e.value.status == S.SUSP_ESTATE
    with pytest.raises(S.SuspError) as e:
        batch.attach(b, S.make_shear())
    assert e.value.status == S.SUSP_ENOMEM    # full (max_boxes = 1)
    batch.detach(a)
    two = S.Batch(2)
    two.attach(a, S.make_shear(kind=0, rate=1e-3))
    with pytest.raises(S.SuspError) as e:
        two.attach(b, S.make_shear())         # boxes of one batch share the precision
    assert e.value.status == S.SUSP_EINVAL
    two.close()
    batch.close()
    a.step(2, S.make_shear(kind=0, rate=1e-3))
    assert a.time()[0] == 2


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_many_particles_per_warp(precision, tol):
    """Four 96^3 boxes at phi_3 = 0.50 (3528 particles, more than the
    particle kernel's resident warps): the batch takes the path that steps two
    particles per warp, the boxes alone the one-particle-per-warp path.  Only
    the order of the per-particle force sums differs."""
    ws = [I.config_dst(seed=1002 + k, phi3=0.50, precision=precision) for k in range(4)]
    assert sum(w.n for w in ws) > 3000

    def make(w):
        return S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=precision, **w.params)

    alone = [make(w) for w in ws]
    mixed = [make(w) for w in ws]
    batch = S.Batch(len(ws))
    for w, g in zip(ws, mixed):
        batch.attach(g, S.make_shear(**w.shear))
    batch.step(8)
    for w, g in zip(ws, alone):
        g.step(8, S.make_shear(**w.shear))
    assert all(e == 0 for e in batch.errors())
    for a, m in zip(alone, mixed):
        _assert_same(m, a, tol)
    batch.close()
    for g in alone + mixed:
        g.close()
