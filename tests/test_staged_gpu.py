"""The staged collide-stream (source rows brought into shared memory by
tensor copies) against the direct one: the same boxes stepped with either
launch shape give the same populations bit for bit without particles (the
per-node arithmetic is the same; only the viscous-stress sums are reduced
in another order), and with moving particles agree as closely as the direct
kernel agrees with itself from run to run.  Covers FP32, FP16 and BF16 storage, BGK and
Ladd's operator, Lees-Edwards shear with moving particles, ragged boxes
(partial x tiles, an odd L_y), boxes whose x rows are not a multiple of 16
bytes (no tensor map: the staged kernel pulls those from global memory),
and a batch mixing all of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu

_, W_LAT, _ = O.lattice()
PRECS = ["fp32", "fp16", "bf16"]


def _particles_box(precision, **extra):
    box = (40, 36, 20)
    r = np.array([4.0, 4.0, 5.0, 4.5, 4.0, 5.0])
    pos = I.place_spheres(box, r, seed=71, min_gap=0.3)
    vel = np.random.default_rng(72).normal(0, 4e-3, (r.size, 3))
    kw = dict(tau=0.9, kn=300.0, kt_ratio=0.5, mu=0.5, lub_delta=0.04, lub_cut=0.5, vel=vel,
              precision=precision)
    kw.update(extra)
    return (box, r, pos, kw, dict(kind=0, rate=2e-3))


def _fluid_box(precision, box, seed):
    return (box, (), (), dict(tau=0.8, precision=precision),
            dict(kind=1, gamma0=0.04, omega=2 * math.pi / 300, theta=0.2), seed)


def _make(spec):
    box, r, pos, kw, sh = spec[:5]
    g = S.Suspension(*box, r, pos, **kw)
    if len(spec) > 5:
        g.set_populations(I.random_populations(*box, seed=spec[5], amplitude=0.02, weights=W_LAT))
    return g, S.make_shear(**sh)


# With moving particles the link forces' FP32 sums take their terms in an
# order that varies from run to run (the link items are listed by atomics),
# so the same kernel differs from itself in the last bits of the FP32
# arithmetic, which 16-bit storage can round one unit apart.
RUN_TO_RUN = {"fp32": 1e-5, "fp16": 1e-4, "bf16": 1e-3}


def _assert_identical(a, b, precision):
    """Bit for bit without particles; with moving particles within the
    run-to-run spread above."""
    assert np.array_equal(a.owner(), b.owner())
    fa, fb = a.populations(), b.populations()
    if a.n == 0:
        assert np.array_equal(fa, fb)
    else:
        tol = RUN_TO_RUN[precision]
        assert np.abs(fa - fb).max() <= tol * np.abs(fb).max()
        for xa, xb in zip(a.particles(), b.particles()):
            assert np.abs(xa - xb).max() <= tol * max(1.0, np.abs(xb).max())
    sa, _ = a.stress(S.VISCOUS)
    sb, _ = b.stress(S.VISCOUS)
    assert np.abs(sa - sb).max() <= 1e-5 * np.abs(sb).max()


def _specs(precision):
    return [
        _particles_box(precision),
        _particles_box(precision, collision="ladd", tau_bulk=1.2),
        _fluid_box(precision, (72, 27, 10), 81),    # partial x tiles, odd L_y
        _fluid_box(precision, (38, 20, 12), 82),    # x rows not a multiple of 16 bytes
    ]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("case", range(4))
def test_staged_equals_direct(precision, case):
    spec = _specs(precision)[case]
    (d, sh), (s, _) = _make(spec), _make(spec)
    d.set_launch_shape(16, 2, False)
    s.set_launch_shape(4, 2, True)
    assert s.launch_shape()["staged"] and not d.launch_shape()["staged"]
    d.step(25, sh)
    s.step(25, sh)
    _assert_identical(s, d, precision)


@pytest.mark.parametrize("precision", PRECS)
def test_staged_batch_equals_direct_batch(precision):
    specs = _specs(precision)
    direct = [_make(sp) for sp in specs]
    staged = [_make(sp) for sp in specs]
    bd, bs = S.Batch(len(specs)), S.Batch(len(specs))
    for (g, sh) in direct:
        bd.attach(g, sh)
    for (g, sh) in staged:
        bs.attach(g, sh)
    bd.set_launch_shape(16, 2, False)
    bs.set_launch_shape(4, 1, True)
    bd.step(20)
    bs.step(20)
    assert bs.errors() == [0] * len(specs)
    for (a, _), (b, _) in zip(staged, direct):
        _assert_identical(a, b, precision)


def test_launch_shape_arguments():
    g, sh = _make(_fluid_box("fp32", (40, 24, 8), 83))
    with pytest.raises(S.SuspError):
        g.set_launch_shape(16, 2, True)     # staged tiles are 128 x 4 nodes
    with pytest.raises(S.SuspError):
        g.set_launch_shape(12, 2, False)
    h, _ = _make(_fluid_box("fp64", (40, 24, 8), 83))
    with pytest.raises(S.SuspError):
        h.set_launch_shape(4, 2, True)      # FP64 storage has no staged kernel
    shape = g.tune()
    assert shape["tile_rows"] in (4, 8, 16) and shape["blocks_per_sm"] >= 1
    assert shape == dict(g.launch_shape(), us=shape["us"])
