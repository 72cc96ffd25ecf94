"""Launch-shape tuner: the collide-stream tile height and grid it picks change
no result.  Per-node arithmetic does not depend on the tile a node falls in,
and the trial launches between two steps leave the state as it was, so a
tuned run agrees with an untuned one to the last bits that the summation
order of the link-force and viscous-stress reductions allows (the order in
which a particle's surface nodes are collected varies from run to run)."""
import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu


def _box(precision):
    w = I.config_small()
    kw = dict(w.params)
    kw["precision"] = precision
    return S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)


def _same(a, b, tol):
    fa, fb = a.populations(), b.populations()
    assert np.array_equal(a.owner(), b.owner())
    assert np.abs(fa - fb).max() <= tol * np.abs(fb).max()
    if a.n:
        for xa, xb in zip(a.particles(), b.particles()):
            assert np.abs(xa - xb).max() <= tol * max(1.0, np.abs(xb).max())
    sa, _ = a.stress(S.TOTAL)
    sb, _ = b.stress(S.TOTAL)
    assert np.abs(sa - sb).max() <= max(tol, 1e-6) * np.abs(sb).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("bf16", 1e-3)])
def test_tuned_box_gives_the_untuned_results(precision, tol):
    sh = S.make_shear(kind=1, gamma0=0.05, omega=6e-4, theta=0.3)
    a, b = _box(precision), _box(precision)
    a.step(7, sh)
    b.step(7, sh)
    choice = a.tune()                       # between two steps, mid-run
    assert choice["tile_rows"] in (4, 8, 16)
    assert choice["blocks_per_sm"] >= 1 and choice["us"] > 0.0
    a.step(25, sh)
    b.step(25, sh)
    _same(a, b, tol)
    assert a.time() == b.time()


def test_tuned_batch_gives_the_untuned_results():
    """Uneven boxes (one with an odd x extent); the choice survives a detach."""
    sh = S.make_shear(kind=0, rate=5e-4)
    specs = [(None, "small"), ((37, 21, 13), None), ((48, 40, 24), None)]

    def make():
        out = []
        for shape, _ in specs:
            if shape is None:
                out.append(_box("fp64"))
            else:
                out.append(S.Suspension(*shape, precision="fp64", tau=0.8))
        return out

    tuned, plain = make(), make()
    bt, bp = S.Batch(3), S.Batch(3)
    for x in tuned:
        bt.attach(x, sh)
    for x in plain:
        bp.attach(x, sh)
    bt.step(3)
    bp.step(3)
    with pytest.raises(S.SuspError) as e:
        tuned[0].tune()                     # attached: tune the batch instead
    assert e.value.status == S.SUSP_ESTATE
    choice = bt.tune()
    assert choice["tile_rows"] in (4, 8, 16)
    bt.step(10)
    bp.step(10)
    bt.detach(tuned[1])
    bp.detach(plain[1])
    bt.step(5)
    bp.step(5)
    for a, b in zip(tuned, plain):
        _same(a, b, 1e-12)
    bt.close()
    bp.close()
