"""The overlapped step (the collide-stream on a second stream beside the
particle kernel, the finalisation after both) against the sequential one:
the same boxes give the same populations, particles and stresses up to the
summation order of the link forces (FP64: 1e-13; FP32: the run-to-run
spread, 1e-5; BF16 storage: one unit in its eighth significant bit, 2^-8,
of the largest population, since an FP32 difference in the last bits can
round a stored population one unit apart and the flow carries it on).  The runs cross the Lees-Edwards planes with moving
spheres, so the collide-stream's wall terms read the particle copy of the
step while the particle kernel writes the next one into a second buffer
(which the finalisation then copies over).
"""
import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu


def _box(precision, dense=False, move=True):
    if dense:
        w = I.config_dst(phi3=0.50, L=48)
        kw = dict(w.params)
        kw.pop("quasi2d", None)
        sh = dict(kind=0, rate=1e-3)
    else:
        w = I.config_small()
        kw = dict(w.params)
        sh = dict(kind=0, rate=2e-3)
    kw["precision"] = precision
    if not move:
        kw["move_particles"] = False
    return S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, **kw), S.make_shear(**sh)


def _assert_close(a, b, tol):
    assert np.array_equal(a.owner(), b.owner())
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= tol * np.abs(fb).max()
    for xa, xb in zip(a.particles(), b.particles()):
        assert np.abs(xa - xb).max() <= tol * max(1.0, np.abs(xb).max())
    for kind in (S.VISCOUS, S.CONTACT, S.TOTAL):
        sa, _ = a.stress(kind)
        sb, _ = b.stress(kind)
        assert np.abs(sa - sb).max() <= 10 * tol * max(np.abs(sb).max(), 1e-300), kind
    assert a.time() == b.time()


@pytest.mark.parametrize("precision,dense,tol", [("fp64", False, 1e-13), ("fp32", False, 1e-5),
                                                 ("fp32", True, 1e-5), ("bf16", True, 2.0 ** -8)])
def test_overlapped_step_equals_sequential(precision, dense, tol):
    (seq, sh), (ovl, _) = _box(precision, dense), _box(precision, dense)
    seq.set_overlap(False)
    ovl.set_overlap(True)
    assert ovl.info().overlap == 1 and seq.info().overlap == 0
    assert ovl.launch_shape()["blocks_per_sm"] == 1
    seq.step(40, sh)
    ovl.step(40, sh)
    _assert_close(ovl, seq, tol)


def test_overlap_needs_moving_particles():
    (seq, sh), (ovl, _) = _box("fp32", move=False), _box("fp32", move=False)
    ovl.set_overlap(True)
    assert ovl.info().overlap == 0          # no particle kernel to overlap
    seq.step(20, sh)
    ovl.step(20, sh)
    _assert_close(ovl, seq, 1e-6)


def test_overlapped_batch_equals_boxes_alone():
    alone = [_box("fp32"), _box("fp32", dense=True)]
    mixed = [_box("fp32"), _box("fp32", dense=True)]
    batch = S.Batch(2)
    for g, sh in mixed:
        batch.attach(g, sh)
    batch.set_overlap(True)
    assert batch.launch_shape()["overlap"]
    batch.step(30)
    for g, sh in alone:
        g.step(30, sh)
    assert batch.errors() == [0, 0]
    for (a, _), (m, _) in zip(alone, mixed):
        _assert_close(m, a, 1e-5)


def test_overlapped_stage_times():
    g, sh = _box("fp32", dense=True)
    g.set_overlap(True)
    g.step(2, sh)
    S.susp_profile(g.h, True)
    g.step(10, sh)
    st, n = S.susp_profile_stages(g.h)
    S.susp_profile(g.h, False)
    assert n == 10
    assert st["collide_stream"] > 0 and min(st.values()) >= 0


def test_tuner_keeps_the_step_in_sequence():
    g, sh = _box("fp32", dense=True)
    g.set_overlap(True)
    assert g.info().overlap == 1
    out = g.tune()
    assert out["overlap"] is False and g.info().overlap == 0
    g.step(5, sh)
    assert g.time()[0] == 5
