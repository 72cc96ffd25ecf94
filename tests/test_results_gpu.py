"""One-transfer read-back of a step's results (susp_read_results): the block
decoded on the host gives exactly what the synchronous getters give at the
same point of the stream, the asynchronous form follows the stream's order
(each block holds the step it was enqueued after), and the block carries the
device status.
"""
import numpy as np
import pytest
import torch

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu

KINDS = (S.VISCOUS, S.CONTACT, S.REPULSIVE, S.LUBRICATION, S.TOTAL, S.ANGULAR)


def _box(precision):
    w = I.config_small()
    kw = dict(w.params)
    kw["precision"] = precision
    return S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, **kw), S.make_shear(kind=0, rate=2e-3)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_results_block_equals_getters(precision):
    g, sh = _box(precision)
    g.step(7, sh)
    buf = g.results_buffer()
    g.read_results(buf)
    for a, b in zip(g.results_particles(buf), g.particles()):
        assert np.array_equal(a, b)
    for kind in KINDS:
        (sa, ha), (sb, hb) = g.results_stress(buf, kind), g.stress(kind)
        assert np.array_equal(sa, sb) and np.array_equal(ha, hb), kind


def test_asynchronous_results_follow_the_stream():
    g, sh = _box("fp64")
    twin, _ = _box("fp64")
    bufs = [g.results_buffer(), g.results_buffer()]
    evs = [torch.cuda.Event(), torch.cuda.Event()]
    seen = []
    for k in range(6):
        g.step(1, sh)
        g.read_results(bufs[k % 2], True)
        evs[k % 2].record(g.stream)
        twin.step(1, sh)
        ref = twin.particles()[0]
        if k > 0:
            # the block of the previous step, read while this step runs
            evs[(k - 1) % 2].synchronize()
            seen.append(np.abs(g.results_particles(bufs[(k - 1) % 2])[0] - prev).max())
        prev = ref
    evs[5 % 2].synchronize()
    seen.append(np.abs(g.results_particles(bufs[5 % 2])[0] - prev).max())
    assert max(seen) <= 1e-12
    for a, b in zip(g.results_particles(bufs[5 % 2]), g.particles()):
        assert np.array_equal(a, b)


def test_results_status_word_and_size():
    g, sh = _box("fp32")
    g.step(2, sh)
    buf = g.results_buffer()
    g.read_results(buf)
    bad = buf.clone()
    bad[:4] = torch.tensor([1, 0, 0, 0], dtype=torch.uint8)   # the overlap bit of the error word
    with pytest.raises(S.SuspError) as e:
        g.results_particles(bad)
    assert e.value.status == S.SUSP_EOVERLAP
    with pytest.raises(S.SuspError) as e:
        g.results_stress(bad)
    assert e.value.status == S.SUSP_EOVERLAP
    short = torch.empty(buf.numel() - 8, dtype=torch.uint8).pin_memory()
    with pytest.raises(S.SuspError) as e:
        g.read_results(short)
    assert e.value.status == S.SUSP_EINVAL
