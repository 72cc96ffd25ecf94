"""The serving loop's scheduling on the host, with the device side faked:
FIFO admission within the HBM budget and the batch's slots, chunks no longer
than the shortest remaining request, retirement at the exact step count or
on a device error flag, one launch-shape tuning, and the report's
accounting.  The device path itself is covered by tests/test_serve_gpu.py."""
import numpy as np
import pytest
import torch

from paper_1904_02929_gb300 import serve as V
from paper_1904_02929_gb300 import susp as S

FAILING_NX = 20          # boxes of this width raise an instability flag


class FakeStream:
    cuda_stream = 0

    def synchronize(self):
        pass


class FakeBox:
    def __init__(self, nx, ny, nz, radius=(), pos=(), stream=None, precision=None, **kw):
        self.shape = (nx, ny, nz)
        self.steps = 0
        self.closed = False

    def stress(self, kind=S.TOTAL):
        return np.eye(3) * self.steps, None

    def particles(self):
        return np.zeros((0, 3)), None, None

    def close(self):
        self.closed = True


class FakeBatch:
    log = []

    def __init__(self, max_boxes, stream=None):
        self.members = []
        self.tunes = 0
        FakeBatch.log.append(self)

    def attach(self, box, shear=None):
        self.members.append(box)

    def detach(self, box):
        self.members.remove(box)

    def step(self, n):
        for b in self.members:
            b.steps += n

    def errors(self):
        return [S.SUSP_EUNSTABLE if b.shape[0] == FAILING_NX else 0 for b in self.members]

    def tune(self):
        self.tunes += 1
        return {"tile_rows": 8, "blocks_per_sm": 3, "us": 1.0}

    def close(self):
        pass


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(S, "Suspension", FakeBox)
    monkeypatch.setattr(S, "Batch", FakeBatch)
    clock = {"t": 0.0}

    def tick():
        clock["t"] += 0.001
        return clock["t"]

    def sleep(dt):
        clock["t"] += dt

    monkeypatch.setattr(V.time, "sleep", sleep)
    FakeBatch.log.clear()
    return tick


def _req(rid, steps, arrival=0.0, nx=16):
    return V.Request(rid, nx, 16, 16, np.zeros(0), np.zeros((0, 3)), dict(tau=1.0),
                     dict(kind=0, rate=1e-4), steps, arrival)


def test_budget_fifo_chunks_and_retirement(fake_device):
    one = V.footprint(_req(0, 1), "bf16")
    assert one > 0
    srv = V.Server(hbm_budget=2 * one + one // 2, max_boxes=8, chunk=25)
    reqs = [_req(0, 30), _req(1, 60), _req(2, 10), _req(3, 25, arrival=5.0)]
    done = srv.run(reqs, clock=fake_device)
    rep = srv.report()
    assert rep["requests"] == rep["completed"] == 4 and rep["failed_by_status"] == {}
    # each box ran exactly its request's steps and was released
    for r in done:
        assert r.stress[0, 0] == r.steps and r.box is None
    # two fit the budget: the third waited for the first to retire (no overtaking)
    assert rep["peak_resident_bytes"] <= srv.budget and rep["admissions_deferred_on_memory"] > 0
    admit = {r.rid: r.admit_chunk for r in done}
    assert admit[0] == admit[1] == 0 and admit[2] > 0 and admit[3] >= admit[2]
    assert [r.rid for r in done][:1] == [0]
    assert srv.used == 0 and srv.launch_shape is not None and FakeBatch.log[0].tunes == 1
    # node-steps counted per chunk and per member
    assert srv.node_steps == sum(r.steps for r in reqs) * 16 ** 3


def test_a_failing_box_is_retired_with_its_status(fake_device):
    srv = V.Server(hbm_budget=1 << 40, max_boxes=2, chunk=10)
    reqs = [_req(0, 40), _req(1, 40, nx=FAILING_NX), _req(2, 15)]
    done = srv.run(reqs, clock=fake_device)
    by = {r.rid: r for r in done}
    assert by[1].error == S.SUSP_EUNSTABLE and by[1].stress is None and by[1].done_chunk == 1
    assert by[0].error == 0 and by[0].stress[0, 0] == 40
    # the slot freed by the failure went to the queued request at the next chunk
    assert by[2].admit_chunk == 1 and by[2].stress[0, 0] == 15
    rep = srv.report()
    assert rep["completed"] == 2 and rep["failed_by_status"] == {str(S.SUSP_EUNSTABLE): 1}


def test_a_request_larger_than_the_budget_is_refused(fake_device):
    srv = V.Server(hbm_budget=1024, max_boxes=2)
    with pytest.raises(ValueError):
        srv.submit(_req(0, 10))
