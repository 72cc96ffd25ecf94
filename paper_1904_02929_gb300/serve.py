"""Serving loop: simulation requests admitted into one running batch.

A request is one box (geometry, physical parameters, shear protocol) to be
advanced a given number of lattice steps, answered with its time-averaged
stress and final particle state.  The server keeps every admitted box
resident in HBM and steps all of them together (``susp_batch_step``) in
chunks; between chunks it

  * retires the requests that reached their step count (read-back, detach,
    workspace released), and those whose box raised a device error flag
    (the request completes with that status; the others carry on),
  * admits queued requests in arrival order while their workspace fits the
    HBM budget and a batch slot is free (continuous batching: a request that
    arrives while others run joins them at the next chunk boundary and its
    steps run in the same launches).

New boxes are created on a stream of their own while the batch's chunk runs
on the GPU, so the set-up of arriving requests overlaps the running work.
After the first chunk the batch's collide-stream launch shape is tuned once
(``susp_batch_tune``) and kept for every later membership.  A
box's results do not depend on the company it keeps: per-node and
per-particle arithmetic is the same alone and in a batch.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import susp as S


@dataclass
class Request:
    """One simulation: geometry + parameters (``params``), shear protocol,
    step count, arrival time (seconds from the start of the run)."""
    rid: int
    nx: int
    ny: int
    nz: int
    radius: np.ndarray
    pos: np.ndarray
    params: dict
    shear: dict
    steps: int
    arrival: float = 0.0
    # filled by the server
    admitted: float | None = None
    done: float | None = None
    stress: np.ndarray | None = None
    positions: np.ndarray | None = None
    remaining: int = 0
    nbytes: int = 0
    error: int = 0            # device status of a failed simulation (0 = completed)
    admit_chunk: int = -1     # server chunk count at admission and at completion
    done_chunk: int = -1
    box: S.Suspension | None = field(default=None, repr=False)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint(req: Request, precision: str) -> int:
    """Device bytes a request holds while resident (its workspace)."""
    p, keep = S.make_params(req.nx, req.ny, req.nz, req.radius, req.pos, precision=precision,
                            **req.params)
    return S.susp_workspace_bytes(p)


class Server:
    """Continuous-batching server on the current CUDA device."""

    def __init__(self, hbm_budget: int, max_boxes: int = 64, chunk: int = 25,
                 precision: str = "bf16", tune: bool = True):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget)
        self.max_boxes = int(max_boxes)
        self.chunk = int(chunk)
        self.precision = precision
        self.stream = torch.cuda.Stream()
        self.setup_stream = torch.cuda.Stream()
        self.batch = S.Batch(self.max_boxes, stream=self.stream)
        self.queue: deque[Request] = deque()
        self.active: list[Request] = []
        self.finished: list[Request] = []
        self.used = 0
        self.peak_used = 0
        self.node_steps = 0
        self.chunks = 0
        self.waits_on_memory = 0
        self.tune = tune
        self.launch_shape = None      # collide-stream shape from the tuner (first full chunk)

    # ---------------------------------------------------------------- intake
    def submit(self, req: Request) -> None:
        req.nbytes = footprint(req, self.precision)
        if req.nbytes == 0 or req.nbytes > self.budget:
            raise ValueError(f"request {req.rid} cannot fit the HBM budget")
        req.remaining = req.steps
        self.queue.append(req)

    def _create(self, now: float) -> list[Request]:
        """Create boxes for queued requests that fit (FIFO; no overtaking)."""
        out = []
        slots = self.max_boxes - len(self.active)
        while self.queue and len(out) < slots:
            r = self.queue[0]
            if self.used + r.nbytes > self.budget:
                self.waits_on_memory += 1
                break
            self.queue.popleft()
            r.box = S.Suspension(r.nx, r.ny, r.nz, r.radius, r.pos, stream=self.setup_stream,
                                 precision=self.precision, **r.params)
            r.admitted = now
            r.admit_chunk = self.chunks
            self.used += r.nbytes
            self.peak_used = max(self.peak_used, self.used)
            out.append(r)
        return out

    def _retire(self, r: Request, now: float, error: int = 0) -> None:
        r.error = error
        if not error:
            try:
                r.stress, _ = r.box.stress(S.TOTAL)
                r.positions = r.box.particles()[0]
            except S.SuspError as e:       # a flag raised in the last chunk
                r.error = e.status
        self.batch.detach(r.box)
        r.box.close()
        r.box = None
        self.used -= r.nbytes
        r.done = now
        r.done_chunk = self.chunks
        self.finished.append(r)

    # ------------------------------------------------------------------ loop
    def run(self, requests: list[Request], clock=time.perf_counter) -> list[Request]:
        """Serve ``requests`` (arrival times relative to the start) to the
        end; returns them in completion order."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        t0 = clock()
        now = lambda: clock() - t0
        while pending or self.queue or self.active:
            t = now()
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            n = 0
            if self.active:
                n = min(self.chunk, min(r.remaining for r in self.active))
                self.batch.step(n)                  # asynchronous on the batch stream
            joining = self._create(now())           # overlaps the chunk on the GPU
            if n:
                self.stream.synchronize()
                self.chunks += 1
                self.node_steps += n * sum(r.ncell for r in self.active)
                t = now()
                status = dict(zip(self.batch.members, self.batch.errors()))
                for r in list(self.active):
                    r.remaining -= n
                    err = status[r.box]
                    if r.remaining == 0 or err:
                        self.active.remove(r)
                        self._retire(r, t, err)
            for r in joining:
                self.batch.attach(r.box, S.make_shear(**r.shear))
                self.active.append(r)
            if self.tune and self.launch_shape is None and self.active and n:
                # once, between two chunks: the choice then holds for every
                # membership (results do not depend on it)
                self.launch_shape = self.batch.tune()
            if not self.active and not self.queue and pending:
                time.sleep(max(0.0, pending[0].arrival - now()))
        self.wall = now()
        return self.finished

    def report(self) -> dict:
        ok = [r for r in self.finished if not r.error]
        lat = np.array([r.latency for r in ok])
        per_k = np.array([r.latency * 1000.0 / r.steps for r in ok])
        wait = np.array([r.admitted - r.arrival for r in ok])
        svc = np.array([r.done - r.admitted for r in ok])
        svc_k = np.array([(r.done - r.admitted) * 1000.0 / r.steps for r in ok])
        pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))}
        failed = {}
        for r in self.finished:
            if r.error:
                failed[str(r.error)] = failed.get(str(r.error), 0) + 1
        return {
            "requests": len(self.finished),
            "completed": len(ok),
            "failed_by_status": failed,
            "wall_s": self.wall,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "latency_per_1000_steps_s": {"p50": float(np.percentile(per_k, 50)),
                                         "p99": float(np.percentile(per_k, 99))},
            "queue_wait_s": pct(wait),
            "service_s": pct(svc),
            "service_per_1000_steps_s": pct(svc_k),
            "aggregate_mlups": self.node_steps / self.wall / 1e6,
            "chunks": self.chunks,
            "hbm_budget_bytes": self.budget,
            "peak_resident_bytes": self.peak_used,
            "admissions_deferred_on_memory": self.waits_on_memory,
            "launch_shape": self.launch_shape,
        }

    def close(self) -> None:
        for r in self.active:
            if r.box is not None:
                r.box.close()
        self.batch.close()


def poisson_requests(pool, rate: float, duration: float, steps: int, seed: int,
                     oscillatory_only: bool = False, amplitudes=(0.1, 1.0),
                     count: int | None = None) -> list[Request]:
    """Requests arriving as a Poisson process of the given rate over
    ``duration`` seconds (or the first ``count`` arrivals, whatever their
    times, when ``count`` is given), each a geometry drawn from ``pool``
    (Workload objects) with a shear protocol drawn from the sweep's ranges:
    constant rate 10^U(-5,-3) (unless ``oscillatory_only``), or oscillatory
    (Eq. 16) with an amplitude from ``amplitudes``, omega 6e-4 and phase
    {0, pi/2}."""
    rng = np.random.default_rng(seed)
    out, t, rid = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate)
        if count is None and t >= duration:
            break
        if count is not None and rid >= count:
            break
        w = pool[int(rng.integers(len(pool)))]
        if not oscillatory_only and rng.random() < 0.5:
            sh = dict(kind=0, rate=float(10 ** rng.uniform(-5, -3)))
        else:
            sh = dict(kind=1, gamma0=float(rng.choice(list(amplitudes))), omega=6e-4,
                      theta=float(rng.choice([0.0, np.pi / 2])))
        out.append(Request(rid, w.nx, w.ny, w.nz, w.radius, w.pos, dict(w.params), sh, steps, t))
        rid += 1
    return out
