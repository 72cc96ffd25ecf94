"""Serving loop: requests that arrive while others run are admitted into the
running batch (continuous batching), within an HBM budget, and each result is
the one the same request gives when run alone."""
import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import serve as V
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu


def _pool():
    w = I.config_small()
    kw = dict(w.params)
    small = I.Workload("small", w.nx, w.ny, w.nz, w.radius, w.pos, kw)
    a_min = 4.0
    box = (40, 40, 40)
    n = I.n_for_phi3(0.35, box, a_min, 1.4 * a_min)
    r = I.bidisperse_radii(n, a_min)
    pos = I.place_spheres(box, r, seed=31, min_gap=0.02)
    dense = I.Workload("dense", *box, r, pos, dict(tau=1.0, kn=1e3, kt_ratio=0.5, mu=1.0, F0=0.2,
                                                  debye=0.08, lub_delta=0.04, lub_cut=0.5))
    fluid = I.Workload("fluid", 37, 21, 13, np.zeros(0), np.zeros((0, 3)), dict(tau=0.8))
    return [small, dense, fluid]


def _alone(r, precision):
    g = S.Suspension(r.nx, r.ny, r.nz, r.radius, r.pos, precision=precision, **r.params)
    g.step(r.steps, S.make_shear(**r.shear))
    s, _ = g.stress(S.TOTAL)
    R, _, _ = g.particles()
    g.close()
    return s, R


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("bf16", 1e-5)])
def test_continuous_batching_results_equal_alone(precision, tol):
    pool = _pool()
    reqs = []
    shears = [dict(kind=0, rate=1e-3), dict(kind=1, gamma0=0.05, omega=2e-2, theta=0.0),
              dict(kind=0, rate=3e-3), dict(kind=1, gamma0=0.1, omega=1e-2, theta=1.5707963)]
    for k in range(8):
        w = pool[k % 3]
        # uneven lengths: boxes leave and others join while the rest run on
        reqs.append(V.Request(k, w.nx, w.ny, w.nz, w.radius, w.pos, dict(w.params),
                              shears[k % 4], steps=30 + 10 * (k % 3)))
    # a request that fails: held spheres whose sheared images meet at step 17
    w = pool[0]
    bad = V.Request(8, w.nx, w.ny, w.nz, w.radius, w.pos, dict(w.params, move_particles=False),
                    dict(kind=0, rate=-2e-3), steps=40)
    reqs.insert(2, bad)
    budget = sum(V.footprint(r, precision) for r in reqs[:3])   # ~3 resident at a time
    srv = V.Server(budget, max_boxes=4, chunk=10, precision=precision)
    done = srv.run(reqs)
    rep = srv.report()
    srv.close()
    assert len(done) == 9 and rep["completed"] == 8
    assert rep["peak_resident_bytes"] <= budget
    assert rep["admissions_deferred_on_memory"] > 0
    assert rep["launch_shape"]["tile_rows"] in (4, 8, 16)   # tuned once, mid-run
    # the failure (step 17 of 40) is reported at the first chunk boundary
    # after it happened: the request leaves with steps still to run
    assert bad.error == S.SUSP_EOVERLAP and 0 < bad.remaining <= 40 - 17
    # continuous batching: some request joined after the first chunk while a
    # request admitted before it was still running
    assert any(0 < b.admit_chunk < a.done_chunk and a.admit_chunk < b.admit_chunk
               for a in done for b in done)
    for r in done:
        if r is bad:
            continue
        assert r.error == 0
        s_alone, R_alone = _alone(r, precision)
        scale = max(np.abs(s_alone).max(), 1e-300)
        assert np.abs(r.stress - s_alone).max() <= tol * scale, r.rid
        if len(R_alone):
            assert np.abs(r.positions - R_alone).max() <= tol * 100.0, r.rid
