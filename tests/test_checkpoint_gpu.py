"""Checkpoint and resume: a run saved mid-way and restored into a fresh handle
continues like the uninterrupted run (same kernels, same order, same inputs;
equal to rounding); mismatched parameters are refused."""
import math

import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_save_load_continues_the_run(precision):
    w = I.config_small()
    kw = dict(w.params)
    sh = S.make_shear(kind=1, gamma0=0.05, omega=2 * math.pi / 400, theta=0.4)
    a = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=precision, **kw)
    a.step(20, sh)
    ck = a.save()
    a.step(15, sh)
    b = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=precision, **kw)
    b.step(3, S.make_shear(kind=0, rate=1e-3))        # unrelated history, then overwritten
    b.load(ck)
    assert b.time()[0] == 20
    b.step(15, sh)
    assert a.time() == b.time()
    fa, fb = a.populations(), b.populations()
    fl = (a.owner() < 0) & (b.owner() < 0)
    assert (a.owner() == b.owner()).all()
    # link-force block sums depend on the order in which surface nodes are
    # staged (shared-memory atomics), so runs agree to rounding, and in BF16
    # storage to one step of the stored deviation
    tol = {"fp64": 1e-12, "fp32": 1e-6, "bf16": 1e-3}[precision]
    assert np.abs(fa[:, fl] - fb[:, fl]).max() <= tol * np.abs(fa[:, fl]).max()
    for xa, xb in zip(a.particles(), b.particles()):
        assert np.abs(xa - xb).max() <= tol * max(1.0, np.abs(xa).max())
    sa, _ = a.stress(S.TOTAL)
    sb, _ = b.stress(S.TOTAL)
    assert np.abs(sa - sb).max() <= 1e-6 * np.abs(sa).max()


def test_load_refuses_other_parameters():
    w = I.config_small()
    a = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision="fp32", **dict(w.params))
    ck = a.save()
    b = S.Suspension(w.nx, w.ny, w.nz, precision="fp32")
    with pytest.raises(S.SuspError) as e:
        b.load(ck)
    assert e.value.status == S.SUSP_EINVAL
    with pytest.raises(S.SuspError):
        a.load(ck[:100])
