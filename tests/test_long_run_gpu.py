"""Time-averaged stresses of long sheared runs of a dense box against the FP64
oracle, in FP32 and in the reduced-precision storages.

The references are the oracle's own time averages, written by
tests/golden/make_long_run.py (which calls only oracle/): a 48^3 box of
bidisperse spheres (radii 4 / 5.6) at phi_3 = 0.50 with contacts,
double-layer force and lubrication, sheared at 1e-4 for 2000 steps ("slow")
and at 1e-3 for 10000 steps ("chaotic", strain 10).  The bound is the 2 %
that the method's reduced-precision target sets on time-averaged stresses:
on the total stress tensor (as a fraction of its largest component), and on
the shear components of the total stress and of the contact virial.  The
golden files also record how far FP64 runs whose centres differ by 1e-9
drift apart from the reference over the same window, chaos alone (two runs
for the slow case, five for the chaotic one).  In the slow case that spread
is below 5e-4 and the 2 % bound applies as it stands.  In the chaotic case
the FP64 runs themselves differ by up to 8 % in the total shear stress, 11 %
in the contact shear stress and 1 % in the total tensor (a 110-sphere box is
not averaged to 2 % by strain 10), so there each component is held to the
larger of 2 % and three times that spread: a GPU run must stay about as
close to the reference as another FP64 run.  The FP32 and 16-bit paths
round at ~1e-7 of a value in every step, not once at 1e-9, so the chaotic
case also records the spread of FP64 runs whose centres differ by 1e-7
(six runs); the spread used is the larger of the two.  A chaotic
reduced-precision trajectory can also bring two mapped spheres within one
node of each other, which raises the overlap flag (reading R-gap: the
dense boxes sit near that limit at rate 1e-3) where the FP64 reference did
not; the run is then repeated once from the start (the FP32 link sums take
their terms in an order set by atomics, so the repeat follows another
trajectory), and a second flag fails the test.  The measured errors are
printed beside the spread.
"""
import json
import os

import numpy as np
import pytest

from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
KINDS = {"viscous": S.VISCOUS, "contact": S.CONTACT, "total": S.TOTAL}


def _golden(case):
    with open(os.path.join(GOLDEN, f"long_run_{case}.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", ["slow", "chaotic"])
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_time_averaged_stress_of_a_long_dense_run(case, prec):
    ref = _golden(case)
    w = I.config_dst(phi3=0.50, L=48)
    assert [w.nx, w.ny, w.nz] == ref["box"] and w.radius.size == ref["n"]
    kw = dict(w.params)
    kw.pop("quasi2d", None)
    def run():
        g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=prec, **kw)
        g.step(ref["steps"], S.make_shear(kind=0, rate=ref["rate"]))
        return {name: g.stress(kind)[0] for name, kind in KINDS.items()}   # raises on a device flag

    try:
        sgs = run()
    except S.SuspError as e:
        if not (case == "chaotic" and e.status == S.SUSP_EOVERLAP):
            raise
        print(f"{case} {prec}: overlap flag, repeated once")
        sgs = run()
    errs = {}
    for name in KINDS:
        so = np.array(ref["stress"][name])
        sg = sgs[name]
        errs[name] = (np.abs(sg - so).max() / np.abs(so).max(), abs(sg[0, 1] - so[0, 1]) / abs(so[0, 1]))
    # the larger spread of the perturbation scales on record
    scales = [ref[k] for k in ref if k.startswith("chaos_spread_")]
    spread = {name: {c: max(sc[name][c] for sc in scales) for c in ("tensor", "xy")} for name in scales[0]}
    print(f"{case} {prec}: " + ", ".join(
        f"{k} tensor {e[0]:.2e} xy {e[1]:.2e} (FP64 spread {spread[k]['tensor']:.1e} / {spread[k]['xy']:.1e})"
        for k, e in errs.items()))
    k = 3.0 if case == "chaotic" else 0.0
    assert errs["total"][0] <= max(0.02, k * spread["total"]["tensor"])
    assert errs["total"][1] <= max(0.02, k * spread["total"]["xy"])
    assert errs["contact"][1] <= max(0.02, k * spread["contact"]["xy"])
