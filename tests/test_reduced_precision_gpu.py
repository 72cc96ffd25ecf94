"""Reduced-precision population storage (FP16 / BF16 deviations n - C^q rho0,
FP32 arithmetic) against the FP64 oracle.

Storage rounding bounds the per-step error: FP16 keeps 11 significant bits of
the scaled deviation (relative 2^-11), BF16 8 bits (2^-8); the deviations are
~1e-3 of the populations in these flows, so the population error after many
steps stays near 1e-5 (FP16) and 1e-4 (BF16) of the populations.  The
time-averaged total stress must agree with the oracle's within 2 % (the
reduced-precision target), checked as a fraction of its largest component
and on the shear component alone; measured on GB300 the errors are about
1e-6 for both storages, so a second bound of 1e-4 guards against a
regression far inside the target.
"""
import numpy as np
import pytest

import oracle as O
from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import susp as S
from parity_helpers import fp32_particle_pop_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,pop_tol", [("fp16", 2e-4), ("bf16", 2e-3)])
def test_deviation_storage_against_oracle(prec, pop_tol):
    stress_tol = 0.02
    w = I.config_small(precision=prec)
    kw = dict(w.params)
    g = S.Suspension(w.nx, w.ny, w.nz, w.radius, w.pos, precision=prec, **kw)
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, w.pos, **kw)
    sh = dict(kind=0, rate=1e-3)
    # FP32 arithmetic moves the centres off the oracle's in the last bits:
    # node-map disagreements are allowed on mapped surfaces (checked inside)
    err = fp32_particle_pop_err(g, o, 200, w.radius, pop_tol, **sh)
    so, _ = o.stress(O.TOTAL)
    sg, _ = g.stress(S.TOTAL)
    serr = np.abs(sg - so).max() / np.abs(so).max()
    print(f"{prec}: population error {err:.2e}, total-stress error {serr:.2e}")
    assert serr < stress_tol
    assert abs(sg[0, 1] - so[0, 1]) <= stress_tol * abs(so[0, 1])
    assert serr < 1e-4


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_deviation_storage_round_trip(prec):
    """set_populations / get_populations round trip loses only storage rounding."""
    _, w, _ = O.lattice()
    f0 = I.random_populations(16, 12, 8, seed=5, amplitude=0.01, weights=w)
    g = S.Suspension(16, 12, 8, precision=prec)
    g.set_populations(f0)
    f1 = g.populations()
    rel = 2.0 ** -11 if prec == "fp16" else 2.0 ** -8
    dev = np.abs(f0 - w[:, None, None, None])
    assert (np.abs(f1 - f0) <= rel * dev + 1e-7).all()
