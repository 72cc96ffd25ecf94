"""The constants the paper prints (tests/golden/paper_parameters.txt, each
line citing its passage) are the ones the oracle's lattice, the input
presets and the observables use."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1904_02929_gb300 import inputs as I
from paper_1904_02929_gb300 import observables as X

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_parameters.txt")):
        if line.startswith("#") or not line.strip():
            continue
        key, rest = line.split("=", 1)
        value, cite = rest.split("|", 1)
        assert cite.strip(), key                   # every value carries its citation
        out[key.strip()] = float(value)
    return out


G = _golden()


def test_lattice_weights():
    C, W, _ = O.lattice()
    C, W = np.asarray(C), np.asarray(W)
    speed2 = (C * C).sum(1)
    assert W[speed2 == 0] == pytest.approx([G["weight_rest"]])
    assert W[speed2 == 1] == pytest.approx([G["weight_nearest"]] * 6)
    assert W[speed2 == 2] == pytest.approx([G["weight_next_nearest"]] * 12)


def test_bidisperse_ratio():
    r = I.bidisperse_radii(8, 3.0)
    assert r.max() / r.min() == pytest.approx(G["radius_ratio"])


def test_monolayer_preset_uses_the_printed_constants():
    w = I.config_monolayer(Lx=64, Ly=64, Lz=28, precision="fp32")
    p = w.params
    a_max = w.nz / G["lz_over_amax"]
    a_min = a_max / G["radius_ratio"]
    assert w.radius.max() == pytest.approx(a_max) and w.radius.min() == pytest.approx(a_min)
    assert p["kt_ratio"] == G["kt_over_kn"] and p["mu"] == G["friction_mu"]
    assert p["lub_delta"] == pytest.approx(G["roughness_over_amin"] * a_min)
    assert p["F0"] == pytest.approx(G["F0_over_kn"] * p["kn"])
    assert p["a_map_ratio"] == G["amap_over_acontact"]
    assert p["lub_cut"] == G["link_scheme_gap"]
    # Delta t = 0.6 tau with tau = sqrt(m0 / kn), lattice time step 1
    m0 = 0.5 * (4 / 3 * math.pi * (a_min ** 3 + a_max ** 3))
    tau_c = math.sqrt(m0 / p["kn"])
    assert 1.0 / tau_c == pytest.approx(G["dt_over_tau"])
    assert w.shear["omega"] * tau_c == pytest.approx(G["omega_tau"])


def test_simple_shear_preset_and_window():
    w = I.config_dst(L=48, phi3=0.3, precision="fp32")
    p = w.params
    a_min = w.radius.min()
    assert p["mu"] == G["friction_mu"] and p["a_map_ratio"] == G["amap_over_acontact"]
    assert p["lub_delta"] == pytest.approx(G["roughness_over_amin"] * a_min)
    assert p["lub_cut"] == G["link_scheme_gap"]
    rate = 1e-3
    assert X.strain_window(rate) == (round(G["strain_window_start"] / rate),
                                     round(G["strain_window_end"] / rate))
