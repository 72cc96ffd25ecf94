"""Write the FP64 oracle's time-averaged stresses of two long sheared runs of
a dense bidisperse box (test infrastructure: calls only oracle/ and the
seeded input presets).

The box is the 96^3 bulk-shear preset scaled to 48^3: radii 4 / 5.6 (1:1 by
number, Sec. 2), phi_3 = 0.50 (N = 110), k_n = 1e3, k_t = 0.5 k_n, mu = 1,
double-layer force and lubrication correction on.  Cases:

  slow     rate 1e-4 for 2000 steps (strain 0.2);
  chaotic  rate 1e-3 for 10000 steps (strain 10).

Besides the reference run, the script runs the same case with the centres
perturbed by 1e-9 (two seeds for the slow case, five for the chaotic one)
and stores the largest relative difference of each stress kind from the
reference: the spread that chaos alone produces, so that a precision bound
on the time average can be read against it.

    python tests/golden/make_long_run.py slow
    python tests/golden/make_long_run.py chaotic

A stored case can be extended with runs perturbed at another scale, without
running its reference again (the FP64 oracle is deterministic): the spread
of those runs is stored beside the first as chaos_spread_<eps>.  The FP32
and 16-bit paths round at ~1e-7 of a value every step, so the chaotic case
also carries the spread of centres perturbed by 1e-7:

    python tests/golden/make_long_run.py chaotic --extend 1e-7 6
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

CASES = {"slow": dict(rate=1e-4, steps=2000, seeds=2), "chaotic": dict(rate=1e-3, steps=10000, seeds=5)}
KINDS = {"viscous": 0, "contact": 1, "repulsive": 2, "total": 3, "lubrication": 5}


def workload():
    sys.path.insert(0, ROOT)
    from paper_1904_02929_gb300 import inputs as I
    w = I.config_dst(phi3=0.50, L=48)
    kw = dict(w.params)
    kw.pop("quasi2d", None)
    return w, kw


def run(args):
    case, eps, seed = args
    sys.path.insert(0, ROOT)
    import oracle as O
    w, kw = workload()
    pos = w.pos + eps * np.random.default_rng(seed).standard_normal(w.pos.shape)
    c = CASES[case]
    o = O.Oracle(w.nx, w.ny, w.nz, w.radius, pos, **kw)
    t0 = time.time()
    o.step(c["steps"], O.shear(kind=0, rate=c["rate"]))
    out = {name: o.stress(k)[0].tolist() for name, k in KINDS.items()}
    _, hist = o.stress(O.CONTACT)
    return {"stress": out, "hist": hist.tolist(), "error": o.error(), "seconds": time.time() - t0}


def main(case: str) -> None:
    c = CASES[case]
    jobs = [(case, 0.0, 0)] + [(case, 1e-9, k) for k in range(1, 1 + c["seeds"])]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(run, jobs)
    ref = res[0]
    assert ref["error"] == 0, "the reference run raised a flag"
    spread = {}
    for name in KINDS:
        a = np.array(ref["stress"][name])
        dev = [np.abs(np.array(r["stress"][name]) - a).max() / np.abs(a).max() for r in res[1:]]
        dxy = [abs(r["stress"][name][0][1] - a[0, 1]) / abs(a[0, 1]) for r in res[1:]]
        spread[name] = {"tensor": max(dev), "xy": max(dxy)}
    w, _ = workload()
    doc = {
        "written_by": "tests/golden/make_long_run.py (FP64 oracle only)",
        "workload": w.name, "box": [w.nx, w.ny, w.nz], "n": int(w.radius.size),
        "rate": c["rate"], "steps": c["steps"],
        "stress": ref["stress"], "hist": ref["hist"],
        "chaos_spread_1e-9": spread,
        "perturbed_runs": c["seeds"],
        "oracle_seconds": ref["seconds"],
    }
    path = os.path.join(HERE, f"long_run_{case}.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    print(path, json.dumps(spread))


def extend(case: str, eps: float, seeds: int) -> None:
    path = os.path.join(HERE, f"long_run_{case}.json")
    with open(path) as f:
        doc = json.load(f)
    c = CASES[case]
    # seeds beyond those of the first perturbed runs
    first = 1 + c["seeds"]
    jobs = [(case, eps, k) for k in range(first, first + seeds)]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(run, jobs)
    spread = {}
    for name in KINDS:
        a = np.array(doc["stress"][name])
        dev = [np.abs(np.array(r["stress"][name]) - a).max() / np.abs(a).max() for r in res]
        dxy = [abs(r["stress"][name][0][1] - a[0, 1]) / abs(a[0, 1]) for r in res]
        spread[name] = {"tensor": max(dev), "xy": max(dxy)}
    doc[f"chaos_spread_{eps:g}"] = spread
    doc[f"perturbed_runs_{eps:g}"] = seeds
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    print(path, json.dumps(spread))


if __name__ == "__main__":
    if len(sys.argv) > 3 and sys.argv[2] == "--extend":
        extend(sys.argv[1], float(sys.argv[3]), int(sys.argv[4]) if len(sys.argv) > 4 else 6)
    else:
        main(sys.argv[1] if len(sys.argv) > 1 else "slow")
