"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/susp.h; host-side parameter validation works without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1904_02929_gb300 import build as B
from paper_1904_02929_gb300 import susp as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(susp_\w+)\s*\(", src))
    return names


def test_library_builds_and_exports_all_declared_symbols():
    lib = C.CDLL(B.build())
    syms = declared_symbols()
    assert {"susp_create", "susp_step", "susp_stress"} <= syms
    for name in sorted(syms):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_params_struct_layout_matches_header():
    # the binding mirrors the C struct field by field
    src = open(os.path.join(ROOT, "include", "susp.h")).read()
    body = src[src.index("typedef struct {\n  int nx, ny, nz;"):src.index("} susp_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
            if not decl:
                continue
        toks = decl.replace("const", "").replace("*", " ").split()
        for name in " ".join(toks[1:]).split(","):
            fields.append(name.strip().split("[")[0])
    assert fields == [f[0] for f in S.susp_params._fields_]


def test_workspace_bytes_and_validation_on_host():
    p, keep = S.make_params(32, 32, 32, [4.5], [[16, 16, 16]], precision="fp32")
    nb = S.susp_workspace_bytes(p)
    # two population copies dominate: 2 * 19 * 32^3 * 4 bytes
    assert nb >= 2 * 19 * 32 ** 3 * 4
    p64, keep64 = S.make_params(32, 32, 32, [4.5], [[16, 16, 16]], precision="fp64")
    assert S.susp_workspace_bytes(p64) > nb
    bad, k2 = S.make_params(3, 32, 32, precision="fp32")
    assert S.susp_workspace_bytes(bad) == 0
    assert "dims" in S.susp_last_error()
    bad, k3 = S.make_params(32, 32, 32, tau=0.5)
    assert S.susp_workspace_bytes(bad) == 0
    bad, k4 = S.make_params(16, 16, 16, [9.0], [[8, 8, 8]])
    assert S.susp_workspace_bytes(bad) == 0 and "too large" in S.susp_last_error()


def test_lattice_limits_and_parameter_checks_on_host():
    # the largest accepted box: just under 2^27 nodes
    ok, k0 = S.make_params(512, 512, 511, precision="fp16")
    assert S.susp_workspace_bytes(ok) >= 2 * 19 * 512 * 512 * 511 * 2
    for dims, msg in [((512, 512, 512), "2^27"), ((2048, 8, 8), "2047"), ((8, 8, 1024), "2047")]:
        bad, kb = S.make_params(*dims, precision="fp16")
        assert S.susp_workspace_bytes(bad) == 0 and msg in S.susp_last_error(), dims
    cases = [dict(collision=2), dict(collision="ladd", tau_bulk=0.5), dict(rho0=0.0)]
    for kw in cases:
        bad, kb = S.make_params(16, 16, 16, **kw)
        assert S.susp_workspace_bytes(bad) == 0, kw
    bad, kb = S.make_params(32, 32, 32, [4.0], [[16.0, float("nan"), 16.0]])
    assert S.susp_workspace_bytes(bad) == 0 and "finite" in S.susp_last_error()
    bad, kb = S.make_params(32, 32, 32, [4.0], [[16, 16, 16]], a_map_ratio=1.5)
    assert S.susp_workspace_bytes(bad) == 0
    # driven flags: one per particle; they add one int32 per particle to the layout
    with pytest.raises(ValueError):
        S.make_params(32, 32, 32, [4.0, 4.0], [[8, 8, 8], [24, 24, 24]], driven=[1])
    d, kd = S.make_params(32, 32, 32, [4.0, 4.0], [[8, 8, 8], [24, 24, 24]], driven=[1, 0])
    assert d.driven and d.driven[0] == 1 and d.driven[1] == 0
    assert S.susp_workspace_bytes(d) > 0


def test_create_rejects_bad_workspace_without_touching_the_device():
    p, keep = S.make_params(16, 16, 16, precision="fp32")
    h = C.c_void_p()
    lib = S.library()
    st = lib.susp_create(C.byref(p), C.c_void_p(0), 0, None, C.byref(h))
    assert st == S.SUSP_EINVAL and not h.value
    st = lib.susp_create(C.byref(p), C.c_void_p(0x1001), 1 << 30, None, C.byref(h))
    assert st == S.SUSP_EINVAL and "aligned" in S.susp_last_error()
    st = lib.susp_create(C.byref(p), C.c_void_p(0x100000), 16, None, C.byref(h))
    assert st == S.SUSP_ENOMEM


def test_step_rejects_bad_arguments_on_host():
    lib = S.library()
    sh = S.make_shear(kind=3)
    assert lib.susp_step(None, 1, C.byref(sh)) == S.SUSP_EINVAL


def test_batch_workspace_bytes_on_host():
    assert S.susp_batch_workspace_bytes(0) == 0
    one, many = S.susp_batch_workspace_bytes(1), S.susp_batch_workspace_bytes(64)
    assert 0 < one < many and many % 256 == 0


def test_serving_requests_and_footprint_on_host():
    from paper_1904_02929_gb300 import inputs as I
    from paper_1904_02929_gb300 import serve as V
    w = I.config_small()
    pool = [I.Workload("s", w.nx, w.ny, w.nz, w.radius, w.pos, dict(w.params))]
    reqs = V.poisson_requests(pool, rate=20.0, duration=50.0, steps=1000, seed=3)
    t = np.array([r.arrival for r in reqs])
    assert (np.diff(t) > 0).all() and t.max() < 50.0
    assert abs(len(reqs) / 50.0 - 20.0) < 3.0            # ~1000 arrivals, sd ~ 32
    gaps = np.diff(t)
    assert abs(gaps.mean() - 0.05) < 0.005 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    kinds = {r.shear["kind"] for r in reqs}
    assert kinds == {0, 1}
    p, keep = S.make_params(w.nx, w.ny, w.nz, w.radius, w.pos, precision="bf16", **w.params)
    assert V.footprint(reqs[0], "bf16") == S.susp_workspace_bytes(p)
