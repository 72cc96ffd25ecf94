"""Python binding of the C ABI in include/susp.h (argument marshalling only).

Every function keeps the C name and signature; the library ``libsusp.so`` is
built in-tree by ``paper_1904_02929_gb300.build``.  There is no fallback: if
the library cannot be loaded, importing the binding raises.

``Suspension`` is a convenience owner of one box: it allocates the device
workspace as a torch uint8 tensor and passes the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SUSP_OK, SUSP_EINVAL, SUSP_ENOMEM, SUSP_ECUDA = 0, -1, -2, -3
SUSP_EOVERLAP, SUSP_EUNSTABLE, SUSP_ETIMEOUT, SUSP_ESTATE = -4, -5, -6, -7
STATUS_NAMES = {0: "SUSP_OK", -1: "SUSP_EINVAL", -2: "SUSP_ENOMEM", -3: "SUSP_ECUDA", -4: "SUSP_EOVERLAP",
                -5: "SUSP_EUNSTABLE", -6: "SUSP_ETIMEOUT", -7: "SUSP_ESTATE"}


def status_name(status: int) -> str:
    """Name of a susp_status value (the number itself if unknown)."""
    return STATUS_NAMES.get(int(status), str(status))
SUSP_FP64, SUSP_FP32, SUSP_FP16_DEV, SUSP_BF16_DEV = 0, 1, 2, 3
PRECISIONS = {"fp64": SUSP_FP64, "fp32": SUSP_FP32, "fp16": SUSP_FP16_DEV, "bf16": SUSP_BF16_DEV}
VISCOUS, CONTACT, REPULSIVE, TOTAL, ANGULAR, LUBRICATION = range(6)


class susp_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double),
        ("n", C.c_int),
        ("radius", C.POINTER(C.c_double)), ("pos", C.POINTER(C.c_double)),
        ("vel", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
        ("rho_p", C.c_double), ("mu", C.c_double), ("kn", C.c_double),
        ("kt_ratio", C.c_double), ("eta_n", C.c_double),
        ("F0", C.c_double), ("debye", C.c_double),
        ("lub_delta", C.c_double), ("lub_cut", C.c_double),
        ("a_map_ratio", C.c_double),
        ("dem_substeps", C.c_int), ("quasi2d", C.c_int),
        ("move_particles", C.c_int), ("nbins", C.c_int),
        ("body_force", C.c_double * 3),
        ("prec", C.c_int),
        ("collision", C.c_int), ("tau_bulk", C.c_double),
        ("driven", C.POINTER(C.c_int)),
    ]


class susp_info(C.Structure):
    _fields_ = [("dem_substeps", C.c_int), ("launches_per_step", C.c_int),
                ("brute_force_pairs", C.c_int), ("ncell", C.c_longlong),
                ("workspace_bytes", C.c_size_t), ("overlap", C.c_int)]


class susp_shear(C.Structure):
    _fields_ = [("kind", C.c_int), ("rate", C.c_double), ("gamma0", C.c_double),
                ("omega", C.c_double), ("theta", C.c_double)]


_D = C.POINTER(C.c_double)
_lib = None


def library() -> C.CDLL:
    """Load libsusp.so (building it first if needed); raises if unavailable."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            path = _build.build()
        L = C.CDLL(path)
        L.susp_workspace_bytes.restype = C.c_size_t
        L.susp_workspace_bytes.argtypes = [C.POINTER(susp_params)]
        L.susp_create.restype = C.c_int
        L.susp_create.argtypes = [C.POINTER(susp_params), C.c_void_p, C.c_size_t, C.c_void_p,
                                  C.POINTER(C.c_void_p)]
        L.susp_step.restype = C.c_int
        L.susp_step.argtypes = [C.c_void_p, C.c_int, C.POINTER(susp_shear)]
        L.susp_stress.restype = C.c_int
        L.susp_stress.argtypes = [C.c_void_p, C.c_int, _D, _D, C.c_int]
        L.susp_stress_reset.restype = C.c_int
        L.susp_stress_reset.argtypes = [C.c_void_p]
        L.susp_get_particles.restype = C.c_int
        L.susp_get_particles.argtypes = [C.c_void_p, _D, _D, _D]
        L.susp_get_hydro.restype = C.c_int
        L.susp_get_hydro.argtypes = [C.c_void_p, _D, _D]
        L.susp_get_populations.restype = C.c_int
        L.susp_get_populations.argtypes = [C.c_void_p, _D]
        L.susp_set_populations.restype = C.c_int
        L.susp_set_populations.argtypes = [C.c_void_p, _D]
        L.susp_get_owner.restype = C.c_int
        L.susp_get_owner.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
        L.susp_get_time.restype = C.c_int
        L.susp_get_time.argtypes = [C.c_void_p, C.POINTER(C.c_int64), _D]
        L.susp_get_info.restype = C.c_int
        L.susp_get_info.argtypes = [C.c_void_p, C.POINTER(susp_info)]
        L.susp_profile.restype = C.c_int
        L.susp_profile.argtypes = [C.c_void_p, C.c_int]
        L.susp_profile_read.restype = C.c_int
        L.susp_profile_read.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int)]
        L.susp_save.restype = C.c_int
        L.susp_save.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]
        L.susp_load.restype = C.c_int
        L.susp_load.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.susp_profile_stages.restype = C.c_int
        L.susp_profile_stages.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int)]
        L.susp_batch_profile_stages.restype = C.c_int
        L.susp_batch_profile_stages.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int)]
        L.susp_fluid_step_noalloc.restype = C.c_int
        L.susp_fluid_step_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                              C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p]
        L.susp_set_graphs.restype = C.c_int
        L.susp_set_graphs.argtypes = [C.c_void_p, C.c_int]
        L.susp_moduli.restype = C.c_int
        L.susp_moduli.argtypes = [C.c_void_p, _D, _D]
        for name in ("susp_tune", "susp_batch_tune"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), _D]
        for name in ("susp_set_launch_shape", "susp_batch_set_launch_shape"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
        L.susp_results_bytes.restype = C.c_size_t
        L.susp_results_bytes.argtypes = [C.c_void_p]
        L.susp_read_results.restype = C.c_int
        L.susp_read_results.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        L.susp_results_particles.restype = C.c_int
        L.susp_results_particles.argtypes = [C.c_void_p, C.c_void_p, _D, _D, _D]
        L.susp_results_stress.restype = C.c_int
        L.susp_results_stress.argtypes = [C.c_void_p, C.c_void_p, C.c_int, _D, _D, C.c_int]
        for name in ("susp_set_overlap", "susp_batch_set_overlap"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_void_p, C.c_int]
        L.susp_batch_get_overlap.restype = C.c_int
        L.susp_batch_get_overlap.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        for name in ("susp_get_launch_shape", "susp_batch_get_launch_shape"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.susp_destroy.restype = None
        L.susp_destroy.argtypes = [C.c_void_p]
        L.susp_batch_workspace_bytes.restype = C.c_size_t
        L.susp_batch_workspace_bytes.argtypes = [C.c_int]
        L.susp_batch_create.restype = C.c_int
        L.susp_batch_create.argtypes = [C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                        C.POINTER(C.c_void_p)]
        L.susp_batch_attach.restype = C.c_int
        L.susp_batch_attach.argtypes = [C.c_void_p, C.c_void_p]
        L.susp_batch_detach.restype = C.c_int
        L.susp_batch_detach.argtypes = [C.c_void_p, C.c_void_p]
        L.susp_batch_size.restype = C.c_int
        L.susp_batch_size.argtypes = [C.c_void_p]
        L.susp_batch_step.restype = C.c_int
        L.susp_batch_step.argtypes = [C.c_void_p, C.c_int]
        L.susp_batch_profile.restype = C.c_int
        L.susp_batch_profile.argtypes = [C.c_void_p, C.c_int]
        L.susp_batch_profile_read.restype = C.c_int
        L.susp_batch_profile_read.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int)]
        L.susp_batch_errors.restype = C.c_int
        L.susp_batch_errors.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.c_int]
        L.susp_batch_destroy.restype = None
        L.susp_batch_destroy.argtypes = [C.c_void_p]
        L.susp_last_error.restype = C.c_char_p
        L.susp_last_error.argtypes = []
        _lib = L
    return _lib


class SuspError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = library().susp_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def _check(st: int, where: str) -> None:
    if st != SUSP_OK:
        raise SuspError(st, where)


# ---- thin wrappers with the C names -------------------------------------
def susp_workspace_bytes(p: susp_params) -> int:
    return int(library().susp_workspace_bytes(C.byref(p)))


def susp_create(p: susp_params, dev_workspace: int, nbytes: int, stream: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(library().susp_create(C.byref(p), C.c_void_p(dev_workspace), nbytes,
                                 C.c_void_p(stream), C.byref(h)), "susp_create")
    return h


def susp_step(h, nsteps: int, sh: susp_shear) -> None:
    _check(library().susp_step(h, int(nsteps), C.byref(sh)), "susp_step")


def susp_stress(h, kind: int, nbins: int):
    out = np.zeros(9)
    hist = np.zeros(3 * nbins)
    _check(library().susp_stress(h, int(kind), out.ctypes.data_as(_D), hist.ctypes.data_as(_D),
                                 int(nbins)), "susp_stress")
    return out.reshape(3, 3), hist.reshape(nbins, 3)


def susp_stress_reset(h) -> None:
    _check(library().susp_stress_reset(h), "susp_stress_reset")


def susp_get_particles(h, n: int):
    R, U, W = np.zeros(3 * max(n, 1)), np.zeros(3 * max(n, 1)), np.zeros(3 * max(n, 1))
    _check(library().susp_get_particles(h, R.ctypes.data_as(_D), U.ctypes.data_as(_D),
                                        W.ctypes.data_as(_D)), "susp_get_particles")
    return R[:3 * n].reshape(n, 3), U[:3 * n].reshape(n, 3), W[:3 * n].reshape(n, 3)


def susp_results_bytes(h) -> int:
    return int(library().susp_results_bytes(h))


def susp_read_results(h, buf_ptr: int, nbytes: int, asynchronous: bool) -> None:
    """Gather the step's results and copy them to the host buffer at buf_ptr
    (pinned memory when asynchronous)."""
    _check(library().susp_read_results(h, C.c_void_p(buf_ptr), int(nbytes), int(bool(asynchronous))),
           "susp_read_results")


def susp_results_particles(h, buf_ptr: int, n: int):
    R, U, W = np.zeros(3 * max(n, 1)), np.zeros(3 * max(n, 1)), np.zeros(3 * max(n, 1))
    _check(library().susp_results_particles(h, C.c_void_p(buf_ptr), R.ctypes.data_as(_D), U.ctypes.data_as(_D),
                                            W.ctypes.data_as(_D)), "susp_results_particles")
    return R[:3 * n].reshape(n, 3), U[:3 * n].reshape(n, 3), W[:3 * n].reshape(n, 3)


def susp_results_stress(h, buf_ptr: int, kind: int, nbins: int):
    out = np.zeros(9)
    hist = np.zeros(3 * nbins)
    _check(library().susp_results_stress(h, C.c_void_p(buf_ptr), int(kind), out.ctypes.data_as(_D),
                                         hist.ctypes.data_as(_D), int(nbins)), "susp_results_stress")
    return out.reshape(3, 3), hist.reshape(nbins, 3)


def susp_get_hydro(h, n: int):
    F, T = np.zeros(3 * max(n, 1)), np.zeros(3 * max(n, 1))
    _check(library().susp_get_hydro(h, F.ctypes.data_as(_D), T.ctypes.data_as(_D)), "susp_get_hydro")
    return F[:3 * n].reshape(n, 3), T[:3 * n].reshape(n, 3)


def susp_get_populations(h, shape):
    nx, ny, nz = shape
    f = np.empty(19 * nx * ny * nz)
    _check(library().susp_get_populations(h, f.ctypes.data_as(_D)), "susp_get_populations")
    return f.reshape(19, nz, ny, nx)


def susp_set_populations(h, f) -> None:
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    _check(library().susp_set_populations(h, f.ctypes.data_as(_D)), "susp_set_populations")


def susp_get_owner(h, shape):
    nx, ny, nz = shape
    o = np.empty(nx * ny * nz, dtype=np.int32)
    _check(library().susp_get_owner(h, o.ctypes.data_as(C.POINTER(C.c_int32))), "susp_get_owner")
    return o.reshape(nz, ny, nx)


def susp_get_time(h):
    t = C.c_int64(0)
    d = C.c_double(0.0)
    _check(library().susp_get_time(h, C.byref(t), C.byref(d)), "susp_get_time")
    return int(t.value), float(d.value)


def susp_get_info(h) -> susp_info:
    info = susp_info()
    _check(library().susp_get_info(h, C.byref(info)), "susp_get_info")
    return info


def susp_profile(h, enable: bool) -> None:
    _check(library().susp_profile(h, int(bool(enable))), "susp_profile")


def susp_profile_read(h):
    ms = C.c_double(0.0)
    n = C.c_int(0)
    _check(library().susp_profile_read(h, C.byref(ms), C.byref(n)), "susp_profile_read")
    return float(ms.value), int(n.value)


def susp_save(h) -> np.ndarray:
    n = C.c_size_t(0)
    _check(library().susp_save(h, None, C.byref(n)), "susp_save")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(library().susp_save(h, C.c_void_p(buf.ctypes.data), C.byref(n)), "susp_save")
    return buf


def susp_load(h, buf) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(library().susp_load(h, C.c_void_p(buf.ctypes.data), buf.size), "susp_load")


STAGES = ("collide_stream", "particles", "finalize", "node_map", "links")


def susp_profile_stages(h):
    ms = np.zeros(len(STAGES))
    n = C.c_int(0)
    _check(library().susp_profile_stages(h, ms.ctypes.data_as(_D), C.byref(n)), "susp_profile_stages")
    return dict(zip(STAGES, ms.tolist())), int(n.value)


def susp_batch_profile_stages(b):
    ms = np.zeros(len(STAGES))
    n = C.c_int(0)
    _check(library().susp_batch_profile_stages(b, ms.ctypes.data_as(_D), C.byref(n)),
           "susp_batch_profile_stages")
    return dict(zip(STAGES, ms.tolist())), int(n.value)


def susp_fluid_step_noalloc(nx, ny, nz, tau, delta, u_le, f_in_ptr, f_out_ptr, visc_out_ptr,
                            stream) -> None:
    """Allocation-free particle-free FP32 step; all pointers are device addresses."""
    _check(library().susp_fluid_step_noalloc(int(nx), int(ny), int(nz), float(tau), float(delta),
                                             float(u_le), C.c_void_p(f_in_ptr), C.c_void_p(f_out_ptr),
                                             C.c_void_p(visc_out_ptr), C.c_void_p(stream)),
           "susp_fluid_step_noalloc")


def susp_set_graphs(h, enable: bool) -> None:
    _check(library().susp_set_graphs(h, int(bool(enable))), "susp_set_graphs")


def susp_moduli(h):
    """(G', G'') of Eq. 17, 18 over the steps since the last stress reset."""
    gp, gpp = C.c_double(0.0), C.c_double(0.0)
    _check(library().susp_moduli(h, C.byref(gp), C.byref(gpp)), "susp_moduli")
    return float(gp.value), float(gpp.value)


def _get_shape(fn, handle, where) -> dict:
    rows, bps, staged = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(fn(handle, C.byref(rows), C.byref(bps), C.byref(staged)), where)
    return {"tile_rows": int(rows.value), "blocks_per_sm": int(bps.value), "staged": bool(staged.value)}


def _tune(fn, get, handle, where):
    rows, bps, us = C.c_int(0), C.c_int(0), C.c_double(0.0)
    _check(fn(handle, C.byref(rows), C.byref(bps), C.byref(us)), where)
    out = _get_shape(get, handle, where)
    out["us"] = float(us.value)
    return out


def susp_tune(h) -> dict:
    """Collide-stream launch shape chosen by timing (tile rows, blocks per SM,
    staged, us) and whether the step overlaps it with the particle kernel."""
    out = _tune(library().susp_tune, library().susp_get_launch_shape, h, "susp_tune")
    out["overlap"] = susp_get_overlap(h)
    return out


def susp_batch_tune(b) -> dict:
    out = _tune(library().susp_batch_tune, library().susp_batch_get_launch_shape, b, "susp_batch_tune")
    out["overlap"] = susp_batch_get_overlap(b)
    return out


def susp_set_overlap(h, enable: bool) -> None:
    _check(library().susp_set_overlap(h, int(bool(enable))), "susp_set_overlap")


def susp_get_overlap(h) -> bool:
    return bool(susp_get_info(h).overlap)


def susp_batch_set_overlap(b, enable: bool) -> None:
    _check(library().susp_batch_set_overlap(b, int(bool(enable))), "susp_batch_set_overlap")


def susp_batch_get_overlap(b) -> bool:
    v = C.c_int(0)
    _check(library().susp_batch_get_overlap(b, C.byref(v)), "susp_batch_get_overlap")
    return bool(v.value)


def susp_set_launch_shape(h, tile_rows: int, blocks_per_sm: int, staged: bool) -> None:
    _check(library().susp_set_launch_shape(h, int(tile_rows), int(blocks_per_sm), int(bool(staged))),
           "susp_set_launch_shape")


def susp_get_launch_shape(h) -> dict:
    return _get_shape(library().susp_get_launch_shape, h, "susp_get_launch_shape")


def susp_batch_set_launch_shape(b, tile_rows: int, blocks_per_sm: int, staged: bool) -> None:
    _check(library().susp_batch_set_launch_shape(b, int(tile_rows), int(blocks_per_sm), int(bool(staged))),
           "susp_batch_set_launch_shape")


def susp_batch_get_launch_shape(b) -> dict:
    return _get_shape(library().susp_batch_get_launch_shape, b, "susp_batch_get_launch_shape")


def susp_destroy(h) -> None:
    library().susp_destroy(h)


def susp_batch_workspace_bytes(max_boxes: int) -> int:
    return int(library().susp_batch_workspace_bytes(int(max_boxes)))


def susp_batch_create(max_boxes: int, dev_workspace: int, nbytes: int, stream: int) -> C.c_void_p:
    b = C.c_void_p()
    _check(library().susp_batch_create(int(max_boxes), C.c_void_p(dev_workspace), nbytes,
                                       C.c_void_p(stream), C.byref(b)), "susp_batch_create")
    return b


def susp_batch_attach(b, h) -> None:
    _check(library().susp_batch_attach(b, h), "susp_batch_attach")


def susp_batch_detach(b, h) -> None:
    _check(library().susp_batch_detach(b, h), "susp_batch_detach")


def susp_batch_size(b) -> int:
    return int(library().susp_batch_size(b))


def susp_batch_step(b, nsteps: int) -> None:
    _check(library().susp_batch_step(b, int(nsteps)), "susp_batch_step")


def susp_batch_profile(b, enable: bool) -> None:
    _check(library().susp_batch_profile(b, int(bool(enable))), "susp_batch_profile")


def susp_batch_profile_read(b):
    ms = C.c_double(0.0)
    n = C.c_int(0)
    _check(library().susp_batch_profile_read(b, C.byref(ms), C.byref(n)), "susp_batch_profile_read")
    return float(ms.value), int(n.value)


def susp_batch_errors(b, n: int):
    out = (C.c_int * max(n, 1))()
    _check(library().susp_batch_errors(b, out, int(max(n, 1))), "susp_batch_errors")
    return [int(out[k]) for k in range(n)]


def susp_batch_destroy(b) -> None:
    library().susp_batch_destroy(b)


def susp_last_error() -> str:
    return library().susp_last_error().decode(errors="replace")


# ---- parameter marshalling ------------------------------------------------
def make_params(nx, ny, nz, radius=(), pos=(), vel=None, omega=None, tau=1.0, rho0=1.0,
                rho_p=1.0, mu=1.0, kn=100.0, kt_ratio=0.2, eta_n=-1.0, F0=0.0, debye=0.08,
                lub_delta=0.04, lub_cut=0.5, a_map_ratio=0.95, dem_substeps=0, quasi2d=False,
                move_particles=True, nbins=36, body_force=(0.0, 0.0, 0.0), precision="fp32",
                collision="bgk", tau_bulk=0.0, driven=None):
    """Fill a susp_params; returns (params, keepalive) — keep the second alive."""
    radius = np.ascontiguousarray(np.asarray(radius, dtype=np.float64).ravel())
    n = radius.size
    keep = [radius]
    p = susp_params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.tau, p.rho0, p.n = float(tau), float(rho0), n
    if n:
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(n, 3).ravel())
        keep.append(pos)
        p.radius, p.pos = radius.ctypes.data_as(_D), pos.ctypes.data_as(_D)
        if vel is not None:
            v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64).reshape(n, 3).ravel())
            keep.append(v)
            p.vel = v.ctypes.data_as(_D)
        if omega is not None:
            w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(n, 3).ravel())
            keep.append(w)
            p.omega = w.ctypes.data_as(_D)
    p.rho_p, p.mu, p.kn, p.kt_ratio, p.eta_n = rho_p, mu, kn, kt_ratio, eta_n
    p.F0, p.debye, p.lub_delta, p.lub_cut, p.a_map_ratio = F0, debye, lub_delta, lub_cut, a_map_ratio
    p.dem_substeps, p.quasi2d = int(dem_substeps), int(bool(quasi2d))
    p.move_particles, p.nbins = int(bool(move_particles)), int(nbins)
    p.body_force = (C.c_double * 3)(*[float(g) for g in body_force])
    p.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.collision = {"bgk": 0, "ladd": 1}[collision] if isinstance(collision, str) else int(collision)
    p.tau_bulk = float(tau_bulk)
    if driven is not None and n:
        dv = np.ascontiguousarray(np.asarray(driven, dtype=np.int32).ravel())
        if dv.size != n:
            raise ValueError("driven needs one flag per particle")
        keep.append(dv)
        p.driven = dv.ctypes.data_as(C.POINTER(C.c_int))
    return p, keep


def make_shear(kind=0, rate=0.0, gamma0=0.0, omega=0.0, theta=0.0) -> susp_shear:
    return susp_shear(int(kind), float(rate), float(gamma0), float(omega), float(theta))


class Suspension:
    """One box on the current CUDA device; workspace held as a torch tensor.

    All work goes to ``self.stream`` (a new torch stream unless one is given);
    the calls that return host data synchronise it."""

    def __init__(self, nx, ny, nz, radius=(), pos=(), stream=None, **kw):
        import torch
        self.p, keep = make_params(nx, ny, nz, radius, pos, **kw)
        self.shape = (int(nx), int(ny), int(nz))
        self.n = int(self.p.n)
        self.nbins = int(self.p.nbins) if self.p.nbins > 0 else 36
        self.precision = int(self.p.prec)
        self.nbytes = susp_workspace_bytes(self.p)
        if self.nbytes == 0:
            raise SuspError(SUSP_EINVAL, "susp_workspace_bytes")
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        self.ptr = (base + 255) & ~255
        # a stream of its own: the legacy default stream cannot be graph-captured
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.h = susp_create(self.p, self.ptr, self.nbytes, self.stream.cuda_stream)
        del keep

    def step(self, nsteps, shear=None):
        susp_step(self.h, nsteps, shear if shear is not None else make_shear())

    def stress(self, kind=TOTAL):
        return susp_stress(self.h, kind, self.nbins)

    def stress_reset(self):
        susp_stress_reset(self.h)

    def particles(self):
        return susp_get_particles(self.h, self.n)

    def hydro(self):
        return susp_get_hydro(self.h, self.n)

    def populations(self):
        return susp_get_populations(self.h, self.shape)

    def set_populations(self, f):
        susp_set_populations(self.h, f)

    def owner(self):
        return susp_get_owner(self.h, self.shape)

    def time(self):
        return susp_get_time(self.h)

    def info(self):
        return susp_get_info(self.h)

    def save(self) -> np.ndarray:
        return susp_save(self.h)

    def load(self, buf):
        susp_load(self.h, buf)

    def set_graphs(self, enable: bool):
        susp_set_graphs(self.h, enable)

    def tune(self) -> dict:
        return susp_tune(self.h)

    def set_launch_shape(self, tile_rows: int, blocks_per_sm: int, staged: bool) -> None:
        susp_set_launch_shape(self.h, tile_rows, blocks_per_sm, staged)

    def launch_shape(self) -> dict:
        return dict(susp_get_launch_shape(self.h), overlap=susp_get_overlap(self.h))

    def set_overlap(self, enable: bool) -> None:
        susp_set_overlap(self.h, enable)

    def results_buffer(self):
        """A pinned host buffer for read_results."""
        import torch
        return torch.empty(susp_results_bytes(self.h), dtype=torch.uint8).pin_memory()

    def read_results(self, buf, asynchronous: bool = False) -> None:
        """Copy the step's results into buf (a results_buffer) with one transfer;
        asynchronous: only enqueue it on self.stream."""
        susp_read_results(self.h, buf.data_ptr(), buf.numel(), asynchronous)

    def results_particles(self, buf):
        return susp_results_particles(self.h, buf.data_ptr(), self.n)

    def results_stress(self, buf, kind=TOTAL):
        return susp_results_stress(self.h, buf.data_ptr(), kind, self.nbins)

    def moduli(self):
        return susp_moduli(self.h)

    def close(self):
        if getattr(self, "h", None):
            susp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Boxes stepped in lockstep by one launch sequence (include/susp.h,
    "batches").  Holds the descriptor workspace and a stream of its own; keeps
    its members alive while they are attached."""

    def __init__(self, max_boxes, stream=None):
        import torch
        self.max_boxes = int(max_boxes)
        self.nbytes = susp_batch_workspace_bytes(self.max_boxes)
        if self.nbytes == 0:
            raise SuspError(SUSP_EINVAL, "susp_batch_workspace_bytes")
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        self.ptr = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.b = susp_batch_create(self.max_boxes, self.ptr, self.nbytes, self.stream.cuda_stream)
        self.members = []

    def attach(self, box: Suspension, shear=None):
        """Attach a box; ``shear`` (if given) is set as its protocol first."""
        if shear is not None:
            box.step(0, shear)
        susp_batch_attach(self.b, box.h)
        self.members.append(box)

    def detach(self, box: Suspension):
        susp_batch_detach(self.b, box.h)
        self.members.remove(box)

    def __len__(self):
        return susp_batch_size(self.b)

    def step(self, nsteps=1):
        susp_batch_step(self.b, nsteps)

    def errors(self):
        """Device status of each member, in ``self.members`` order."""
        return susp_batch_errors(self.b, len(self.members))

    def tune(self) -> dict:
        return susp_batch_tune(self.b)

    def set_launch_shape(self, tile_rows: int, blocks_per_sm: int, staged: bool) -> None:
        susp_batch_set_launch_shape(self.b, tile_rows, blocks_per_sm, staged)

    def launch_shape(self) -> dict:
        return dict(susp_batch_get_launch_shape(self.b), overlap=susp_batch_get_overlap(self.b))

    def set_overlap(self, enable: bool) -> None:
        susp_batch_set_overlap(self.b, enable)

    def profile(self, enable: bool):
        susp_batch_profile(self.b, enable)

    def profile_read(self):
        return susp_batch_profile_read(self.b)

    def close(self):
        if getattr(self, "b", None):
            susp_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
