"""Plain FP64 CPU oracle for the sheared-suspension LB + particle step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg and reference arm of ``bench.py`` may import this package
(``__graft_entry__.build()`` compiles it); the product path
(``paper_1904_02929_gb300``) never does.  The C source (``oracle.c``) is
written from arXiv:1904.02929 independently of the CUDA library and shares
no code with it.

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` next to this
file (``-ffp-contract=off`` so that results are the same on x86 and Arm).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

VISCOUS, CONTACT, REPULSIVE, TOTAL, ANGULAR, LUBRICATION = range(6)
EOVERLAP, EUNSTABLE, EHIST = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C11, FP64)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class OrcParams(C.Structure):
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
        ("collision", C.c_int), ("tau_bulk", C.c_double),
        ("driven", C.POINTER(C.c_int)),
    ]


class OrcShear(C.Structure):
    _fields_ = [("kind", C.c_int), ("rate", C.c_double), ("gamma0", C.c_double),
                ("omega", C.c_double), ("theta", C.c_double)]


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_int, C.POINTER(OrcShear)]
        L.orc_error.argtypes = [C.c_void_p]
        L.orc_ncell.restype = C.c_long
        L.orc_ncell.argtypes = [C.c_void_p]
        L.orc_nsub.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_long
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_delta.restype = C.c_double
        L.orc_delta.argtypes = [C.c_void_p]
        for name in ("orc_get_populations", "orc_set_populations"):
            getattr(L, name).argtypes = [C.c_void_p, _D]
        L.orc_get_owner.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        L.orc_get_particles.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_get_hydro.argtypes = [C.c_void_p, _D, _D]
        L.orc_get_pending.argtypes = [C.c_void_p, _D, _D]
        L.orc_stress.restype = C.c_int
        L.orc_stress.argtypes = [C.c_void_p, C.c_int, _D, _D, C.c_int]
        L.orc_stress_reset.argtypes = [C.c_void_p]
        L.orc_moduli.restype = C.c_int
        L.orc_moduli.argtypes = [C.c_void_p, C.c_double, _D, _D]
        L.orc_lattice.argtypes = [C.POINTER(C.c_int), _D, C.POINTER(C.c_int)]
        L.orc_equilibrium.argtypes = [C.c_double, _D, _D]
        L.orc_contact.restype = C.c_int
        L.orc_contact.argtypes = [C.c_double, C.c_double, _D, _D, _D, _D, C.c_double,
                                  C.c_double, C.c_double, C.c_double, C.c_double, _D,
                                  _D, _D, _D, _D, _D]
        L.orc_lubrication.argtypes = [C.c_double, C.c_double, _D, _D, _D, _D, C.c_double,
                                      C.c_double, C.c_double, _D, _D, _D]
        L.orc_lubrication_stresslet.argtypes = [C.c_double, C.c_double, _D, _D, _D, _D, C.c_double,
                                                C.c_double, C.c_double, _D]
        L.orc_gamma.restype = C.c_double
        L.orc_gamma.argtypes = [C.POINTER(OrcShear), C.c_double]
        L.orc_le_increment.restype = C.c_double
        L.orc_le_increment.argtypes = [C.POINTER(OrcShear), C.c_long, C.c_double]
        L.orc_angular_stress.argtypes = [_D, C.c_int, C.c_double, C.c_double, C.c_double,
                                         C.c_int, _D]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D)


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def shear(kind=0, rate=0.0, gamma0=0.0, omega=0.0, theta=0.0) -> OrcShear:
    return OrcShear(int(kind), float(rate), float(gamma0), float(omega), float(theta))


def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    o = np.zeros(19, dtype=np.int32)
    lib().orc_lattice(c.ctypes.data_as(C.POINTER(C.c_int)), _ptr(w),
                      o.ctypes.data_as(C.POINTER(C.c_int)))
    return c, w, o


def equilibrium(rho, j):
    out = np.zeros(19)
    lib().orc_equilibrium(float(rho), _ptr(_vec(j)), _ptr(out))
    return out


def contact(ra, rb, d, uab, wa, wb, kn, kt, eta_n, mu, dt, hist_t):
    """One contact pair; returns (touching, Fa, Ta, Tb, fn, Ftan, new_hist)."""
    ht = _vec(hist_t).copy()
    Fa, Ta, Tb, Ft = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    fn = C.c_double(0.0)
    d, uab, wa, wb = _vec(d), _vec(uab), _vec(wa), _vec(wb)
    t = lib().orc_contact(float(ra), float(rb), _ptr(d), _ptr(uab), _ptr(wa), _ptr(wb),
                          float(kn), float(kt), float(eta_n), float(mu), float(dt),
                          _ptr(ht), _ptr(Fa), _ptr(Ta), _ptr(Tb), C.byref(fn), _ptr(Ft))
    return bool(t), Fa, Ta, Tb, fn.value, Ft, ht


def lubrication(ra, rb, d, uab, wa, wb, eta0, delta, hcut):
    Fa, Ta, Tb = np.zeros(3), np.zeros(3), np.zeros(3)
    d, uab, wa, wb = _vec(d), _vec(uab), _vec(wa), _vec(wb)
    lib().orc_lubrication(float(ra), float(rb), _ptr(d), _ptr(uab), _ptr(wa), _ptr(wb),
                          float(eta0), float(delta), float(hcut), _ptr(Fa), _ptr(Ta), _ptr(Tb))
    return Fa, Ta, Tb


def lubrication_stresslet(ra, rb, d, uab, wa, wb, eta0, delta, hcut):
    """S_a + S_b of one pair (3 x 3)."""
    S = np.zeros(9)
    d, uab, wa, wb = _vec(d), _vec(uab), _vec(wa), _vec(wb)
    lib().orc_lubrication_stresslet(float(ra), float(rb), _ptr(d), _ptr(uab), _ptr(wa), _ptr(wb),
                                    float(eta0), float(delta), float(hcut), _ptr(S))
    return S.reshape(3, 3)


def gamma(sh: OrcShear, t: float) -> float:
    return lib().orc_gamma(C.byref(sh), float(t))


def le_increment(sh: OrcShear, t: int, ly: float) -> float:
    return lib().orc_le_increment(C.byref(sh), int(t), float(ly))


def angular_stress(hist, phi, z_coord, a, two_d):
    h = _vec(hist).ravel()
    out = np.zeros(9)
    lib().orc_angular_stress(_ptr(h), len(h) // 3, float(phi), float(z_coord), float(a),
                             int(bool(two_d)), _ptr(out))
    return out.reshape(3, 3)


class Oracle:
    """One simulation box held by the C oracle."""

    def __init__(self, nx, ny, nz, radius=(), pos=(), vel=None, omega=None, tau=1.0,
                 rho0=1.0, rho_p=1.0, mu=1.0, kn=100.0, kt_ratio=0.2, eta_n=-1.0, F0=0.0,
                 debye=0.08, lub_delta=0.04, lub_cut=0.5, a_map_ratio=0.95,
                 dem_substeps=0, quasi2d=False, move_particles=True, nbins=36,
                 body_force=(0.0, 0.0, 0.0), collision="bgk", tau_bulk=0.0, driven=None):
        self._keep = []
        radius = _vec(radius).ravel()
        n = radius.size
        pos = _vec(pos).reshape(n, 3).ravel() if n else np.zeros(3)
        self.n = n
        p = OrcParams()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.tau, p.rho0 = float(tau), float(rho0)
        p.n = n
        rad = radius if n else np.zeros(1)
        self._keep += [rad, pos]
        p.radius, p.pos = _ptr(rad), _ptr(pos)
        if vel is not None:
            v = _vec(vel).reshape(n, 3).ravel(); self._keep.append(v); p.vel = _ptr(v)
        if omega is not None:
            w = _vec(omega).reshape(n, 3).ravel(); self._keep.append(w); p.omega = _ptr(w)
        p.rho_p, p.mu, p.kn, p.kt_ratio, p.eta_n = rho_p, mu, kn, kt_ratio, eta_n
        p.F0, p.debye, p.lub_delta, p.lub_cut = F0, debye, lub_delta, lub_cut
        p.a_map_ratio, p.dem_substeps = a_map_ratio, int(dem_substeps)
        p.quasi2d, p.move_particles, p.nbins = int(quasi2d), int(move_particles), int(nbins)
        p.body_force = (C.c_double * 3)(*[float(g) for g in body_force])
        p.collision = {"bgk": 0, "ladd": 1}[collision] if isinstance(collision, str) else int(collision)
        p.tau_bulk = float(tau_bulk)
        if driven is not None and n:
            dv = np.ascontiguousarray(np.asarray(driven, dtype=np.int32).ravel())
            assert dv.size == n
            self._keep.append(dv)
            p.driven = dv.ctypes.data_as(C.POINTER(C.c_int))
        self.shape = (int(nx), int(ny), int(nz))
        self.nbins = int(nbins)
        self.h = lib().orc_create(C.byref(p))
        self._keep = []

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ncell(self):
        return int(lib().orc_ncell(self.h))

    @property
    def nsub(self):
        return int(lib().orc_nsub(self.h))

    @property
    def time(self):
        return int(lib().orc_time(self.h))

    @property
    def delta(self):
        return float(lib().orc_delta(self.h))

    def error(self):
        return int(lib().orc_error(self.h))

    def step(self, nsteps, sh: OrcShear | None = None):
        sh = sh if sh is not None else shear()
        return int(lib().orc_step(self.h, int(nsteps), C.byref(sh)))

    def populations(self):
        """Post-collision populations, shape (19, nz, ny, nx)."""
        f = np.empty(19 * self.ncell)
        lib().orc_get_populations(self.h, _ptr(f))
        nx, ny, nz = self.shape
        return f.reshape(19, nz, ny, nx)

    def set_populations(self, f):
        f = _vec(f).ravel()
        assert f.size == 19 * self.ncell
        lib().orc_set_populations(self.h, _ptr(f))

    def owner(self):
        o = np.empty(self.ncell, dtype=np.int32)
        lib().orc_get_owner(self.h, o.ctypes.data_as(C.POINTER(C.c_int)))
        nx, ny, nz = self.shape
        return o.reshape(nz, ny, nx)

    def particles(self):
        n = max(self.n, 1)
        R, U, W = np.zeros(3 * n), np.zeros(3 * n), np.zeros(3 * n)
        lib().orc_get_particles(self.h, _ptr(R), _ptr(U), _ptr(W))
        k = self.n
        return R[:3 * k].reshape(k, 3), U[:3 * k].reshape(k, 3), W[:3 * k].reshape(k, 3)

    def hydro(self):
        n = max(self.n, 1)
        F, T = np.zeros(3 * n), np.zeros(3 * n)
        lib().orc_get_hydro(self.h, _ptr(F), _ptr(T))
        k = self.n
        return F[:3 * k].reshape(k, 3), T[:3 * k].reshape(k, 3)

    def pending(self):
        n = max(self.n, 1)
        F, T = np.zeros(3 * n), np.zeros(3 * n)
        lib().orc_get_pending(self.h, _ptr(F), _ptr(T))
        k = self.n
        return F[:3 * k].reshape(k, 3), T[:3 * k].reshape(k, 3)

    def stress(self, kind=TOTAL):
        out = np.zeros(9)
        hist = np.zeros(3 * self.nbins)
        rc = lib().orc_stress(self.h, int(kind), _ptr(out), _ptr(hist), self.nbins)
        assert rc == 0
        return out.reshape(3, 3), hist.reshape(self.nbins, 3)

    def stress_reset(self):
        lib().orc_stress_reset(self.h)

    def moduli(self, gamma0):
        """(G', G'') of Eq. 17, 18 over the steps since the last reset."""
        gp, gpp = np.zeros(1), np.zeros(1)
        assert lib().orc_moduli(self.h, float(gamma0), _ptr(gp), _ptr(gpp)) == 0
        return float(gp[0]), float(gpp[0])
