"""FP64 CPU oracle for the D3Q27 colour-gradient CM-MRT step (arXiv 2309.07801).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and the two share no code.

The arithmetic lives in ``cg_oracle.c`` (D3Q27) and ``cg_oracle2d.c`` (D2Q9, App. A)
(plain C11 + OpenMP, FP64); this module compiles them with gcc and exposes them
through ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_SRC2 = os.path.join(_HERE, "cg_oracle2d.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODEL_A, MODEL_B, MODEL_C, MODEL_D = 0, 1, 2, 3
BC_PERIODIC, BC_BOUNCEBACK, BC_SLIP, BC_MOVING = 0, 1, 2, 3
FORCE_NONE, FORCE_CONST, FORCE_GRAVITY, FORCE_BUOYANCY = 0, 1, 2, 3
FIELDS = {"grad_phi": (0, 3), "n": (1, 3), "kappa": (2, 1), "F": (3, 3),
          "Q": (4, 3), "omega1": (5, 1), "w": (6, 3), "R": (7, 3)}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    deps = [_SRC, _SRC2, os.path.join(_HERE, "cg_oracle.h"), os.path.join(_HERE, "cg_oracle2d.h")]
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(os.path.getmtime(p) for p in deps)
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, _SRC2, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 3),
                ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
                ("alpha_r", ctypes.c_double), ("alpha_b", ctypes.c_double),
                ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double),
                ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("omega", ctypes.c_double * 11), ("g", ctypes.c_double * 3),
                ("rho_ref", ctypes.c_double),
                ("force_mode", ctypes.c_int32), ("model", ctypes.c_int32),
                ("use_Q", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("wall_u", (ctypes.c_double * 3) * 6)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.ocg_create.restype = ctypes.c_void_p
        L.ocg_create.argtypes = [ctypes.POINTER(Params)]
        L.ocg_destroy.argtypes = [ctypes.c_void_p]
        L.ocg_init.argtypes = [ctypes.c_void_p, dp, dp, dp, ctypes.c_void_p]
        L.ocg_set_populations.argtypes = [ctypes.c_void_p, dp, dp]
        L.ocg_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.ocg_read_macros.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        L.ocg_read_populations.argtypes = [ctypes.c_void_p, dp, dp]
        L.ocg_read_field.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.ocg_mass.argtypes = [ctypes.c_void_p, dp]
        L.ocg_cells.restype = ctypes.c_int64
        L.ocg_cells.argtypes = [ctypes.c_void_p]
        L.ocg_hermite.restype = ctypes.c_double
        L.ocg_hermite.argtypes = [ctypes.c_int] * 4
        L.ocg_lattice.argtypes = [ctypes.c_void_p, dp]
        L.ocg_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.ocg_raw_moments.argtypes = [dp, dp]
        L.ocg_central_moments.argtypes = [dp, dp, dp]
        L.ocg_moment_matrix.argtypes = [dp]
        L.ocg_moment_matrix_inverse.argtypes = [dp]
        L.ocg_collide_cm.argtypes = [dp, dp, dp, dp, dp, dp]
        L.ocg_cm_to_f.argtypes = [dp, dp, dp]
        L.ocg_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- single-cell routines ---------------------------------------------------

def lattice():
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().ocg_lattice(c.ctypes.data_as(ctypes.c_void_p), _p(w))
    return c, w


def hermite(i: int, a: int, b: int, c: int) -> float:
    return lib().ocg_hermite(i, a, b, c)


def feq(model: int, rho: float, p: float, u) -> np.ndarray:
    out = np.zeros(27)
    uu = _d(u)
    lib().ocg_feq(model, rho, p, _p(uu), _p(out))
    return out


def raw_moments(f) -> np.ndarray:
    f = _d(f); m = np.zeros(27)
    lib().ocg_raw_moments(_p(f), _p(m))
    return m


def central_moments(f, u) -> np.ndarray:
    f = _d(f); u = _d(u); k = np.zeros(27)
    lib().ocg_central_moments(_p(f), _p(u), _p(k))
    return k


def moment_matrix() -> np.ndarray:
    M = np.zeros(27 * 27)
    lib().ocg_moment_matrix(_p(M))
    return M.reshape(27, 27)


def moment_matrix_inverse() -> np.ndarray:
    M = np.zeros(27 * 27)
    lib().ocg_moment_matrix_inverse(_p(M))
    return M.reshape(27, 27)


def collide_cm(k, keq, omega, F, Q) -> np.ndarray:
    k = _d(k); keq = _d(keq); om = _d(omega); F = _d(F); Q = _d(Q)
    ks = np.zeros(27)
    lib().ocg_collide_cm(_p(k), _p(keq), _p(om), _p(F), _p(Q), _p(ks))
    return ks


def cm_to_f(k, u) -> np.ndarray:
    k = _d(k); u = _d(u); f = np.zeros(27)
    lib().ocg_cm_to_f(_p(k), _p(u), _p(f))
    return f


def moment_index(a: int, b: int, c: int) -> int:
    """Index of the moment of orders (a, b, c) in the oracle's moment vectors."""
    return a + 3 * b + 9 * c


def threads() -> int:
    return lib().ocg_threads()


# ---- whole domain -------------------------------------------------------------

def make_params(nx, ny, nz, *, bc=(0, 0, 0), rho_r0=1.0, rho_b0=1.0,
                alpha_r=8.0 / 27.0, alpha_b=8.0 / 27.0, nu_r=0.1, nu_b=0.1,
                sigma=0.01, beta=0.7, omega=None, g=(0.0, 0.0, 0.0), rho_ref=0.0,
                force_mode=FORCE_NONE, model=MODEL_D, use_Q=1, wall_u=None) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = nx, ny, nz
    for a in range(3):
        P.bc[a] = int(bc[a])
        P.g[a] = float(g[a])
    P.rho_r0, P.rho_b0 = rho_r0, rho_b0
    P.alpha_r, P.alpha_b = alpha_r, alpha_b
    P.nu_r, P.nu_b = nu_r, nu_b
    P.sigma, P.beta = sigma, beta
    om = [1.0] * 11 if omega is None else list(omega)
    for q in range(11):
        P.omega[q] = float(om[q])
    P.rho_ref = rho_ref
    P.force_mode, P.model, P.use_Q = force_mode, model, use_Q
    if wall_u is not None:
        for f in range(6):
            for b in range(3):
                P.wall_u[f][b] = float(wall_u[f][b])
    return P


class Domain:
    """Whole-domain FP64 reference run (paper layout: two colours x 27)."""

    def __init__(self, params: Params):
        self.params = params
        self._h = lib().ocg_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle: invalid domain size")
        self.shape = (params.nz, params.ny, params.nx)
        self.N = int(params.nx) * params.ny * params.nz

    def close(self):
        if self._h:
            lib().ocg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho_r, rho_b, u, solid: Optional[np.ndarray] = None):
        rr = _d(rho_r).reshape(-1); rb = _d(rho_b).reshape(-1); uu = _d(u).reshape(-1)
        sp = None
        if solid is not None:
            s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
            self._solid_keep = s
            sp = s.ctypes.data_as(ctypes.c_void_p)
        lib().ocg_init(self._h, _p(rr), _p(rb), _p(uu), sp)

    def set_populations(self, fr, fb):
        fr = _d(fr).reshape(-1); fb = _d(fb).reshape(-1)
        lib().ocg_set_populations(self._h, _p(fr), _p(fb))

    def step(self, n: int = 1):
        lib().ocg_step(self._h, int(n))

    def macros(self) -> dict:
        N = self.N
        rr, rb, p, phi = (np.zeros(N) for _ in range(4))
        u = np.zeros(3 * N)
        lib().ocg_read_macros(self._h, _p(rr), _p(rb), _p(u), _p(p), _p(phi))
        sh = self.shape
        return {"rho_r": rr.reshape(sh), "rho_b": rb.reshape(sh),
                "u": u.reshape((3,) + sh), "p": p.reshape(sh), "phi": phi.reshape(sh)}

    def populations(self):
        fr = np.zeros(27 * self.N); fb = np.zeros(27 * self.N)
        lib().ocg_read_populations(self._h, _p(fr), _p(fb))
        sh = (27,) + self.shape
        return fr.reshape(sh), fb.reshape(sh)

    def field(self, name: str) -> np.ndarray:
        which, ncomp = FIELDS[name]
        out = np.zeros(ncomp * self.N)
        lib().ocg_read_field(self._h, which, _p(out))
        return out.reshape(((ncomp,) if ncomp > 1 else ()) + self.shape)

    def mass(self) -> np.ndarray:
        out = np.zeros(2)
        lib().ocg_mass(self._h, _p(out))
        return out


# ---- D2Q9 (App. A) ---------------------------------------------------------------

class Params2D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc", ctypes.c_int32 * 2),
                ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
                ("alpha_r", ctypes.c_double), ("alpha_b", ctypes.c_double),
                ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double),
                ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("omega", ctypes.c_double * 5), ("g", ctypes.c_double * 2),
                ("rho_ref", ctypes.c_double), ("force_mode", ctypes.c_int32), ("use_Q", ctypes.c_int32)]


_lib2 = None


def lib2() -> ctypes.CDLL:
    global _lib2
    if _lib2 is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.o2_create.restype = ctypes.c_void_p
        L.o2_create.argtypes = [ctypes.POINTER(Params2D)]
        L.o2_destroy.argtypes = [ctypes.c_void_p]
        L.o2_init.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.o2_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.o2_read_macros.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        L.o2_read_populations.argtypes = [ctypes.c_void_p, dp, dp]
        L.o2_mass.argtypes = [ctypes.c_void_p, dp]
        L.o2_lattice.argtypes = [ctypes.c_void_p, dp]
        L.o2_hermite.restype = ctypes.c_double
        L.o2_hermite.argtypes = [ctypes.c_int] * 3
        L.o2_feq.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
        L.o2_central_moments.argtypes = [dp, dp, dp]
        L.o2_moment_matrix.argtypes = [dp]
        L.o2_moment_matrix_inverse.argtypes = [dp]
        L.o2_cm_to_f.argtypes = [dp, dp, dp]
        L.o2_collide_cm.argtypes = [dp, dp, dp, dp, dp, dp]
        _lib2 = L
    return _lib2


def lattice2d():
    c = np.zeros((9, 2), dtype=np.int32)
    w = np.zeros(9)
    lib2().o2_lattice(c.ctypes.data_as(ctypes.c_void_p), _p(w))
    return c, w


def hermite2d(i, a, b) -> float:
    return lib2().o2_hermite(i, a, b)


def feq2d(rho, p, u):
    f = np.zeros(9)
    lib2().o2_feq(rho, p, _p(_d(u)), _p(f))
    return f


def central_moments2d(f, u):
    k = np.zeros(9)
    lib2().o2_central_moments(_p(_d(f)), _p(_d(u)), _p(k))
    return k


def moment_matrix2d():
    M = np.zeros(81)
    lib2().o2_moment_matrix(_p(M))
    return M.reshape(9, 9)


def moment_matrix_inverse2d():
    M = np.zeros(81)
    lib2().o2_moment_matrix_inverse(_p(M))
    return M.reshape(9, 9)


def cm_to_f2d(k, u):
    f = np.zeros(9)
    lib2().o2_cm_to_f(_p(_d(k)), _p(_d(u)), _p(f))
    return f


def collide_cm2d(k, keq, om, F, Q):
    ks = np.zeros(9)
    lib2().o2_collide_cm(_p(_d(k)), _p(_d(keq)), _p(_d(om)), _p(_d(F)), _p(_d(Q)), _p(ks))
    return ks


def make_params2d(nx, ny, *, bc=(0, 0), rho_r0=1.0, rho_b0=1.0, alpha_r=4.0 / 9.0, alpha_b=4.0 / 9.0,
                  nu_r=1.0 / 6.0, nu_b=1.0 / 6.0, sigma=0.01, beta=0.7, omega=None, g=(0.0, 0.0),
                  rho_ref=0.0, force_mode=FORCE_NONE, use_Q=1) -> Params2D:
    P = Params2D()
    P.nx, P.ny = nx, ny
    for a in range(2):
        P.bc[a] = int(bc[a])
        P.g[a] = float(g[a])
    P.rho_r0, P.rho_b0, P.alpha_r, P.alpha_b = rho_r0, rho_b0, alpha_r, alpha_b
    P.nu_r, P.nu_b, P.sigma, P.beta = nu_r, nu_b, sigma, beta
    om = [1.0] * 5 if omega is None else list(omega)
    for q in range(5):
        P.omega[q] = float(om[q])
    P.rho_ref, P.force_mode, P.use_Q = rho_ref, force_mode, use_Q
    return P


class Domain2D:
    """Whole-domain FP64 reference run on D2Q9 (paper layout: two colours x 9)."""

    def __init__(self, params: Params2D):
        self.params = params
        self.N = params.nx * params.ny
        self.shape = (params.ny, params.nx)
        self.h = lib2().o2_create(ctypes.byref(params))

    def __del__(self):
        if getattr(self, "h", None):
            lib2().o2_destroy(self.h)
            self.h = None

    def init(self, rho_r, rho_b, u):
        lib2().o2_init(self.h, _p(_d(rho_r).reshape(-1)), _p(_d(rho_b).reshape(-1)), _p(_d(u).reshape(-1)))

    def step(self, n=1):
        lib2().o2_step(self.h, int(n))

    def macros(self):
        N, sh = self.N, self.shape
        rr, rb, p, phi = (np.zeros(N) for _ in range(4))
        u = np.zeros(2 * N)
        lib2().o2_read_macros(self.h, _p(rr), _p(rb), _p(u), _p(p), _p(phi))
        return {"rho_r": rr.reshape(sh), "rho_b": rb.reshape(sh), "u": u.reshape((2,) + sh),
                "p": p.reshape(sh), "phi": phi.reshape(sh)}

    def populations(self):
        fr, fb = np.zeros(9 * self.N), np.zeros(9 * self.N)
        lib2().o2_read_populations(self.h, _p(fr), _p(fb))
        return fr.reshape((9,) + self.shape), fb.reshape((9,) + self.shape)

    def mass(self):
        m = np.zeros(2)
        lib2().o2_mass(self.h, _p(m))
        return m
