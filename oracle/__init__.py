"""FP64 CPU oracle for the D3Q27 colour-gradient CM-MRT step (arXiv 2309.07801).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product package never
does, and the two share no code.

The arithmetic lives in ``cg_oracle.c`` (plain C11 + OpenMP, FP64); this module
compiles it with gcc and exposes it through ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODEL_A, MODEL_B, MODEL_C, MODEL_D = 0, 1, 2, 3
BC_PERIODIC, BC_BOUNCEBACK, BC_SLIP, BC_MOVING = 0, 1, 2, 3
FORCE_NONE, FORCE_CONST, FORCE_GRAVITY, FORCE_BUOYANCY = 0, 1, 2, 3
FIELDS = {"grad_phi": (0, 3), "n": (1, 3), "kappa": (2, 1), "F": (3, 3),
          "Q": (4, 3), "omega1": (5, 1), "w": (6, 3), "R": (7, 3)}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or (
        os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                     os.path.getmtime(os.path.join(_HERE, "cg_oracle.h"))))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
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
