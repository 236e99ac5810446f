"""Python binding of the C ABI in ``include/cg27.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``libcg27.so``; this module
only converts numpy arrays to pointers, lets PyTorch own the device workspace
and the stream, and turns error codes into exceptions.  There is no fallback:
if the library is missing, importing the binding fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcg27.so")

CG_OK = 0
CG_BC_PERIODIC, CG_BC_BOUNCEBACK, CG_BC_SLIP, CG_BC_MOVING = 0, 1, 2, 3
CG_FORCE_NONE, CG_FORCE_CONST, CG_FORCE_GRAVITY, CG_FORCE_BUOYANCY = 0, 1, 2, 3
CG_MODEL_A, CG_MODEL_B, CG_MODEL_C, CG_MODEL_D = 0, 1, 2, 3
CG_F64, CG_F32, CG_F16S, CG_BF16S = 0, 1, 2, 3
CG_D3Q27, CG_D2Q9 = 0, 1
CG_STREAM_TWO_BUFFERS, CG_STREAM_IN_PLACE = 0, 1
PRECISIONS = {"f64": CG_F64, "f32": CG_F32, "f16s": CG_F16S, "bf16s": CG_BF16S}


class CGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("cg27 error %d: %s" % (code, msg))
        self.code = code


class cg_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 3),
                ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
                ("alpha_r", ctypes.c_double), ("alpha_b", ctypes.c_double),
                ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double),
                ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("omega", ctypes.c_double * 11), ("g", ctypes.c_double * 3),
                ("rho_ref", ctypes.c_double),
                ("force_mode", ctypes.c_int32), ("model", ctypes.c_int32),
                ("use_Q", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("solid_mask", ctypes.c_int32), ("lattice", ctypes.c_int32),
                ("wall_u", (ctypes.c_double * 3) * 6),
                ("streaming", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class cg_diagnostics(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2), ("red_volume", ctypes.c_double),
                ("momentum", (ctypes.c_double * 3) * 2), ("centroid", (ctypes.c_double * 3) * 2),
                ("second_moment", ctypes.c_double * 6), ("p_in", ctypes.c_double),
                ("p_out", ctypes.c_double), ("n_in", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("u_max", ctypes.c_double), ("nonfinite", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# exported entry points of include/cg27.h: name -> (restype, argtypes)
_VP, _DP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "cg_params_default": (ctypes.c_int, [ctypes.POINTER(cg_params), ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32]),
    "cg_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(cg_params), ctypes.POINTER(ctypes.c_size_t)]),
    "cg_create": (ctypes.c_int, [ctypes.POINTER(cg_params), _VP, ctypes.c_size_t, _VP,
                                 ctypes.POINTER(_VP)]),
    "cg_init_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cg_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "cg_read_macros": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "cg_read_populations": (ctypes.c_int, [_VP, _VP, _VP]),
    "cg_reduce": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int32)]),
    "cg_reduce_diagnostics": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(cg_diagnostics)]),
    "cg_state_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_save_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "cg_load_state": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "cg_steps_taken": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "cg_set_schedule": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "cg_schedule": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32)]),
    "cg_set_schedule_form": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "cg_schedule_form": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cg_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "cg_profile_read": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_int64)]),
    "cg_mass_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP]),
    "cg_destroy": (ctypes.c_int, [_VP]),
    "cg_last_error": (ctypes.c_char_p, []),
    "cg_abi_version": (ctypes.c_int, []),
    "cg_batch_workspace_bytes": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_size_t, _VP,
                                       ctypes.POINTER(_VP)]),
    "cg_batch_add": (ctypes.c_int, [_VP, _VP]),
    "cg_batch_remove": (ctypes.c_int, [_VP, _VP]),
    "cg_batch_size": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "cg_batch_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "cg_batch_sync": (ctypes.c_int, [_VP]),
    "cg_batch_set_depth": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "cg_batch_depth": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cg_batch_set_persistent": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "cg_batch_persistent": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "cg_batch_set_tile": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "cg_batch_set_stop": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "cg_batch_tile": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "cg_batch_destroy": (ctypes.c_int, [_VP])
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libcg27.so (built by paper_2309_07801_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcg27.so not found at %s: run paper_2309_07801_gb300.build.build() "
                               "(needs nvcc); there is no CPU fallback" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != CG_OK:
        raise CGError(rc, lib().cg_last_error().decode())


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- the C ABI, one wrapper per entry point ----------------------------------------

def cg_params_default(nx: int, ny: int, nz: int) -> cg_params:
    p = cg_params()
    _check(lib().cg_params_default(ctypes.byref(p), nx, ny, nz))
    return p


def cg_workspace_bytes(p: cg_params) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().cg_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def cg_create(p: cg_params, d_workspace: int, nbytes: int, stream: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().cg_create(ctypes.byref(p), ctypes.c_void_p(d_workspace), nbytes,
                           ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def cg_init_fields(h, rho_r: np.ndarray, rho_b: np.ndarray, u: np.ndarray,
                   solid: Optional[np.ndarray] = None):
    _check(lib().cg_init_fields(h, _ptr(rho_r), _ptr(rho_b), _ptr(u), _ptr(solid)))


def cg_step(h, nsteps: int):
    _check(lib().cg_step(h, int(nsteps)))


def cg_read_macros(h, rho_r=None, rho_b=None, u=None, p=None, phi=None):
    _check(lib().cg_read_macros(h, _ptr(rho_r), _ptr(rho_b), _ptr(u), _ptr(p), _ptr(phi)))


def cg_read_populations(h, fr=None, fb=None):
    _check(lib().cg_read_populations(h, _ptr(fr), _ptr(fb)))


def cg_reduce(h):
    m = np.zeros(2)
    flag = ctypes.c_int32(0)
    _check(lib().cg_reduce(h, _ptr(m), ctypes.byref(flag)))
    return m, int(flag.value)


def cg_reduce_diagnostics(h, center=(0.0, 0.0, 0.0), r_in=0.0, r_out=float("inf")) -> dict:
    """Device-side FP64 diagnostics of the latest state (see the C header)."""
    c = np.ascontiguousarray(center, dtype=np.float64)
    out = cg_diagnostics()
    _check(lib().cg_reduce_diagnostics(h, _ptr(c), float(r_in), float(r_out), ctypes.byref(out)))
    return {"mass": np.array(out.mass[:]), "red_volume": out.red_volume,
            "momentum": np.array([out.momentum[k][:] for k in range(2)]),
            "centroid": np.array([out.centroid[k][:] for k in range(2)]),
            "second_moment": np.array(out.second_moment[:]), "p_in": out.p_in, "p_out": out.p_out,
            "n_in": int(out.n_in), "n_out": int(out.n_out), "u_max": out.u_max,
            "nonfinite": int(out.nonfinite)}


def cg_state_bytes(h) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().cg_state_bytes(h, ctypes.byref(n)))
    return n.value


def cg_save_state(h, buf: np.ndarray):
    _check(lib().cg_save_state(h, _ptr(buf), buf.nbytes))


def cg_load_state(h, buf: np.ndarray):
    _check(lib().cg_load_state(h, _ptr(buf), buf.nbytes))


def cg_steps_taken(h) -> int:
    n = ctypes.c_int64(0)
    _check(lib().cg_steps_taken(h, ctypes.byref(n)))
    return n.value


def cg_set_schedule(h, planes: int, tz: int):
    _check(lib().cg_set_schedule(h, int(planes), int(tz)))


def cg_schedule(h):
    """(planes, tz, tuning) of the step graphs."""
    a, b, t = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cg_schedule(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)))
    return a.value, b.value, bool(t.value)


def cg_set_schedule_form(h, planes: int, tz: int, fused_tz: int):
    _check(lib().cg_set_schedule_form(h, int(planes), int(tz), int(fused_tz)))


def cg_schedule_form(h):
    """(planes, tz, fused_tz, tuning): the schedule and the step form
    (fused_tz = 0: four passes, else the fused collision pass)."""
    a, b, f, t = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cg_schedule_form(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(f), ctypes.byref(t)))
    return a.value, b.value, f.value, bool(t.value)


def cg_profile_enable(h, max_steps: int):
    _check(lib().cg_profile_enable(h, int(max_steps)))


CG_NUM_PASSES = 4


def cg_profile_read(h):
    ms = np.zeros(CG_NUM_PASSES)
    n = ctypes.c_int64(0)
    _check(lib().cg_profile_read(h, _ptr(ms), ctypes.byref(n)))
    return ms, n.value


PASS_NAMES = ("k_macro", "k_fields", "k_div", "k_collide")

CG_NOALLOC_MAX_CELLS = 67108864


def cg_mass_noalloc(d_rho_r: int, d_rho_b: int, n: int, precision: int, stream: int) -> np.ndarray:
    """Per-colour mass of two device density fields (device pointers), using the
    library's static scratch instead of a workspace."""
    out = np.zeros(2)
    _check(lib().cg_mass_noalloc(ctypes.c_void_p(d_rho_r), ctypes.c_void_p(d_rho_b), int(n),
                                 int(precision), ctypes.c_void_p(stream), _ptr(out)))
    return out


def cg_destroy(h):
    _check(lib().cg_destroy(h))


def cg_last_error() -> str:
    return lib().cg_last_error().decode()


def cg_abi_version() -> int:
    return lib().cg_abi_version()


# ---- convenience: a domain whose device memory and stream belong to PyTorch -------------

def make_params(nx, ny, nz, *, precision="f32", **kw) -> cg_params:
    """cg_params with the library defaults, overridden by keyword arguments
    (names as in the C struct; bc, omega, g given as sequences)."""
    p = cg_params_default(nx, ny, nz)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for key, val in kw.items():
        if key in ("bc", "omega", "g"):
            arr = getattr(p, key)
            for i, v in enumerate(val):
                arr[i] = v
        elif key == "wall_u":
            for f, vec in enumerate(val):
                for b, v in enumerate(vec):
                    p.wall_u[f][b] = v
        else:
            setattr(p, key, val)
    return p


class Domain:
    """One simulation domain: workspace is a uint8 CUDA tensor, work runs on a
    torch CUDA stream (the current one unless given)."""

    def __init__(self, params: cg_params, device="cuda", stream=None):
        import torch
        self.params = params
        self.nbytes = cg_workspace_bytes(params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        self.h = cg_create(params, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self.nq = 9 if params.lattice == CG_D2Q9 else 27

    def close(self):
        if getattr(self, "h", None):
            cg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho_r, rho_b, u, solid=None):
        rr, rb, uu = _f64(rho_r).reshape(-1), _f64(rho_b).reshape(-1), _f64(u).reshape(-1)
        if rr.size != self.N or rb.size != self.N or uu.size != 3 * self.N:
            raise ValueError("field sizes do not match the domain")
        s = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        cg_init_fields(self.h, rr, rb, uu, s)

    def step(self, n: int = 1):
        cg_step(self.h, n)

    def macros(self) -> dict:
        N, sh = self.N, self.shape
        rr, rb, p, phi = (np.empty(N) for _ in range(4))
        u = np.empty(3 * N)
        cg_read_macros(self.h, rr, rb, u, p, phi)
        return {"rho_r": rr.reshape(sh), "rho_b": rb.reshape(sh), "u": u.reshape((3,) + sh),
                "p": p.reshape(sh), "phi": phi.reshape(sh)}

    def populations(self):
        fr = np.empty(self.nq * self.N)
        fb = np.empty(self.nq * self.N)
        cg_read_populations(self.h, fr, fb)
        return fr.reshape((self.nq,) + self.shape), fb.reshape((self.nq,) + self.shape)

    def mass(self):
        return cg_reduce(self.h)

    def diagnostics(self, center=(0.0, 0.0, 0.0), r_in=0.0, r_out=float("inf")) -> dict:
        return cg_reduce_diagnostics(self.h, center, r_in, r_out)

    def save(self) -> np.ndarray:
        buf = np.empty(cg_state_bytes(self.h), dtype=np.uint8)
        cg_save_state(self.h, buf)
        return buf

    def load(self, buf: np.ndarray):
        cg_load_state(self.h, np.ascontiguousarray(buf, dtype=np.uint8))

    @property
    def steps(self) -> int:
        return cg_steps_taken(self.h)

    @property
    def schedule(self):
        return cg_schedule(self.h)

    def set_schedule(self, planes: int, tz: int, fused_tz: int = 0):
        """Fix the schedule (and the step form: fused_tz > 0 takes the fused
        collision pass with tiles of fused_tz planes); all 0: tune again."""
        cg_set_schedule_form(self.h, planes, tz, fused_tz)

    @property
    def schedule_form(self):
        return cg_schedule_form(self.h)

    def tune(self, max_steps: int = 400) -> int:
        """Step until the schedule tuner has chosen (at most max_steps steps);
        returns the steps taken."""
        n = 0
        self.step(1)
        n += 1
        while self.schedule[2] and n < max_steps:
            self.step(8)
            n += 8
        return n


# ---- batches --------------------------------------------------------------------------------

def cg_batch_workspace_bytes(max_domains: int, precision) -> int:
    n = ctypes.c_size_t(0)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().cg_batch_workspace_bytes(int(max_domains), prec, ctypes.byref(n)))
    return n.value


def cg_batch_create(max_domains: int, precision, d_ws: int, nbytes: int, stream: int):
    out = _VP()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().cg_batch_create(int(max_domains), prec, ctypes.c_void_p(d_ws), nbytes,
                                 ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def cg_batch_add(b, h):
    _check(lib().cg_batch_add(b, h))


def cg_batch_remove(b, h):
    _check(lib().cg_batch_remove(b, h))


def cg_batch_size(b) -> int:
    n = ctypes.c_int32(0)
    _check(lib().cg_batch_size(b, ctypes.byref(n)))
    return n.value


def cg_batch_step(b, nsteps: int):
    _check(lib().cg_batch_step(b, int(nsteps)))


def cg_batch_sync(b):
    _check(lib().cg_batch_sync(b))


def cg_batch_set_depth(b, tz: int):
    _check(lib().cg_batch_set_depth(b, int(tz)))


def cg_batch_depth(b):
    tz, tuning = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cg_batch_depth(b, ctypes.byref(tz), ctypes.byref(tuning)))
    return tz.value, bool(tuning.value)


def cg_batch_set_persistent(b, mode: int):
    _check(lib().cg_batch_set_persistent(b, int(mode)))


def cg_batch_persistent(b) -> int:
    m = ctypes.c_int32(0)
    _check(lib().cg_batch_persistent(b, ctypes.byref(m)))
    return m.value


def cg_batch_set_stop(b, h, total_steps: int):
    _check(lib().cg_batch_set_stop(b, h, int(total_steps)))


def cg_batch_set_tile(b, shape: int):
    _check(lib().cg_batch_set_tile(b, int(shape)))


def cg_batch_tile(b):
    """(threads in x, threads in y) of the tile shape in use."""
    tx, ty = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cg_batch_tile(b, ctypes.byref(tx), ctypes.byref(ty)))
    return tx.value, ty.value


def cg_batch_destroy(b):
    _check(lib().cg_batch_destroy(b))


class Batch:
    """Domains advanced together in shared launches (see cg_batch_* in the C
    header).  The descriptor workspace is a uint8 CUDA tensor; launches go to a
    torch CUDA stream (a new one unless given)."""

    def __init__(self, max_domains: int, precision="f32", device="cuda", stream=None):
        import torch
        self.nbytes = cg_batch_workspace_bytes(max_domains, precision)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.workspace.device)
        self.h = cg_batch_create(max_domains, precision, self.workspace.data_ptr(), self.nbytes,
                                 self.stream.cuda_stream)
        self.members = []

    def add(self, dom: Domain):
        cg_batch_add(self.h, dom.h)
        self.members.append(dom)

    def remove(self, dom: Domain):
        cg_batch_remove(self.h, dom.h)
        self.members.remove(dom)

    def step(self, n: int = 1):
        cg_batch_step(self.h, n)

    def sync(self):
        cg_batch_sync(self.h)

    def set_depth(self, tz: int):
        cg_batch_set_depth(self.h, tz)

    @property
    def depth(self):
        return cg_batch_depth(self.h)

    def set_persistent(self, mode: int):
        cg_batch_set_persistent(self.h, mode)

    @property
    def persistent(self) -> int:
        return cg_batch_persistent(self.h)

    def set_stop(self, dom: Domain, total_steps: int):
        cg_batch_set_stop(self.h, dom.h, total_steps)

    def set_tile(self, shape: int):
        cg_batch_set_tile(self.h, shape)

    @property
    def tile(self):
        return cg_batch_tile(self.h)

    def __len__(self):
        return cg_batch_size(self.h)

    def close(self):
        if getattr(self, "h", None):
            cg_batch_destroy(self.h)
            self.h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
