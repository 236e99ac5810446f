"""The C-ABI library loads and exports every symbol include/cg27.h declares;
host-side validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cg27.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def cg():
    from paper_2309_07801_gb300 import build, cg as binding
    build.build()
    binding.lib()
    return binding


def test_every_declared_symbol_is_exported(cg):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(cg.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    # and the binding wraps each of them under the same name
    assert set(names) == set(cg.SIGNATURES)


def test_params_struct_layout_matches_header(cg):
    # offsets follow the C declaration order; size includes the trailing ints
    p = cg.cg_params()
    assert ctypes.sizeof(p) == 4 * 6 + 8 * 8 + 8 * 11 + 8 * 3 + 8 + 4 * 6 + 8 * 18 + 4 * 2
    assert cg.cg_abi_version() == 5


def test_defaults_and_workspace(cg):
    p = cg.cg_params_default(32, 16, 8)
    assert (p.nx, p.ny, p.nz) == (32, 16, 8)
    assert p.model == cg.CG_MODEL_D and p.use_Q == 1 and p.precision == cg.CG_F32
    assert all(p.omega[q] == 1.0 for q in range(11))
    assert abs(p.alpha_r - 8 / 27) < 1e-16 and p.beta == 0.7
    n = 32 * 16 * 8
    b32 = cg.cg_workspace_bytes(p)
    # two population copies (27) + two recoloring states (5) + 15 side fields
    # (rho_r, rho_b, j, phi, F, (p - rho c_s^2) u, Q)
    assert b32 >= n * 4 * (2 * 27 + 2 * 5 + 15)
    p.precision = cg.CG_F64
    assert cg.cg_workspace_bytes(p) >= 2 * n * 4 * (2 * 27 + 2 * 5 + 15)
    p.precision = cg.CG_F32
    p.bc[2] = cg.CG_BC_BOUNCEBACK
    assert cg.cg_workspace_bytes(p) > b32  # walls reserve the blue part and the mask


@pytest.mark.parametrize("field,value", [("nx", 0), ("rho_r0", 0.0), ("alpha_b", 1.0),
                                         ("nu_r", -1.0), ("model", 7), ("force_mode", 9),
                                         ("precision", 5), ("lattice", 2)])
def test_invalid_params_rejected(cg, field, value):
    p = cg.cg_params_default(8, 8, 8)
    setattr(p, field, value)
    with pytest.raises(cg.CGError) as e:
        cg.cg_workspace_bytes(p)
    assert e.value.code in (-1, -2)
    assert cg.cg_last_error()


def test_bounceback_axis_needs_three_cells(cg):
    p = cg.cg_params_default(8, 8, 2)
    p.bc[2] = cg.CG_BC_BOUNCEBACK
    with pytest.raises(cg.CGError):
        cg.cg_workspace_bytes(p)


def test_create_rejects_bad_workspace(cg):
    p = cg.cg_params_default(8, 8, 8)
    need = cg.cg_workspace_bytes(p)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(p, 0, need, 0)
    assert e.value.code == -5
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(p, 256, need - 1, 0)
    assert e.value.code == -5
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(p, 257, need, 0)
    assert e.value.code == -5


@pytest.mark.parametrize("prec", ["f16s", "bf16s"])
def test_walls_rejected_with_16_bit_storage(cg, prec):
    p = cg.make_params(8, 8, 8, precision=prec)
    assert cg.cg_workspace_bytes(p) > 0
    p.bc[2] = cg.CG_BC_BOUNCEBACK
    with pytest.raises(cg.CGError) as e:
        cg.cg_workspace_bytes(p)
    assert e.value.code == -2
    p.bc[2] = cg.CG_BC_PERIODIC
    p.solid_mask = 1
    with pytest.raises(cg.CGError) as e:
        cg.cg_workspace_bytes(p)
    assert e.value.code == -2


def test_16_bit_storage_size_limit(cg):
    """27 x cells must stay below 2^32 with 16-bit populations (32-bit indices)."""
    p = cg.make_params(540, 540, 540, precision="f16s")
    assert cg.cg_workspace_bytes(p) > 0
    p = cg.make_params(600, 600, 600, precision="bf16s")
    with pytest.raises(cg.CGError) as e:
        cg.cg_workspace_bytes(p)
    assert e.value.code == -2
    p.precision = cg.CG_F32
    assert cg.cg_workspace_bytes(p) > 0


def test_wall_kinds_validated(cg):
    wall_u = [[0.0] * 3 for _ in range(6)]
    wall_u[5] = [0.02, 0.0, 0.0]
    p = cg.make_params(8, 8, 8, bc=(cg.CG_BC_SLIP, 0, cg.CG_BC_MOVING), wall_u=wall_u)
    assert cg.cg_workspace_bytes(p) > cg.cg_workspace_bytes(cg.make_params(8, 8, 8))  # walls reserve AUX
    wall_u[5] = [0.0, 0.0, 0.01]  # a moving wall must move in its own plane
    with pytest.raises(cg.CGError):
        cg.cg_workspace_bytes(cg.make_params(8, 8, 8, bc=(0, 0, cg.CG_BC_MOVING), wall_u=wall_u))
    wall_u[5] = [float("nan"), 0.0, 0.0]
    with pytest.raises(cg.CGError):
        cg.cg_workspace_bytes(cg.make_params(8, 8, 8, bc=(0, 0, cg.CG_BC_MOVING), wall_u=wall_u))
    with pytest.raises(cg.CGError):
        cg.cg_workspace_bytes(cg.make_params(8, 8, 2, bc=(0, 0, cg.CG_BC_SLIP)))
    with pytest.raises(cg.CGError):
        cg.cg_workspace_bytes(cg.make_params(8, 8, 8, bc=(0, 4, 0)))


def test_d2q9_parameters_validated(cg):
    p = cg.make_params(16, 8, 1, lattice=cg.CG_D2Q9, bc=(0, 1, 0))
    assert cg.cg_workspace_bytes(p) > 0
    for bad in (dict(nz=2), dict(bc=(0, 0, 1)), dict(bc=(2, 0, 0)), dict(model=cg.CG_MODEL_A),
                dict(precision="f16s"), dict(solid_mask=1)):
        kw = dict(lattice=cg.CG_D2Q9)
        kw.update(bad)
        nz = kw.pop("nz", 1)
        with pytest.raises(cg.CGError):
            cg.cg_workspace_bytes(cg.make_params(16, 8, nz, **kw))


@pytest.mark.parametrize("precision,walls", [("f64", False), ("f32", True), ("f16s", False)])
def test_in_place_streaming_saves_one_population_copy(cg, precision, walls):
    """CG_STREAM_IN_PLACE keeps one population buffer (and one wall buffer)."""
    p = cg.make_params(40, 24, 16, precision=precision, bc=(0, 0, 1) if walls else (0, 0, 0))
    two = cg.cg_workspace_bytes(p)
    p.streaming = cg.CG_STREAM_IN_PLACE
    one = cg.cg_workspace_bytes(p)
    stride = (40 * 24 * 16 + 63) // 64 * 64
    pop = {"f64": 8, "f32": 4, "f16s": 2}[precision]
    saved = 27 * stride * pop + (27 * stride * 4 if walls else 0)
    assert abs((two - one) - saved) <= 2 * 256, (two, one, saved)


def test_in_place_streaming_validation(cg):
    p = cg.make_params(16, 16, 1, lattice=cg.CG_D2Q9, streaming=cg.CG_STREAM_IN_PLACE)
    with pytest.raises(cg.CGError) as e:
        cg.cg_workspace_bytes(p)
    assert e.value.code == -2 and "D3Q27" in str(e.value)
    for bad in (("streaming", 2), ("streaming", -1), ("reserved0", 1)):
        p = cg.make_params(8, 8, 8, **dict([bad]))
        with pytest.raises(cg.CGError) as e:
            cg.cg_workspace_bytes(p)
        assert e.value.code == -1


def test_batch_entry_points_validate_without_a_gpu(cg):
    """The batch calls reject bad arguments before touching the device."""
    L = cg.lib()
    n = ctypes.c_size_t(0)
    assert L.cg_batch_workspace_bytes(8, cg.CG_F32, ctypes.byref(n)) == 0 and n.value > 0
    small = n.value
    assert L.cg_batch_workspace_bytes(64, cg.CG_F32, ctypes.byref(n)) == 0 and n.value >= small
    for bad in ((0, cg.CG_F32), ((1 << 20) + 1, cg.CG_F32)):
        assert L.cg_batch_workspace_bytes(bad[0], bad[1], ctypes.byref(n)) == -1
    assert L.cg_batch_workspace_bytes(4, 7, ctypes.byref(n)) == -2       # unknown precision
    assert L.cg_batch_workspace_bytes(4, cg.CG_F32, None) == -1
    out = ctypes.c_void_p()
    assert L.cg_batch_create(4, cg.CG_F32, None, 1 << 20, None, ctypes.byref(out)) == -5  # no workspace
    i32 = ctypes.c_int32(0)
    for rc in (L.cg_batch_step(None, 1), L.cg_batch_sync(None), L.cg_batch_set_depth(None, 2),
               L.cg_batch_set_persistent(None, 0), L.cg_batch_persistent(None, ctypes.byref(i32)),
               L.cg_batch_size(None, ctypes.byref(i32)), L.cg_batch_add(None, None),
               L.cg_batch_remove(None, None), L.cg_batch_destroy(None)):
        assert rc == -1
    assert "NULL" in cg.cg_last_error() or "batch" in cg.cg_last_error()


def test_diagnostics_struct_layout_and_null_arguments(cg):
    """cg_diagnostics: 23 doubles, two int64 counts, one double, two int32."""
    assert ctypes.sizeof(cg.cg_diagnostics) == 8 * 23 + 8 * 2 + 8 + 4 * 2
    assert cg.cg_diagnostics.n_in.offset == 8 * 23
    out = cg.cg_diagnostics()
    rc = cg.lib().cg_reduce_diagnostics(None, None, 0.0, 0.0, ctypes.byref(out))
    assert rc == -1 and "NULL" in cg.cg_last_error()
