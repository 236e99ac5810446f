"""cg_mass_noalloc: the per-colour mass without any device allocation.

Callers that cannot allocate device memory where they need the sums (they hold
only device pointers to density fields, or must not call cudaMalloc) use this
entry point; its partial sums live in a static array inside the library.  The
test calls it through the C ABI on device density fields and checks it against
cg_reduce() of the same state, twice in a row, for both precisions and for a
large field followed by a small one (the shared array keeps the previous
call's contents).  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-13  # relative, as in the mass checks of the parity tests


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2309_07801_gb300 import build, cg as binding
    build.build()
    binding.lib()
    return binding


def _device_fields(cg, edge, precision, steps):
    import torch
    from paper_2309_07801_gb300 import inputs
    wl = inputs.translating_droplet(edge)
    d = cg.Domain(cg.make_params(precision=precision, **wl.params()))
    d.init(*inputs.workload_fields(wl))
    d.step(steps)
    ref, flag = d.mass()
    assert flag == 0
    m = d.macros()
    dtype = torch.float32 if precision == "f32" else torch.float64
    # the macroscopic read-back is exact (FP32 -> FP64), so the device copies
    # hold the very values cg_reduce() summed
    rr = torch.from_numpy(m["rho_r"].reshape(-1).copy()).to(device="cuda", dtype=dtype)
    rb = torch.from_numpy(m["rho_b"].reshape(-1).copy()).to(device="cuda", dtype=dtype)
    stream = torch.cuda.current_stream().cuda_stream
    d.close()
    return rr, rb, ref, stream


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_mass_noalloc_matches_cg_reduce(cg, precision):
    code = cg.CG_F32 if precision == "f32" else cg.CG_F64
    big = _device_fields(cg, 128, precision, 10)
    small = _device_fields(cg, 32, precision, 10)
    for rr, rb, ref, stream in (big, small, big):
        for _ in range(2):
            out = cg.cg_mass_noalloc(rr.data_ptr(), rb.data_ptr(), rr.numel(), code, stream)
            assert np.all(np.abs(out - ref) / ref < MASS_TOL), (out, ref)


def test_mass_noalloc_rejects_oversize_and_empty(cg):
    with pytest.raises(cg.CGError) as e:
        cg.cg_mass_noalloc(0, 0, cg.CG_NOALLOC_MAX_CELLS + 1, cg.CG_F32, 0)
    assert e.value.code == -1 and "limit" in str(e.value)
    assert np.array_equal(cg.cg_mass_noalloc(0, 0, 0, cg.CG_F64, 0), np.zeros(2))
