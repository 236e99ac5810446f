"""In-place population streaming (CG_STREAM_IN_PLACE, the AA pattern) against
the FP64 oracle and against the two-buffer layout.

With one population buffer, even steps read and write each cell's own slots
(directions reversed) and odd steps the neighbours' slots; the arithmetic is
that of the two-buffer pull, so results must be bitwise equal to it in every
precision, through single steps and chained step graphs of both parities,
walls, host read-backs and checkpoints.
"""
import numpy as np
import pytest

from paper_2309_07801_gb300 import inputs
from parity_util import compare_macros, compare_populations, run_pair

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2309_07801_gb300 import build, cg
    build.build()
    cg.lib()
    import oracle
    oracle.build()


def _ratio_params(nx, ny, nz, ratio=10.0, **kw):
    ar, ab = inputs.rest_fractions(1.0, 1.0 / ratio)
    d = dict(nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0 / ratio, alpha_r=ar, alpha_b=ab,
             nu_r=0.05, nu_b=0.08, sigma=0.01, beta=0.7)
    d.update(kw)
    return d


def _droplet(params, seed, u0=(0.02, -0.01, 0.015)):
    nx, ny, nz = params["nx"], params["ny"], params["nz"]
    return inputs.droplet_fields((nz, ny, nx), (nx / 2 - 0.3, ny / 2 + 0.2, nz / 2 - 0.1),
                                 min(nx, ny, nz) / 4.0, params["rho_r0"], params["rho_b0"],
                                 u0=u0, noise=1e-3, seed=seed)


def _assert_f64(od, gd):
    m = compare_macros(od, gd)
    f = compare_populations(od, gd)
    bad = {k: v for k, v in {**m, **f}.items() if k not in ("u_abs", "rho_cellrel") and v > F64_TOL}
    assert not bad, {**m, **f}


def test_f64_static_droplet_vs_oracle():
    wl = inputs.static_droplet_32()
    od, gd = run_pair(wl.params(), inputs.workload_fields(wl, noise=1e-3, seed=1), 200, "f64", streaming=1)
    _assert_f64(od, gd)
    assert np.all(np.abs(gd.mass()[0] - od.mass()) / od.mass() < 1e-13)


@pytest.mark.parametrize("bc", [(0, 0, 1), (1, 3, 2)])
def test_f64_walls_vs_oracle(bc):
    """Bounce-back z walls; and no-slip x, moving y, slip z walls (every edge
    and corner rule) on a ragged box, an odd number of steps."""
    wall_u = [[0.0] * 3, [0.0] * 3, [0.0, 0.0, 0.01], [-0.015, 0.0, 0.02], [0.0] * 3, [0.0] * 3]
    params = _ratio_params(9, 10, 11, bc=bc, force_mode=1, g=(0.0, 0.0, 1e-5), wall_u=wall_u)
    od, gd = run_pair(params, _droplet(params, seed=19), 51, "f64", streaming=1)
    _assert_f64(od, gd)


def _run(prec, streaming, params, fields, pieces, solid=None):
    from paper_2309_07801_gb300 import cg
    d = cg.Domain(cg.make_params(precision=prec, streaming=streaming,
                                 solid_mask=1 if solid is not None else 0, **params))
    d.init(*fields, solid=solid)
    for k in pieces:
        d.step(k)
    out = d.macros(), d.populations(), d.mass()
    d.close()
    return out


def _assert_same(a, b):
    ma, (fra, fba), (mass_a, _) = a
    mb, (frb, fbb), (mass_b, _) = b
    for key in ma:
        assert np.array_equal(ma[key], mb[key]), key
    assert np.array_equal(fra, frb) and np.array_equal(fba, fbb)
    assert np.array_equal(mass_a, mass_b)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s", "bf16s"])
def test_bitwise_equal_to_two_buffers_slab_graphs(prec):
    """64^3 (slab-pipeline graphs): single steps and chains of eight steps
    starting at both parities, host read-backs after odd and even counts."""
    wl = inputs.translating_droplet(64)
    fields = inputs.workload_fields(wl, noise=1e-3, seed=2)
    pieces = (3, 8, 1, 17, 2) if prec in ("f64", "f32") else (3, 17)
    a = _run(prec, 0, wl.params(), fields, pieces)
    b = _run(prec, 1, wl.params(), fields, pieces)
    _assert_same(a, b)


def test_bitwise_equal_to_two_buffers_walls_and_mask():
    """FP32 with moving and slip walls and a solid obstacle (plain launches:
    nz < 48) over an odd number of steps."""
    wall_u = [[0.0] * 3, [0.0] * 3, [0.0] * 3, [0.0] * 3, [0.02, 0.0, 0.0], [-0.02, 0.0, 0.0]]
    params = _ratio_params(20, 14, 22, ratio=3.0, bc=(2, 0, 3), wall_u=wall_u)
    fields = _droplet(params, seed=23)
    solid = np.zeros((22, 14, 20), dtype=np.uint8)
    solid[4:7, 3:6, 2:5] = 1
    a = _run("f32", 0, params, fields, (5, 8, 2), solid)
    b = _run("f32", 1, params, fields, (5, 8, 2), solid)
    _assert_same(a, b)


def test_checkpoint_resume_in_place():
    """A checkpoint taken after an odd step count resumes bitwise; a
    two-buffer checkpoint does not load into an in-place domain."""
    from paper_2309_07801_gb300 import cg
    params = _ratio_params(16, 12, 10, bc=(0, 0, 1))
    fields = _droplet(params, seed=4)
    p = cg.make_params(precision="f32", streaming=1, **params)
    a = cg.Domain(p)
    a.init(*fields)
    a.step(7)
    blob = a.save()
    a.step(9)
    ref = a.populations()
    b = cg.Domain(p)
    b.load(blob)
    b.step(9)
    got = b.populations()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    two = cg.Domain(cg.make_params(precision="f32", **params))
    two.init(*fields)
    with pytest.raises(cg.CGError):
        b.load(two.save())


def test_full_size_128_and_workspace():
    """The 128^3 translating droplet: 16 steps bitwise equal to the two-buffer
    layout, in a workspace smaller by one FP32 population copy."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.translating_droplet(128)
    fields = inputs.workload_fields(wl)
    a = _run("f32", 0, wl.params(), fields, (16,))
    b = _run("f32", 1, wl.params(), fields, (16,))
    _assert_same(a, b)
    two = cg.cg_workspace_bytes(cg.make_params(precision="f32", **wl.params()))
    one = cg.cg_workspace_bytes(cg.make_params(precision="f32", streaming=1, **wl.params()))
    assert two - one >= 27 * 4 * wl.cells


def test_batches_refuse_in_place_domains():
    from paper_2309_07801_gb300 import cg
    wl = inputs.static_droplet_32()
    d = cg.Domain(cg.make_params(precision="f32", streaming=1, **wl.params()))
    d.init(*inputs.workload_fields(wl))
    bt = cg.Batch(4, "f32")
    with pytest.raises(cg.CGError) as e:
        bt.add(d)
    assert e.value.code == -2
    bt.close()
    d.close()
