"""GPU: the fused step form (the collision of a step forms the pulled colour and
momentum sums of the next; Sec. II.A streaming, Eq. (recoloring)).

Its tiles recompute a one-cell ring and the planes above and below, with the
same instructions as the blocks that own them, and add the pulled terms in the
order of the macroscopic pass, so every result equals that of the four-pass
step bit for bit: checked on ragged sizes, tile depths that do not divide the
domain, both parities, switches between the forms in the middle of a run,
step graphs, checkpoints and the schedule tuner.  And the form itself against
the FP64 oracle at the FP32 bars of the parity tests.
"""
import numpy as np
import pytest

from paper_2309_07801_gb300 import inputs
from parity_util import compare_macros, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2309_07801_gb300 import build, cg
    build.build()
    cg.lib()
    import oracle
    oracle.build()


def _params(nx, ny, nz, ratio=10.0, **kw):
    ar, ab = inputs.rest_fractions(1.0, 1.0 / ratio)
    d = dict(nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0 / ratio, alpha_r=ar, alpha_b=ab,
             nu_r=0.05, nu_b=0.08, sigma=0.01, beta=0.7)
    d.update(kw)
    return d


def _fields(p, seed=1, u0=(0.03, -0.02, 0.015)):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    R = min(nx, ny, nz) / 3.5
    return inputs.droplet_fields((nz, ny, nx), (nx / 2 - 0.3, ny / 2 + 0.2, nz / 2 - 0.1), R,
                                 p["rho_r0"], p["rho_b0"], u0=u0, noise=1e-3, seed=seed)


def _state(d):
    """Everything a run exposes: macroscopic fields, both colours' populations, mass."""
    m = d.macros()
    fr, fb = d.populations()
    mass, flag = d.mass()
    return m, fr, fb, mass, flag


def _assert_same(a, b):
    ma, fra, fba, massa, flaga = a
    mb, frb, fbb, massb, flagb = b
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    assert np.array_equal(fra, frb) and np.array_equal(fba, fbb)
    assert np.array_equal(massa, massb) and flaga == flagb == 0


def _run(p, fields, plan, seed_sched=None):
    """Run `plan`, a list of (steps, schedule or None); schedule = (planes, tz,
    fused_tz) fixed with cg_set_schedule_form."""
    from paper_2309_07801_gb300 import cg
    d = cg.Domain(cg.make_params(precision="f32", **p))
    d.init(*fields)
    for n, sched in plan:
        if sched is not None:
            d.set_schedule(*sched)
        d.step(n)
    out = _state(d)
    form = d.schedule_form
    d.close()
    return out, form


@pytest.mark.parametrize("shape,ftz", [((40, 20, 24), 7), ((32, 16, 16), 16), ((33, 9, 13), 1),
                                       ((64, 8, 20), 20), ((24, 24, 12), 5)])
def test_fused_plain_launches_equal_four_passes(shape, ftz):
    """Domains below 32 planes take plain launches: the fused form over ragged
    tiles (x, y not multiples of 32 x 8) and depths that leave a short last
    tile equals the four passes bit for bit, for odd and even step counts."""
    p = _params(*shape)
    f = _fields(p, seed=2)
    nz = shape[2]
    ref, _ = _run(p, f, [(11, (nz, min(8, nz), 0))])
    got, form = _run(p, f, [(11, (nz, min(8, nz), ftz))])
    assert form[2] == ftz
    _assert_same(ref, got)


def test_switching_forms_mid_run_keeps_the_bits():
    """Four passes, fused, four passes, fused: the first fused step after the
    four-pass form runs the macroscopic pass once; results stay bitwise."""
    p = _params(40, 24, 20)
    f = _fields(p, seed=3)
    ref, _ = _run(p, f, [(17, (20, 8, 0))])
    got, _ = _run(p, f, [(3, (20, 8, 0)), (5, (20, 8, 6)), (2, (20, 8, 0)), (7, (20, 8, 9))])
    _assert_same(ref, got)


@pytest.mark.parametrize("sched", [(16, 8, 16), (32, 16, 32), (64, 32, 64), (64, 8, 13), (24, 8, 24)])
@pytest.mark.parametrize("first", [3, 4])
def test_fused_step_graphs_equal_four_passes(sched, first):
    """64^3 translating droplet through the fused step graphs (slabs, chains of
    eight of both parities, single steps) against plain four-pass launches."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.translating_droplet(64)
    fields = inputs.workload_fields(wl, noise=1e-3, seed=5)
    out = []
    for mode in ("plain", "fused"):
        d = cg.Domain(cg.make_params(precision="f32", **wl.params()))
        d.init(*fields)
        if mode == "plain":
            cg.cg_profile_enable(d.h, 40)
        else:
            d.set_schedule(*sched)
        d.step(first)
        d.step(16)
        d.step(1)
        d.step(23 - first)
        if mode == "fused":
            assert d.schedule_form[:3] == sched
        out.append(_state(d))
        d.close()
    _assert_same(out[0], out[1])


def test_fused_form_against_the_oracle():
    """The fused form at 32^3, 100 steps (ratio 10, translating droplet) against
    the FP64 oracle at the FP32 bars of the parity tests: total density 1e-5
    relative per cell, velocity 1e-6 absolute."""
    import oracle
    from paper_2309_07801_gb300 import cg
    p = _params(32, 32, 32)
    rr, rb, u = _fields(p, seed=4)
    od = oracle.Domain(oracle.make_params(**p))
    od.init(rr, rb, u)
    od.step(100)
    gd = cg.Domain(cg.make_params(precision="f32", **p))
    gd.init(rr, rb, u)
    gd.set_schedule(32, 8, 11)
    gd.step(100)
    assert gd.schedule_form[2] == 11
    m = compare_macros(od, gd)
    assert m["rho_cellrel"] < 1e-5 and m["u_abs"] < 1e-6, m
    fro, _ = od.populations()
    frg, _ = gd.populations()
    assert rel_err(frg, fro) < 1e-5
    gd.close()


def test_fused_checkpoint_resume_is_bitwise():
    """A checkpoint taken after fused steps holds the last step's sums; the
    resumed run (which starts with the macroscopic pass) equals the
    uninterrupted one."""
    from paper_2309_07801_gb300 import cg
    p = _params(40, 24, 36)
    f = _fields(p, seed=6)
    d = cg.Domain(cg.make_params(precision="f32", **p))
    d.init(*f)
    d.set_schedule(36, 8, 12)
    d.step(9)
    buf = d.save()
    mid = d.macros()
    d.step(10)
    ref = _state(d)
    e = cg.Domain(cg.make_params(precision="f32", **p))
    e.load(buf)
    for k, v in e.macros().items():
        assert np.array_equal(v, mid[k]), k
    e.set_schedule(36, 8, 12)
    e.step(10)
    _assert_same(ref, _state(e))
    d.close()
    e.close()


def test_tuning_after_fused_steps_keeps_the_bits():
    """Fused steps, then tuning again (cg_set_schedule_form(0, 0, 0)): the tuner
    keeps a four-pass schedule, and the whole run equals plain four-pass
    launches bit for bit."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.translating_droplet(64)
    fields = inputs.workload_fields(wl, noise=1e-3, seed=8)
    d = cg.Domain(cg.make_params(precision="f32", **wl.params()))
    d.init(*fields)
    d.set_schedule(32, 16, 32)
    d.step(13)
    d.set_schedule(0, 0, 0)
    n = 13 + d.tune(max_steps=600)
    planes, tz, ftz, tuning = d.schedule_form
    assert not tuning and ftz == 0
    ref = cg.Domain(cg.make_params(precision="f32", **wl.params()))
    ref.init(*fields)
    cg.cg_profile_enable(ref.h, n)
    ref.step(n)
    _assert_same(_state(ref), _state(d))


def test_fused_form_is_refused_where_it_does_not_apply():
    """FP64, 16-bit storage, in-place streaming and walls keep the four passes."""
    from paper_2309_07801_gb300 import cg
    p = _params(32, 16, 16)
    for kw in (dict(precision="f64"), dict(precision="f16s"), dict(precision="f32", streaming=1),
               dict(precision="f32", bc=(0, 0, 1))):
        d = cg.Domain(cg.make_params(**{**p, **kw}))
        with pytest.raises(cg.CGError):
            d.set_schedule(16, 8, 8)
        d.set_schedule(16, 8, 0)
        d.close()
