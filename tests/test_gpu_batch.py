"""Batches of domains in shared launches, and the continuous-batching server:
a member's results equal those of stepping it alone -- bitwise in FP64, and in
FP32 / 16-bit storage within a bound far below the parity bar (the batched and
the single-domain kernels are compiled separately, and the compiler may fuse a
different product of a sum into a fused multiply-add, so their FP32 roundings
can differ in the last bit).  Within the batch path results do not depend on
the tile depth or on the other members: that is bitwise in every precision."""
import numpy as np
import pytest

from paper_2309_07801_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2309_07801_gb300 import build, cg
    build.build()
    cg.lib()


def _case(kind, edge_xyz, ratio, sigma, seed):
    nx, ny, nz = edge_xyz
    ar, ab = inputs.rest_fractions(1.0, 1.0 / ratio)
    params = dict(nx=nx, ny=ny, nz=nz, rho_r0=1.0, rho_b0=1.0 / ratio, alpha_r=ar, alpha_b=ab,
                  nu_r=0.1, nu_b=0.07, sigma=sigma, beta=0.7)
    c = (nx / 2.0, ny / 2.0, nz / 2.0)
    R = 0.3 * min(nx, ny, nz)
    semi = (R * 1.1, R * 0.95, R * 0.95) if kind == "osc" else None
    fields = inputs.droplet_fields((nz, ny, nx), c, R, 1.0, 1.0 / ratio, semi_axes=semi,
                                   u0=(0.02, -0.01, 0.0), noise=1e-3, seed=seed)
    return params, fields


CASES = [("static", (32, 32, 32), 1.0, 0.01, 1), ("osc", (48, 40, 24), 4.0, 0.005, 2),
         ("static", (70, 33, 17), 10.0, 0.02, 3), ("osc", (16, 16, 64), 2.5, 0.001, 4)]


def _solo(prec, params, fields, steps):
    from paper_2309_07801_gb300 import cg
    d = cg.Domain(cg.make_params(precision=prec, **params))
    d.init(*fields)
    d.step(steps)
    out = d.macros(), d.populations() if prec == "f64" else None, d.mass()
    d.close()
    return out


# agreement of a member with its solo run: in FP64 bitwise; in FP32 and FP16S
# the difference (densities, pressure, phi normwise, velocity absolute) must
# stay within twice the solo run's own rounding error, i.e. its difference
# from the FP64 run of the same case -- the mix changes a result by no more
# than the storage precision already does.
def _err(key, a, b):
    d = float(np.abs(a - b).max())
    return d if key == "u" else d / float(np.abs(b).max())


def _within_rounding(key, mix, solo, solo64):
    return _err(key, mix, solo) <= 2.0 * _err(key, solo, solo64) + 1e-9


@pytest.mark.parametrize("prec", ["f32", "f64", "f16s"])
def test_batch_members_equal_solo_runs(prec):
    from paper_2309_07801_gb300 import cg
    steps = 24
    b = cg.Batch(8, prec)
    doms = []
    for k, (kind, shape, ratio, sigma, seed) in enumerate(CASES):
        params, fields = _case(kind, shape, ratio, sigma, seed)
        d = cg.Domain(cg.make_params(precision=prec, **params))
        d.init(*fields)
        doms.append((d, params, fields))
    # the last domain joins after 7 steps (odd parity relative to the others)
    for d, _, _ in doms[:-1]:
        b.add(d)
    b.step(7)
    b.add(doms[-1][0])
    b.step(steps - 7)
    late = doms[-1][0]
    b.remove(late)
    b.step(0)
    b.sync()
    for k, (d, params, fields) in enumerate(doms):
        n = steps if k < len(doms) - 1 else steps - 7
        assert d.steps == n
        ref_mac, ref_pop, ref_mass = _solo(prec, params, fields, n)
        mac = d.macros()
        if prec == "f64":
            for key in ref_mac:
                assert np.array_equal(mac[key], ref_mac[key]), (k, key)
            fr, fb = d.populations()
            assert np.array_equal(fr, ref_pop[0]) and np.array_equal(fb, ref_pop[1])
        else:
            ref64 = _solo("f64", params, fields, n)[0]
            for key in ref_mac:
                assert _within_rounding(key, mac[key], ref_mac[key], ref64[key]), \
                    (prec, k, key, _err(key, mac[key], ref_mac[key]), _err(key, ref_mac[key], ref64[key]))
        m, flag = d.mass()
        assert flag == 0 and np.allclose(m, ref_mass[0], rtol={"f64": 0.0, "f32": 1e-6, "f16s": 1e-5}[prec], atol=0)
    b.close()
    for d, _, _ in doms:
        d.close()


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_batch_member_results_do_not_depend_on_the_mix(prec):
    """The same domain alone in a batch and among three others: bitwise equal."""
    from paper_2309_07801_gb300 import cg
    params, fields = _case(*CASES[1])
    outs = []
    for others in (0, 3):
        b = cg.Batch(8, prec)
        extra = []
        for kind, shape, ratio, sigma, seed in CASES[2:2 + others] + CASES[:max(0, others - 2)]:
            p2, f2 = _case(kind, shape, ratio, sigma, seed)
            e = cg.Domain(cg.make_params(precision=prec, **p2))
            e.init(*f2)
            b.add(e)
            extra.append(e)
        d = cg.Domain(cg.make_params(precision=prec, **params))
        d.init(*fields)
        b.add(d)
        b.step(19)
        b.remove(d)
        outs.append(d.macros())
        b.close()
        for e in extra + [d]:
            e.close()
    for key in outs[0]:
        assert np.array_equal(outs[0][key], outs[1][key]), key


def test_batch_depth_does_not_change_results():
    from paper_2309_07801_gb300 import cg
    params, fields = _case("osc", (48, 40, 24), 4.0, 0.005, 2)
    outs = []
    for tz in (1, 3, 24):
        b = cg.Batch(2, "f32")
        b.set_depth(tz)
        d = cg.Domain(cg.make_params(precision="f32", **params))
        d.init(*fields)
        b.add(d)
        b.step(20)  # four candidates (grid forms x tile shapes) at the fixed depth, four steps each
        assert b.depth == (tz, False)
        b.remove(d)
        outs.append(d.macros())
        b.close()
        d.close()
    for o in outs[1:]:
        for key in o:
            assert np.array_equal(o[key], outs[0][key])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_grid_form_does_not_change_results(prec):
    """One block per work item and the persistent grid (blocks walking the tile
    list) give the same bits, with members of different sizes in several
    groups, through chained and single steps."""
    from paper_2309_07801_gb300 import cg
    cases = [_case("osc", (48, 40, 24), 4.0, 0.005, 2), _case("static", (33, 30, 35), 2.0, 0.01, 3),
             _case("osc", (64, 64, 64), 1.5, 0.008, 4)]
    outs = []
    for mode in (0, 1):
        b = cg.Batch(4, prec)
        b.set_depth(3)
        b.set_persistent(mode)
        doms = []
        for params, fields in cases:
            d = cg.Domain(cg.make_params(precision=prec, **params))
            d.init(*fields)
            b.add(d)
            doms.append(d)
        b.step(3)
        b.step(9)
        assert b.persistent == mode and b.depth == (3, False)
        res = []
        for d in doms:
            b.remove(d)
            res.append(d.macros())
            d.close()
        b.close()
        outs.append(res)
    for a, c in zip(*outs):
        for key in a:
            assert np.array_equal(a[key], c[key]), key
    b = cg.Batch(1, prec)
    with pytest.raises(cg.CGError):
        b.set_persistent(2)
    b.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_tile_shape_does_not_change_results(prec):
    """The two tile shapes of the z-marching batch passes (32 x 8 and 32 x 4
    threads: block size and shared-memory rings) give the same bits, in both
    grid forms, with members of different sizes; the tuner, left alone, picks
    one of them and reports it."""
    from paper_2309_07801_gb300 import cg
    cases = [_case("osc", (48, 40, 24), 4.0, 0.005, 2), _case("static", (33, 30, 35), 2.0, 0.01, 3)]
    outs = []
    for shape, mode in ((0, 0), (1, 0), (1, 1)):
        b = cg.Batch(4, prec)
        b.set_depth(5)
        b.set_persistent(mode)
        b.set_tile(shape)
        doms = []
        for params, fields in cases:
            d = cg.Domain(cg.make_params(precision=prec, **params))
            d.init(*fields)
            b.add(d)
            doms.append(d)
        b.step(2)
        b.step(8)
        assert b.tile == ((32, 8) if shape == 0 else (32, 4))
        res = []
        for d in doms:
            b.remove(d)
            res.append(d.macros())
            d.close()
        b.close()
        outs.append(res)
    for other in outs[1:]:
        for a, c in zip(outs[0], other):
            for key in a:
                assert np.array_equal(a[key], c[key]), key
    b = cg.Batch(2, prec)
    with pytest.raises(cg.CGError):
        b.set_tile(2)
    params, fields = cases[0]
    d = cg.Domain(cg.make_params(precision=prec, **params))
    d.init(*fields)
    b.add(d)
    b.step(60)  # the tuner times 12 candidate schedules, four steps each
    assert b.tile in ((32, 8), (32, 4)) and b.depth[1] is False
    b.remove(d)
    d.close()
    b.close()


def test_batch_rules():
    from paper_2309_07801_gb300 import cg
    b = cg.Batch(2, "f32")
    p1, f1 = _case("static", (32, 32, 32), 1.0, 0.01, 1)
    d1 = cg.Domain(cg.make_params(precision="f32", **p1))
    d1.init(*f1)
    b.add(d1)
    with pytest.raises(cg.CGError):       # already a member
        b.add(d1)
    with pytest.raises(cg.CGError):       # stepping a member on its own
        d1.step(1)
    with pytest.raises(cg.CGError):       # destroying a member
        cg.cg_destroy(d1.h)
    walls = cg.Domain(cg.make_params(precision="f32", bc=(0, 0, 1), **{k: v for k, v in p1.items()}))
    walls.init(*f1)
    with pytest.raises(cg.CGError) as e:  # another kernel variant
        b.add(walls)
    assert e.value.code == -2
    f64 = cg.Domain(cg.make_params(precision="f64", **p1))
    f64.init(*f1)
    with pytest.raises(cg.CGError):       # another precision
        b.add(f64)
    d2 = cg.Domain(cg.make_params(precision="f32", **p1))
    d2.init(*f1)
    b.add(d2)
    d3 = cg.Domain(cg.make_params(precision="f32", **p1))
    d3.init(*f1)
    with pytest.raises(cg.CGError):       # full
        b.add(d3)
    b.step(3)
    b.remove(d2)
    d2.step(2)                            # free again
    assert d2.steps == 5 and d1.steps == 3
    b.close()                             # members become free domains
    d1.step(1)
    for d in (d1, d2, d3, walls, f64):
        d.close()


def _requests(n=6, seed=9):
    reqs = inputs.serving_requests(n=n, rate=200.0, seed=seed)
    for k, r in enumerate(reqs):
        r.edge = (32, 48)[k % 2]
        r.radius = 0.3 * r.edge
        r.steps = 60 + 37 * k
    return reqs


def test_server_results_match_solo_runs_in_both_modes():
    from paper_2309_07801_gb300 import cg, serve
    reqs = _requests()
    out = {}
    for mode in ("batched", "per_run"):
        srv = serve.Server(mode=mode, quantum=25, keep_macros=True)
        res = srv.run(reqs)
        srv.close()
        assert res["runs"] == len(reqs) and res["nonfinite_runs"] == 0
        assert res["p50_s"] > 0 and res["p99_s"] >= res["p50_s"] and res["runs_per_h"] > 0
        out[mode] = {r.rid: r for r in res["results"]}
    for req in reqs:
        ref = {}
        for prec in ("f32", "f64"):
            d = cg.Domain(cg.make_params(precision=prec, **req.workload().params()))
            d.init(*req.fields())
            d.step(req.steps)
            ref[prec] = d.macros()
            d.close()
        for key in ref["f32"]:
            # per-run mode uses the single-domain kernels: bitwise
            assert np.array_equal(out["per_run"][req.rid].macros[key], ref["f32"][key]), (req.rid, key)
            got = out["batched"][req.rid].macros[key]
            assert _within_rounding(key, got, ref["f32"][key], ref["f64"][key]), \
                (req.rid, key, _err(key, got, ref["f32"][key]), _err(key, ref["f32"][key], ref["f64"][key]))


def test_server_admission_respects_the_memory_budget():
    from paper_2309_07801_gb300 import cg, serve
    reqs = _requests(n=5, seed=11)
    one = max(cg.cg_workspace_bytes(cg.make_params(precision="f32", **r.workload().params())) for r in reqs)
    srv = serve.Server(mode="batched", quantum=20, hbm_budget=one)
    res = srv.run(reqs)
    srv.close()
    assert res["runs"] == len(reqs) and res["max_active"] == 1


def test_server_admission_follows_free_device_memory():
    """Without a fixed budget a request is admitted only while the device's
    free memory (less the reserve) holds its workspace: with the reserve set
    so that one and a half workspaces are free, the runs go one at a time."""
    from paper_2309_07801_gb300 import cg, serve
    reqs = _requests(n=4, seed=12)
    for r in reqs:  # one size, so that one and a half workspaces hold exactly one run
        r.edge, r.radius = 48, 0.3 * 48
    one = max(cg.cg_workspace_bytes(cg.make_params(precision="f32", **r.workload().params())) for r in reqs)
    srv = serve.Server(mode="batched", quantum=20)
    srv.reserve += srv.free_bytes() - int(1.5 * one)
    assert one <= srv.free_bytes() < 2 * one
    res = srv.run(reqs)
    srv.close()
    assert res["runs"] == len(reqs) and res["max_active"] == 1 and res["nonfinite_runs"] == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_member_step_budget_sits_out_the_rest_of_the_call(prec):
    """Members with step budgets 5 and 13 and one without share batch steps of
    3 + 8 + 8 (single steps and chains of both parities): they end at 5, 13 and
    19 steps, each bit for bit equal to a batch holding it alone for exactly
    that many steps, and a member that has used its budget is not touched."""
    from paper_2309_07801_gb300 import cg
    cases = [_case("osc", (48, 40, 24), 4.0, 0.005, 2), _case("static", (33, 30, 35), 2.0, 0.01, 3),
             _case("osc", (40, 36, 40), 1.5, 0.008, 4)]
    budgets = (5, 13, None)
    b = cg.Batch(4, prec)
    doms = []
    for (params, fields), n in zip(cases, budgets):
        d = cg.Domain(cg.make_params(precision=prec, **params))
        d.init(*fields)
        b.add(d)
        if n is not None:
            b.set_stop(d, n)
        doms.append(d)
    for k in (3, 8, 8):
        b.step(k)
    b.sync()
    got = []
    for d in doms:
        got.append((d.steps, d.macros()))
    for d in doms:
        b.remove(d)
        d.close()
    b.close()
    assert [g[0] for g in got] == [5, 13, 19]
    for (params, fields), (n, mac) in zip(cases, got):
        r = cg.Batch(1, prec)
        d = cg.Domain(cg.make_params(precision=prec, **params))
        d.init(*fields)
        r.add(d)
        r.step(n)
        r.remove(d)
        ref = d.macros()
        d.close()
        r.close()
        for key in ref:
            assert np.array_equal(ref[key], mac[key]), (n, key)
