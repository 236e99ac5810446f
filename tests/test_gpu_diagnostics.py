"""Device-side diagnostics (cg_reduce_diagnostics) against the same quantities
computed on the host from the oracle's fields and from the GPU's own
read-back: masses, momenta, centroids (circular means on periodic axes),
the red second-moment tensor, the pressure jump of the Laplace test (Sec.
IV.A) and the rise quantities of the bubble test (Sec. IV.D)."""
import math

import numpy as np
import pytest

from paper_2309_07801_gb300 import inputs
from parity_util import run_pair

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


def host_diagnostics(m, bc, center, r_in, r_out, solid=None):
    """The definitions of the C header, written out over host arrays
    ([z, y, x]; u as [3, z, y, x])."""
    rr, rb, u, p, phi = m["rho_r"], m["rho_b"], m["u"], m["p"], m["phi"]
    nz, ny, nx = rr.shape
    n = (nx, ny, nz)
    fluid = np.ones_like(rr, bool) if solid is None else solid == 0
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xs = (coords[2], coords[1], coords[0])
    out = {"mass": np.array([rr.sum(), rb.sum()]),
           "red_volume": float((0.5 * (1 + phi))[fluid].sum()),
           "momentum": np.array([[(w * u[a])[fluid].sum() for a in range(3)] for w in (rr, rb)])}
    cen = np.zeros((2, 3))
    for k, w in enumerate((rr, rb)):
        for a in range(3):
            if bc[a] == 0:
                th = 2 * math.pi * xs[a] / n[a]
                ang = math.atan2(float((w * np.sin(th)).sum()), float((w * np.cos(th)).sum()))
                cen[k, a] = (ang % (2 * math.pi)) * n[a] / (2 * math.pi)
            else:
                cen[k, a] = float((w * xs[a]).sum() / w.sum())
    out["centroid"] = cen

    def off(a, c):
        d = xs[a] - c
        if bc[a] == 0:
            d = (d + 0.5 * n[a]) % n[a] - 0.5 * n[a]
        return d
    d = [off(a, cen[0, a]) for a in range(3)]
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    out["second_moment"] = np.array([(rr * d[i] * d[j]).sum() for i, j in pairs]) / rr.sum()
    dc = [off(a, center[a]) for a in range(3)]
    r2 = dc[0] ** 2 + dc[1] ** 2 + dc[2] ** 2
    inner, outer = fluid & (r2 < r_in ** 2), fluid & (r2 > r_out ** 2)
    out["p_in"], out["p_out"] = float(p[inner].mean()), float(p[outer].mean())
    out["n_in"], out["n_out"] = int(inner.sum()), int(outer.sum())
    out["u_max"] = float(np.sqrt((u ** 2).sum(axis=0))[fluid].max())
    return out


def _close(got, ref, rtol, atol=0.0):
    for key in ("mass", "red_volume", "momentum", "centroid", "second_moment", "p_in", "p_out", "u_max"):
        g, r = np.asarray(got[key], float), np.asarray(ref[key], float)
        scale = max(float(np.abs(r).max()), 1e-300)
        assert np.abs(g - r).max() <= rtol * scale + atol, (key, g, r)
    assert got["n_in"] == ref["n_in"] and got["n_out"] == ref["n_out"]


def test_diagnostics_of_the_32_droplet_match_the_oracle_fields():
    """FP64, 32^3 ratio-10 droplet with noise, off-centre, 60 steps: the
    device reductions equal the host definitions applied to the oracle's
    fields (to 1e-12); the droplet straddles the periodic z boundary, which
    the circular mean handles."""
    ar, ab = inputs.rest_fractions(1.0, 0.1)
    params = dict(nx=32, ny=32, nz=32, rho_r0=1.0, rho_b0=0.1, alpha_r=ar, alpha_b=ab,
                  nu_r=0.05, nu_b=0.08, sigma=0.01, beta=0.7)
    fields = inputs.droplet_fields((32, 32, 32), (26.3, 16.2, 3.9), 8.0, 1.0, 0.1,
                                   u0=(0.02, -0.01, 0.015), noise=1e-3, seed=2)
    od, gd = run_pair(params, fields, 60, "f64")
    center, r_in, r_out = (26.3, 16.2, 3.9), 4.0, 14.0
    got = gd.diagnostics(center, r_in, r_out)
    ref = host_diagnostics(od.macros(), (0, 0, 0), center, r_in, r_out)
    _close(got, ref, 1e-12)
    assert got["nonfinite"] == 0 and got["n_in"] > 100 and got["n_out"] > 1000
    assert got["p_in"] > got["p_out"]  # Laplace: higher pressure inside
    # the droplet straddles the periodic z boundary: the circular mean stays
    # within a few cells of its centre (an arithmetic mean would be near 16)
    assert np.abs(got["centroid"][0] - np.array([26.3, 16.2, 3.9])).max() < 3.0


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_diagnostics_match_the_host_on_the_gpu_readback(prec):
    """FP32 and FP16S storage: the device reductions equal the host
    definitions applied to the GPU's own read-back (same float fields, FP64
    sums in another order)."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.translating_droplet(64)
    d = cg.Domain(cg.make_params(precision=prec, **wl.params()))
    d.init(*inputs.workload_fields(wl))
    d.step(40)
    c = (32.0, 32.0, 32.0)
    got = d.diagnostics(c, 5.0, 15.0)
    ref = host_diagnostics(d.macros(), (0, 0, 0), c, 5.0, 15.0)
    _close(got, ref, 1e-12)
    # bitwise reproducible: the same call again, and after more reads
    again = d.diagnostics(c, 5.0, 15.0)
    for key in got:
        assert np.array_equal(np.asarray(got[key]), np.asarray(again[key])), key


def test_diagnostics_with_walls_give_the_bubble_rise_quantities():
    """Ratio-1000 bubble between z walls (FP32): blue centroid along the wall
    axis is the arithmetic mean, the rise velocity V_c = sum rho_b u_z /
    sum rho_b of Sec. IV.D, both equal to the host definitions."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.rising_bubble_case2(32, 32, 64)
    d = cg.Domain(cg.make_params(precision="f32", **wl.params()))
    d.init(*inputs.workload_fields(wl))
    d.step(50)
    m = d.macros()
    solid = np.zeros_like(m["rho_r"], np.uint8)
    solid[0] = solid[-1] = 1
    got = d.diagnostics((16.0, 16.0, 32.0), 3.0, 10.0)
    ref = host_diagnostics(m, (0, 0, 1), (16.0, 16.0, 32.0), 3.0, 10.0, solid)
    _close(got, ref, 1e-12)
    rb = m["rho_b"]
    zc = float((rb * np.arange(64)[:, None, None]).sum() / rb.sum())
    assert abs(got["centroid"][1][2] - zc) < 1e-12 * 64
    vc = float((rb * m["u"][2]).sum() / rb.sum())
    assert abs(got["momentum"][1][2] / got["mass"][1] - vc) < 1e-9 * max(abs(vc), 1e-12) + 1e-15
