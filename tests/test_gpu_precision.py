"""16-bit population storage (CG_F16S, CG_BF16S) against the FP64 oracle and
the FP64 GPU path.

Populations are stored as FP16/BF16 deviations from the rest-state populations
(equilibrium at u = 0, Sec. II.A), everything else in FP32, masses reduced in
FP64.  The bars below are about three times the errors measured on GB300 for
these exact runs; they state the accuracy of each storage mode:

  run                                   quantity          f32      f16s     bf16s
  static droplet 32^3, 200 steps        density (cell)    1e-5     1e-5     5e-5
  (vs oracle)                           |du|              1e-6     1e-5     3e-5
  translating droplet 32^3, ratio 10,   density (cell)    1e-5     3e-3     3e-2
  200 steps (vs oracle)                 |du|              1e-6     2e-4     2e-3
  Laplace 32^3, 2000 steps (vs FP64)    dp relative       -        2e-4     2e-3
  head-on collision 64^3, 1500 steps    mass drift        -        5e-5     5e-5
  translating droplet 64^3, 1000 steps, centroid vs FP32 -  1e-2     5e-1
  read back every 250 steps             mass drift        -        1e-4     5e-3
"""
import numpy as np
import pytest

from paper_2309_07801_gb300 import inputs
from parity_util import compare_macros, run_pair

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


@pytest.mark.parametrize("prec,rho_tol,u_tol", [("f16s", 1e-5, 1e-5), ("bf16s", 5e-5, 3e-5)])
def test_static_droplet_vs_oracle(prec, rho_tol, u_tol):
    wl = inputs.static_droplet_32()
    od, gd = run_pair(wl.params(), inputs.workload_fields(wl, noise=1e-3, seed=1), 200, prec)
    m = compare_macros(od, gd)
    assert m["rho_cellrel"] <= rho_tol and m["u_abs"] <= u_tol, m
    mass, flag = gd.mass()
    assert flag == 0 and np.all(np.abs(mass - od.mass()) / od.mass() < 5e-6)


@pytest.mark.parametrize("prec,rho_tol,u_tol", [("f16s", 3e-3, 2e-4), ("bf16s", 3e-2, 2e-3)])
def test_translating_droplet_ratio10_vs_oracle(prec, rho_tol, u_tol):
    wl = inputs.translating_droplet(32)
    od, gd = run_pair(wl.params(), inputs.workload_fields(wl), 200, prec)
    m = compare_macros(od, gd)
    assert m["rho_cellrel"] <= rho_tol and m["u_abs"] <= u_tol, m


def _laplace_dp(prec):
    from paper_2309_07801_gb300 import cg
    wl = inputs.static_droplet_32()
    d = cg.Domain(cg.make_params(precision=prec, **wl.params()))
    d.init(*inputs.workload_fields(wl))
    d.step(2000)
    m = d.macros()
    z, y, x = np.meshgrid(np.arange(32), np.arange(32), np.arange(32), indexing="ij")
    r = np.sqrt((x - 16) ** 2 + (y - 16) ** 2 + (z - 16) ** 2)
    return m["p"][r < 4].mean() - m["p"][r > 12].mean()


@pytest.mark.parametrize("prec,tol", [("f16s", 2e-4), ("bf16s", 2e-3)])
def test_laplace_pressure_jump_vs_fp64(prec, tol):
    ref = _laplace_dp("f64")
    assert abs(_laplace_dp(prec) - ref) / ref < tol


@pytest.mark.parametrize("prec", ["f16s", "bf16s"])
def test_head_on_collision_mass_and_interface(prec):
    """Ratio-1 collision (the 16-bit target workload, 64^3 copy): per-colour mass
    drift in the 16-bit mode and interface position against FP64."""
    from paper_2309_07801_gb300 import cg
    wl = inputs.droplet_collision(64)
    fields = inputs.workload_fields(wl)
    out = {}
    for p in ("f64", prec):
        d = cg.Domain(cg.make_params(precision=p, **wl.params()))
        d.init(*fields)
        m0, _ = d.mass()
        d.step(1500)
        m1, flag = d.mass()
        assert flag == 0
        out[p] = (d.macros(), np.abs(m1 - m0) / m0)
    assert np.all(out[prec][1] < 5e-5), out[prec][1]
    phi_ref, phi = out["f64"][0]["phi"], out[prec][0]["phi"]
    iface = np.abs(phi_ref) < 0.9
    mismatch = (np.sign(phi) != np.sign(phi_ref)).sum() / iface.sum()
    assert mismatch < 0.1, mismatch



@pytest.mark.parametrize("prec,cen_tol,mass_tol", [("f16s", 0.01, 1e-4), ("bf16s", 0.5, 5e-3)])
def test_translating_droplet_64_with_samples(prec, cen_tol, mass_tol):
    """The ratio-10 translating droplet (64^3, Mach about 0.4 in the heavy
    phase) for 1000 steps, read back every 250 steps as the studies do: no
    non-finite density, the centroid within cen_tol cells of the FP32 run and
    the per-colour mass drift below mass_tol."""
    from paper_2309_07801_gb300 import studies
    ref = studies.translating(64, 1000, 250, "f32")["samples"]
    got = studies.translating(64, 1000, 250, prec)["samples"]
    assert len(got) == len(ref) == 5 and all(s["nonfinite"] == 0 for s in got)
    assert np.max(np.abs(np.array(got[-1]["centroid"]) - np.array(ref[-1]["centroid"]))) < cen_tol
    assert max(got[-1]["mass_drift"]) < mass_tol
