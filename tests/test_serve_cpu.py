"""Host form of the server's per-run summary (no GPU): the pressure jump and
largest speed from the squared-radius grid equal the direct definition with a
full coordinate grid and square roots (the server itself reduces the same
quantities on the device; tests/test_gpu_diagnostics.py checks those)."""
import numpy as np
import pytest

from paper_2309_07801_gb300 import serve


def _direct(n, radius, p, u):
    c = n / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    inner, outer = r < 0.5 * radius, r > radius + 0.25 * n
    return float(p[inner].mean() - p[outer].mean()), float(np.sqrt((u ** 2).sum(axis=0)).max())


@pytest.mark.parametrize("n,frac", [(32, 0.2), (48, 0.35), (64, 0.27), (33, 0.3)])
def test_summary_diagnostics_match_the_direct_definition(n, frac):
    rng = np.random.default_rng(n)
    p = rng.normal(size=(n, n, n))
    u = rng.normal(size=(3, n, n, n))
    radius = frac * n
    dp, umax = serve.diagnostics(n, radius, p.reshape(-1), u.reshape(-1))
    dp0, umax0 = _direct(n, radius, p, u)
    assert dp == pytest.approx(dp0, rel=1e-12, abs=1e-14) and umax == pytest.approx(umax0, rel=1e-15)
