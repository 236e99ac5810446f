"""Host-side diagnostics of the configuration studies (no GPU): centroid and
shape of a droplet in a periodic box, interface height of a phi column."""
import math

import numpy as np
import pytest

from paper_2309_07801_gb300 import studies


def _blob(shape_zyx, center_xyz, semi_xyz):
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = []
    for coord, c, n in ((x, center_xyz[0], nx), (y, center_xyz[1], ny), (z, center_xyz[2], nz)):
        d.append(((coord - c + n / 2.0) % n) - n / 2.0)  # minimum-image distance
    q = (d[0] / semi_xyz[0]) ** 2 + (d[1] / semi_xyz[1]) ** 2 + (d[2] / semi_xyz[2]) ** 2
    return np.exp(-q)


def test_centroid_of_a_symmetric_blob_and_shape_of_a_sphere():
    rho = _blob((36, 40, 32), (12.0, 25.0, 9.0), (3.0, 3.0, 3.0))
    cen, shape = studies.droplet_centroid_shape(rho)
    assert np.allclose(cen, (12.0, 25.0, 9.0), atol=1e-9)
    assert abs(shape) < 1e-9


def test_shape_of_an_ellipsoid():
    # second moments of exp(-(x/a)^2 - ...) scale as a^2: ratio (2a/a)^2 = 4
    rho = _blob((40, 40, 48), (24.0, 20.0, 20.0), (6.0, 3.0, 3.0))
    _, shape = studies.droplet_centroid_shape(rho)
    assert shape == pytest.approx(3.0, rel=1e-6)


def test_centroid_across_the_periodic_boundary_and_unwrapping():
    n = 32
    rho = _blob((n, n, n), (0.0, 16.0, 16.0), (3.0, 3.0, 3.0))  # straddles x = 0
    cen, _ = studies.droplet_centroid_shape(rho)
    assert min(cen[0], n - cen[0]) < 1e-9
    # a previous sample just right of the boundary unwraps the new one onto the
    # same branch instead of jumping by a box length
    cen2, _ = studies.droplet_centroid_shape(rho, prev=np.array([31.5, 16.0, 16.0]))
    assert cen2[0] == pytest.approx(32.0, abs=1e-9)


def test_interface_height_of_a_tanh_column():
    z = np.arange(64, dtype=np.float64)
    z0, w = 30.4, 4.0
    phi = np.tanh(2.0 * (z - z0) / w)
    # linear interpolation of tanh between its grid values: within 0.02 cells
    assert studies.interface_height(phi) == pytest.approx(z0, abs=0.02)
    assert math.isnan(studies.interface_height(np.ones(10)))
