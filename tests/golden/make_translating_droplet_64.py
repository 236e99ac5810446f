"""Write translating_droplet_64_oracle.txt: the FP64 oracle run of the
translating droplet, 64^3 copy (R = 10, ratio 10, nu = 0.05, sigma = 0.005,
beta = 0.7, u0 = (0.05, 0.05, 0)), sampled every 500 steps up to 4000.

Recorded per sample: the red-mass centroid (per-axis circular mean of rho_r,
unwrapped over time), the shape distortion (ratio of the largest to the
smallest principal second moment of rho_r about the centroid, minus 1) and the
per-colour masses.  Only the oracle is called; the centroid and shape are
computed here, independently of the code that analyses the GPU runs.

    python tests/golden/make_translating_droplet_64.py     (about 20 CPU-minutes on 8 cores)
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2309_07801_gb300 import inputs  # noqa: E402

STEPS, EVERY = 4000, 500


def centroid_and_shape(rho_r, prev=None):
    n = rho_r.shape[0]
    w = rho_r / rho_r.sum()
    cen = []
    for axis in (2, 1, 0):  # x, y, z
        ang = 2.0 * math.pi * np.arange(n) / n
        shape = [1, 1, 1]
        shape[axis] = n
        cs = float((w * np.cos(ang).reshape(shape)).sum())
        sn = float((w * np.sin(ang).reshape(shape)).sum())
        cen.append((math.atan2(sn, cs) % (2.0 * math.pi)) * n / (2.0 * math.pi))
    cen = np.array(cen)
    if prev is not None:  # unwrap against the previous sample
        cen = prev + ((cen - prev + n / 2.0) % n - n / 2.0)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = [((c - cen[a] + n / 2.0) % n) - n / 2.0 for a, c in enumerate((x, y, z))]
    m2 = np.array([[float((w * d[a] * d[b]).sum()) for b in range(3)] for a in range(3)])
    ev = np.linalg.eigvalsh(m2)
    return cen, float(ev[-1] / ev[0] - 1.0)


def main():
    oracle.build()
    wl = inputs.translating_droplet(64)
    dom = oracle.Domain(oracle.make_params(**wl.params()))
    dom.init(*inputs.workload_fields(wl))
    rows = []
    prev = None
    for s in range(0, STEPS + 1, EVERY):
        if s:
            dom.step(EVERY)
        m = dom.macros()
        prev, shape = centroid_and_shape(m["rho_r"], prev)
        mass = dom.mass()
        rows.append((s, prev[0], prev[1], prev[2], shape, mass[0], mass[1]))
        print(rows[-1], flush=True)
    with open(os.path.join(HERE, "translating_droplet_64_oracle.txt"), "w") as fh:
        fh.write("# FP64 oracle, translating droplet 64^3 copy (R=10, ratio 10, nu=0.05, sigma=0.005, beta=0.7,\n"
                 "# u0=(0.05,0.05,0), Model D with Q), written by make_translating_droplet_64.py.\n"
                 "# columns: step centroid_x centroid_y centroid_z shape_distortion mass_red mass_blue\n")
        for r in rows:
            fh.write("%d %.10f %.10f %.10f %.10e %.12e %.12e\n" % r)


if __name__ == "__main__":
    main()
