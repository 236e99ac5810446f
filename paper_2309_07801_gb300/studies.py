"""Runs of the paper-shaped configurations and their diagnostics.

  translating droplet (Galilean invariance, Sec. IV.B as a periodic droplet):
      centroid of rho_r (per-axis circular mean, unwrapped in time) against
      u0 t, and shape distortion (ratio of the extreme principal second moments
      of rho_r about the centroid, minus 1);
  rising bubble (Sec. IV.D in 3D, z vertical): bubble centroid
      z_c = sum rho_b z / sum rho_b and velocity V_c = sum rho_b u_z / sum rho_b
      (the definitions of Sec. IV.D), per-colour mass drift;
  head-on droplet collision: per-colour mass drift and the fraction of
      interface cells whose phi has the other sign than in a reference run;
  Rayleigh-Taylor instability (Sec. IV.E): heights of the bubble, saddle and
      spike points of the phi = 0 surface against T = t / sqrt(W / g).

Everything here runs through the CUDA library; the CPU oracle is not used.
Centroids, shapes, masses and rise quantities are reduced on the device
(cg_reduce_diagnostics); only the interface comparisons read phi back.

    python -m paper_2309_07801_gb300.studies translating --edge 128 --steps 4000 --every 500
    python -m paper_2309_07801_gb300.studies bubble --steps 20000 --every 2000 --precisions f32,f64
    python -m paper_2309_07801_gb300.studies collision --edge 512 --steps 10000 --every 2000
    python -m paper_2309_07801_gb300.studies rti --edge 128 --steps 9600 --every 800 --model D
    python -m paper_2309_07801_gb300.studies rti --edge 64 --steps 6400 --every 800 --model C --re inf
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import cg, inputs


def _axis_coords(n):
    return np.arange(n, dtype=np.float64)


def droplet_centroid_shape(rho_r: np.ndarray, prev=None):
    """Centroid (x, y, z) and shape distortion of the red mass in a periodic box
    (arrays [z, y, x]); `prev` unwraps the centroid against an earlier sample."""
    nz, ny, nx = rho_r.shape
    total = rho_r.sum()
    cen = np.empty(3)
    for a, (axis, n) in enumerate(((2, nx), (1, ny), (0, nz))):
        marg = rho_r.sum(axis=tuple(i for i in range(3) if i != axis)) / total
        th = 2.0 * math.pi * _axis_coords(n) / n
        ang = math.atan2(float(np.dot(marg, np.sin(th))), float(np.dot(marg, np.cos(th))))
        cen[a] = (ang % (2.0 * math.pi)) * n / (2.0 * math.pi)
    if prev is not None:
        size = np.array([nx, ny, nz], dtype=np.float64)
        cen = prev + ((cen - prev + size / 2.0) % size - size / 2.0)
    # second moments about the centroid, minimum-image distances
    d = []
    for a, n in enumerate((nx, ny, nz)):
        d.append(((_axis_coords(n) - cen[a] + n / 2.0) % n) - n / 2.0)
    w = rho_r / total
    dx, dy, dz = d[0][None, None, :], d[1][None, :, None], d[2][:, None, None]
    m = np.empty((3, 3))
    comps = (dx, dy, dz)
    for a in range(3):
        for b in range(a, 3):
            m[a, b] = m[b, a] = float((w * comps[a] * comps[b]).sum())
    ev = np.linalg.eigvalsh(m)
    return cen, float(ev[-1] / ev[0] - 1.0)


def shape_distortion(m6) -> float:
    """Ratio of the extreme principal second moments minus 1, from the six
    moments (xx, yy, zz, xy, xz, yz)."""
    xx, yy, zz, xy, xz, yz = m6
    ev = np.linalg.eigvalsh(np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]))
    return float(ev[-1] / ev[0] - 1.0)


def unwrap(cen, prev, size):
    """Periodic centroid continued from an earlier sample (nearest image)."""
    if prev is None:
        return cen
    size = np.asarray(size, dtype=np.float64)
    return prev + ((cen - prev + size / 2.0) % size - size / 2.0)


def bubble_rise(m: dict):
    """z_c and V_c of Sec. IV.D (z vertical), weights rho_b."""
    rb = m["rho_b"]
    wsum = rb.sum()
    z = np.arange(rb.shape[0], dtype=np.float64)[:, None, None]
    return float((rb * z).sum() / wsum), float((rb * m["u"][2]).sum() / wsum)


def interface_mismatch(phi: np.ndarray, phi_ref: np.ndarray) -> float:
    """Cells where sign(phi) differs from the reference, over the reference's
    interface cells (|phi| < 0.9)."""
    band = int((np.abs(phi_ref) < 0.9).sum())
    return float((np.sign(phi) != np.sign(phi_ref)).sum()) / max(1, band)


def run_series(wl, fields, precision, steps, every, on_sample):
    """Advance a domain in chunks of `every` steps; call on_sample(step, dom)."""
    import torch
    d = cg.Domain(cg.make_params(precision=precision, **wl.params()))
    d.init(*fields)
    out = [on_sample(0, d)]
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        d.step(k)
        done += k
        mass, flag = d.mass()
        if flag:  # a diverged run: record where and stop
            out.append({"step": done, "nonfinite": 1})
            break
        out.append(on_sample(done, d))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    d.close()
    return out, wall


def translating(edge=128, steps=4000, every=500, precision="f32"):
    wl = inputs.translating_droplet(edge)
    fields = inputs.workload_fields(wl)
    state = {"prev": None, "m0": None}

    def sample(step, d):
        # reduced on the device: centroid (circular means) and second moments
        dg = d.diagnostics()
        cen = unwrap(dg["centroid"][0], state["prev"], (wl.nx, wl.ny, wl.nz))
        shape = shape_distortion(dg["second_moment"])
        state["prev"] = cen
        mass, flag = dg["mass"], dg["nonfinite"]
        if state["m0"] is None:
            state["m0"] = mass
        c0 = np.array([wl.nx / 2.0, wl.ny / 2.0, wl.nz / 2.0])
        expect = c0 + np.array([0.05, 0.05, 0.0]) * step
        return {"step": step, "centroid": cen.tolist(), "expected": expect.tolist(),
                "drift": (cen - expect).tolist(), "shape": shape,
                "mass_drift": (np.abs(mass - state["m0"]) / state["m0"]).tolist(), "nonfinite": flag}

    rows, wall = run_series(wl, fields, precision, steps, every, sample)
    return {"study": "translating", "edge": edge, "precision": precision, "steps": steps,
            "wall_s": wall, "samples": rows}


def bubble(steps=20000, every=2000, precision="f32", nx=192, ny=192, nz=384, case="config"):
    """case "config": the configured ratio-1000 bubble (sigma 0.01, g 1e-6);
    "case2": the dimensionless numbers of the paper's case 2 (inputs.rising_bubble_case2)."""
    wl = inputs.rising_bubble(nx, ny, nz) if case == "config" else inputs.rising_bubble_case2(nx, ny, nz)
    fields = inputs.workload_fields(wl)
    state = {"m0": None}

    def sample(step, d):
        # z_c = sum rho_b z / sum rho_b (z a wall axis), V_c = sum rho_b u_z / sum rho_b
        dg = d.diagnostics()
        zc, vc = float(dg["centroid"][1][2]), float(dg["momentum"][1][2] / dg["mass"][1])
        mass, flag = dg["mass"], dg["nonfinite"]
        if state["m0"] is None:
            state["m0"] = mass
        return {"step": step, "z_c": zc, "V_c": vc,
                "mass_drift": (np.abs(mass - state["m0"]) / state["m0"]).tolist(), "nonfinite": flag}

    rows, wall = run_series(wl, fields, precision, steps, every, sample)
    return {"study": "bubble", "case": case, "shape": [nx, ny, nz], "precision": precision, "steps": steps,
            "wall_s": wall, "samples": rows}


def interface_height(phi_col: np.ndarray) -> float:
    """z where phi crosses 0 along a vertical line (heavy fluid, phi > 0, above);
    the crossing closest to the middle, linear interpolation."""
    s = np.sign(phi_col)
    idx = np.nonzero(s[:-1] * s[1:] < 0)[0]
    if len(idx) == 0:
        return float("nan")
    mid = (len(phi_col) - 1) / 2.0
    k = idx[np.argmin(np.abs(idx - mid))]
    a, b = phi_col[k], phi_col[k + 1]
    return float(k + a / (a - b))


def rti(W=128, steps=None, every=None, precision="f32", model=3, Re=1024.0):
    """Rayleigh-Taylor instability (Sec. IV.E): heights of the bubble (x = y = 0),
    saddle (x = 0, y = W/2) and spike (x = y = W/2) relative to the initial
    mid-plane, in units of W, against T = t / sqrt(W / g)."""
    wl = inputs.rayleigh_taylor(W, Re, model)
    fields = inputs.workload_fields(wl)
    g = -wl.g[2]
    t_unit = math.sqrt(W / g)
    steps = wl.steps if steps is None else steps
    every = int(round(0.25 * t_unit)) if every is None else every
    z_mid = (wl.nz - 1) / 2.0
    points = {"bubble": (0, 0), "saddle": (0, W // 2), "spike": (W // 2, W // 2)}

    def sample(step, d):
        m = d.macros()
        mass, flag = d.mass()
        row = {"step": step, "T": step / t_unit, "nonfinite": flag}
        for name, (x, y) in points.items():
            row[name] = (interface_height(m["phi"][:, y, x]) - z_mid) / W
        return row

    rows, wall = run_series(wl, fields, precision, steps, every, sample)
    return {"study": "rti", "W": W, "Re": Re, "model": "ABCD"[model], "precision": precision, "steps": steps,
            "wall_s": wall, "MLUPS": wl.cells * steps / wall / 1e6, "samples": rows}


def collision(edge=512, steps=10000, every=2000, precisions=("f64", "f32", "f16s", "bf16s")):
    """All precisions side by side; the first one is the reference for phi."""
    wl = inputs.droplet_collision(edge)
    fields = inputs.workload_fields(wl)
    phis = {}
    out = []
    for prec in precisions:
        state = {"m0": None}
        ref = phis.get(precisions[0])

        def sample(step, d, prec=prec, state=state):
            m = d.macros()
            mass, flag = d.mass()
            if state["m0"] is None:
                state["m0"] = mass
            row = {"step": step, "mass_drift": (np.abs(mass - state["m0"]) / state["m0"]).tolist(),
                   "nonfinite": flag}
            if prec == precisions[0]:
                phis.setdefault(prec, {})[step] = m["phi"].astype(np.float32)
            elif ref is not None and step in ref:
                row["interface_mismatch_vs_" + precisions[0]] = interface_mismatch(m["phi"], ref[step])
            return row

        rows, wall = run_series(wl, fields, prec, steps, every, sample)
        out.append({"study": "collision", "edge": edge, "precision": prec, "steps": steps,
                    "wall_s": wall, "MLUPS": wl.cells * steps / wall / 1e6, "samples": rows})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["translating", "bubble", "collision", "rti"])
    ap.add_argument("--model", default="D", choices=["A", "B", "C", "D"])
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--every", type=int, default=500)
    ap.add_argument("--precisions", default="f32")
    ap.add_argument("--case", default="config", choices=["config", "case2"])
    ap.add_argument("--re", type=float, default=1024.0, help="Reynolds number of the RTI (inf: nu = 0)")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    precs = args.precisions.split(",")
    if args.study == "translating":
        for p in precs:
            print(json.dumps(translating(args.edge, args.steps, args.every, p)), flush=True)
    elif args.study == "bubble":
        for p in precs:
            print(json.dumps(bubble(args.steps, args.every, p, case=args.case)), flush=True)
    elif args.study == "rti":
        for p in precs:
            print(json.dumps(rti(args.edge, args.steps, args.every, p, "ABCD".index(args.model), args.re)),
                  flush=True)
    else:
        for r in collision(args.edge, args.steps, args.every, tuple(precs)):
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    sys.exit(main())
