"""Shared helpers of the GPU parity tests: run the oracle and the CUDA path on
the same seeded inputs and compare."""
import numpy as np

# velocity scale below which a field is compared in absolute terms
U_FLOOR = 1e-3


def rel_err(a, ref, floor=0.0):
    """max |a - ref| / max(max |ref|, floor): the normwise relative error."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(float(np.abs(ref).max()), floor)
    return float(np.abs(a - ref).max() / scale) if scale > 0 else float(np.abs(a - ref).max())


def run_pair(params: dict, fields, steps, precision="f64", solid=None, oracle_steps=None, streaming=0):
    """Advance the oracle and the GPU domain from the same fields; return both.
    `streaming` selects the GPU population layout (the oracle has one)."""
    import oracle
    from paper_2309_07801_gb300 import cg
    rr, rb, u = fields
    od = oracle.Domain(oracle.make_params(**params))
    od.init(rr, rb, u, solid)
    od.step(steps if oracle_steps is None else oracle_steps)
    gd = cg.Domain(cg.make_params(precision=precision, streaming=streaming,
                                  solid_mask=1 if solid is not None else 0, **params))
    gd.init(rr, rb, u, solid)
    gd.step(steps)
    return od, gd


def compare_macros(od, gd):
    mo, mg = od.macros(), gd.macros()
    return {
        "rho_r": rel_err(mg["rho_r"], mo["rho_r"]),
        "rho_b": rel_err(mg["rho_b"], mo["rho_b"]),
        "p": rel_err(mg["p"], mo["p"]),
        "phi": rel_err(mg["phi"], mo["phi"], floor=1.0),
        "u": rel_err(mg["u"], mo["u"], floor=U_FLOOR),
        "u_abs": float(np.abs(mg["u"] - mo["u"]).max()),
        "rho_cellrel": cell_rel(mg["rho_r"] + mg["rho_b"], mo["rho_r"] + mo["rho_b"]),
    }


def cell_rel(a, ref):
    """max over cells with ref > 0 of |a - ref| / ref."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = ref > 0
    return float((np.abs(a - ref)[m] / ref[m]).max())


def compare_populations(od, gd):
    fro, fbo = od.populations()
    frg, fbg = gd.populations()
    return {"fr": rel_err(frg, fro), "fb": rel_err(fbg, fbo)}
