"""Helpers shared by the GPU parity tests (comparison only)."""
import numpy as np


def rel_err(gpu, ref, mask=None):
    g = np.asarray(gpu, np.float64)
    r = np.asarray(ref, np.float64)
    if mask is not None:
        g, r = g[mask], r[mask]
    if r.size == 0:
        return 0.0
    scale = max(np.max(np.abs(r)), 1e-300)
    return float(np.max(np.abs(g - r)) / scale)


def compare_state(sim, ora, fields=("rho", "u", "alpha", "mass", "conc")):
    """Per-field norm-relative errors of the GPU state against the oracle, on
    the cells that are liquid or interface in both."""
    tg = sim.fields(["flags"])["flags"]
    to = ora.types()
    both = ((tg == 1) | (tg == 2)) & ((to == 1) | (to == 2))
    got = sim.fields(list(fields))
    errs = {}
    for k in fields:
        ref = ora.get(k)
        m = both if ref.ndim == 1 else both
        errs[k] = rel_err(got[k], ref, m)
    return errs, int(np.sum(tg != to))
