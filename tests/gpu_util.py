"""Helpers shared by the GPU parity tests."""
import numpy as np

import dg_inputs as di

# Parity bar: per variable, max |gpu - oracle| / max |oracle| <= 1e-11 (relative
# L-infinity, normwise per variable; pointwise ratios are meaningless where the
# residual vanishes).
TOL = 1e-11


def var_index(nM_per_elem):
    """Index arrays selecting variable v's coefficients in caller layout."""
    idx = [[] for _ in range(5)]
    off = 0
    for nm in nM_per_elem:
        for v in range(5):
            idx[v].append(np.arange(off + v * nm, off + (v + 1) * nm))
        off += 5 * nm
    return [np.concatenate(i) for i in idx]


def rel_err(a, b, vidx, mask=None):
    """max over variables of max|a-b| / max|b| (restricted to mask if given)."""
    worst = 0.0
    for v in range(5):
        i = vidx[v] if mask is None else vidx[v][mask[vidx[v]]]
        if i.size == 0:
            continue
        den = np.abs(b[i]).max()
        worst = max(worst, np.abs(a[i] - b[i]).max() / den if den > 0 else np.abs(a[i]).max())
    return worst


def make_box(kind, m, seed=1, reorder=None):
    box = di.box_mesh(m, kind, seed=seed)
    if reorder is not None:
        box = di.reorder_vertices(box, seed=reorder)
    return box
