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


# Amplitude of the seeded TGV perturbation in the full-size parity checks.  At
# amplitude 1e-2 (Ma 0.1, p0 = 71) the residual of the fine meshes is a
# cancellation of terms up to 100x larger, and two correct evaluations in
# different orders differ by up to 4e-11 of max|R| (see ulp_sensitivity); at
# 0.1 the residual is 10x larger against the same terms.
FULL_SIZE_AMP = 0.1


def assert_sampled_parity(R, Rref, vidx, mask, tol=TOL, volume=None, label=""):
    """Per variable v: max|R - Rref| / max|Rref| over the masked entries
    (the plain normwise metric) below tol[v] (or tol).  The failure message
    also gives the error relative to the volume-term magnitude when `volume`
    (a callable returning the volume term in residual units, full length) is
    given."""
    tols = np.broadcast_to(np.asarray(tol, dtype=np.float64), (5,))
    bad = []
    for v in range(5):
        i = vidx[v][mask[vidx[v]]]
        if i.size == 0:
            continue
        err = np.abs(R[i] - Rref[i]).max()
        plain = err / np.abs(Rref[i]).max()
        if not plain < tols[v]:
            bad.append((v, i, err, plain))
    if bad:
        vol = volume() if volume is not None else None
        msg = []
        for v, i, err, plain in bad:
            rel = err / max(np.abs(Rref[i]).max(), np.abs(vol[i]).max()) if vol is not None else float("nan")
            msg.append(f"var {v}: plain {plain:.3e} (tol {tols[v]:.1e}), against max(|R|, |vol|) {rel:.3e}")
        raise AssertionError(f"{label} " + "; ".join(msg))


def ulp_sensitivity(residual, Q, vidx, mask, seed=0):
    """How far the residual moves, per variable and relative to its maximum,
    when every input coefficient moves by one ulp in a seeded random
    direction: residual(Q) against residual(nextafter(Q, +-inf)).  Two
    correct evaluations of the same residual in different orders differ by
    a small multiple of this (each is the exact residual of an input a few
    ulps away, plus output rounding)."""
    rng = np.random.default_rng(seed)
    up = rng.integers(0, 2, size=Q.size).astype(bool)
    Qp = np.where(up, np.nextafter(Q, np.inf), np.nextafter(Q, -np.inf))
    R0, R1 = residual(Q), residual(Qp)
    out = np.zeros(5)
    for v in range(5):
        i = vidx[v][mask[vidx[v]]]
        out[v] = np.abs(R1[i] - R0[i]).max() / np.abs(R0[i]).max()
    return out
