"""Reference elements, collapsed coordinates and orthonormal modal bases.

Sec. 2 of the paper maps each polytopal reference element onto the unit
hexahedron by a Duffy (collapsed-coordinate) transform and uses element-local
polynomial test functions up to degree N.  The paper does not spell out the
modal space; this oracle takes the standard orthonormal choices:
  hex     Q_N         phi = L_p(a) L_q(b) L_r(c)
  prism   P_N x P_N   phi = L_p(a) ((1-b)/2)^p J_q^(2p+1)(b) L_r(c),         p+q<=N
  tet     P_N         phi = L_p(a) ((1-b)/2)^p J_q^(2p+1)(b)
                              ((1-c)/2)^(p+q) J_r^(2p+2q+2)(c),             p+q+r<=N
  pyramid             phi = L_p(a) L_q(b) ((1-c)/2)^m J_r^(2m+2)(c),
                              m = max(p, q), p,q <= N, r <= N - m
with J_n^(alpha) the Jacobi polynomial P_n^(alpha,0) scaled so that
int_{-1}^{1} ((1-x)/2)^alpha J_n^2 dx = 1, and L_n = J_n^(0).  Mode order is
lexicographic in (p, q, r) with r fastest.

Parity: pinned by orthonormality under an exact rule, reproduction of the
polynomial spaces, finite-difference gradients and the divergence theorem
(tests/test_oracle_basis.py).  The choice of space itself is a reading of the
paper (parity unpinned against the paper's own solver).
"""
from __future__ import annotations

import numpy as np

HEX, PRISM, PYR, TET = 0, 1, 2, 3
NAMES = ("hex", "prism", "pyramid", "tet")

# Reference vertices.  hex: lexicographic, x fastest.  prism: triangle
# {xi,eta>=-1, xi+eta<=0} at zeta=-1 then at zeta=+1.  pyramid: base square at
# zeta=-1 (lexicographic), apex (-1,-1,1).  tet: origin corner then unit axes.
REF_VERTS = {
    HEX: np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1],
                   [-1, -1, 1], [1, -1, 1], [-1, 1, 1], [1, 1, 1]], dtype=float),
    PRISM: np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [-1, 1, 1]], dtype=float),
    PYR: np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1], [-1, -1, 1]], dtype=float),
    TET: np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float),
}

# Local faces as ordered local-vertex lists.  A face with vertices (c0, c1, c2[, c3])
# is parametrised by x(s, t) = c0 + (s+1)/2 (c1-c0) + (t+1)/2 (c2-c0) over
# [-1,1]^2 (quadrilateral) or over {s,t>=-1, s+t<=0} (triangle).
FACES = {
    HEX: [[0, 1, 2, 3], [4, 5, 6, 7], [0, 1, 4, 5], [2, 3, 6, 7], [0, 2, 4, 6], [1, 3, 5, 7]],
    PRISM: [[0, 1, 2], [3, 4, 5], [0, 1, 3, 4], [0, 2, 3, 5], [1, 2, 4, 5]],
    PYR: [[0, 1, 2, 3], [0, 1, 4], [0, 2, 4], [1, 3, 4], [2, 3, 4]],
    TET: [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]],
}

REF_VOLUME = {HEX: 8.0, PRISM: 4.0, PYR: 8.0 / 3.0, TET: 4.0 / 3.0}


def modes(etype: int, N: int):
    """Mode triples (p, q, r), lexicographic with r fastest."""
    out = []
    for p in range(N + 1):
        qmax = N - p if etype in (PRISM, TET) else N
        for q in range(qmax + 1):
            if etype in (HEX, PRISM):
                rmax = N
            elif etype == TET:
                rmax = N - p - q
            else:
                rmax = N - max(p, q)
            for r in range(rmax + 1):
                out.append((p, q, r))
    return out


def n_modes(etype: int, N: int) -> int:
    return len(modes(etype, N))


# ---------------------------------------------------------------- collapse

def collapse(etype, xi, eta, zeta):
    """Reference (xi, eta, zeta) -> collapsed (a, b, c) on [-1, 1]^3."""
    xi, eta, zeta = (np.asarray(v, dtype=float) for v in (xi, eta, zeta))
    if etype == HEX:
        return xi, eta, zeta
    if etype == PRISM:
        return 2.0 * (1.0 + xi) / (1.0 - eta) - 1.0, eta, zeta
    if etype == TET:
        return (2.0 * (1.0 + xi) / (-eta - zeta) - 1.0,
                2.0 * (1.0 + eta) / (1.0 - zeta) - 1.0, zeta)
    if etype == PYR:
        return (2.0 * (1.0 + xi) / (1.0 - zeta) - 1.0,
                2.0 * (1.0 + eta) / (1.0 - zeta) - 1.0, zeta)
    raise ValueError(etype)


def uncollapse(etype, a, b, c):
    """Collapsed (a, b, c) -> reference (xi, eta, zeta)."""
    a, b, c = (np.asarray(v, dtype=float) for v in (a, b, c))
    if etype == HEX:
        return a, b, c
    if etype == PRISM:
        return (1 + a) * (1 - b) / 2 - 1, b, c
    if etype == TET:
        return (1 + a) * (1 - b) * (1 - c) / 4 - 1, (1 + b) * (1 - c) / 2 - 1, c
    if etype == PYR:
        return (1 + a) * (1 - c) / 2 - 1, (1 + b) * (1 - c) / 2 - 1, c
    raise ValueError(etype)


def collapse_jacobian(etype, a, b, c):
    """d(xi, eta, zeta)/d(a, b, c) per point, shape [..., 3, 3] (row = xi_k)."""
    a, b, c = (np.asarray(v, dtype=float) for v in (a, b, c))
    J = np.zeros(a.shape + (3, 3))
    if etype == HEX:
        J[..., 0, 0] = J[..., 1, 1] = J[..., 2, 2] = 1.0
    elif etype == PRISM:
        J[..., 0, 0] = (1 - b) / 2
        J[..., 0, 1] = -(1 + a) / 2
        J[..., 1, 1] = 1.0
        J[..., 2, 2] = 1.0
    elif etype == TET:
        J[..., 0, 0] = (1 - b) * (1 - c) / 4
        J[..., 0, 1] = -(1 + a) * (1 - c) / 4
        J[..., 0, 2] = -(1 + a) * (1 - b) / 4
        J[..., 1, 1] = (1 - c) / 2
        J[..., 1, 2] = -(1 + b) / 2
        J[..., 2, 2] = 1.0
    elif etype == PYR:
        J[..., 0, 0] = (1 - c) / 2
        J[..., 0, 2] = -(1 + a) / 2
        J[..., 1, 1] = (1 - c) / 2
        J[..., 1, 2] = -(1 + b) / 2
        J[..., 2, 2] = 1.0
    else:
        raise ValueError(etype)
    return J


# ---------------------------------------------------------------- 1D factors

def jacobi(n, alpha, beta, x):
    """Jacobi polynomial P_n^(alpha,beta)(x) by its three-term recurrence
    (Abramowitz & Stegun 22.7.1); accurate to a few ulps on [-1, 1], unlike
    hypergeometric-series evaluation for large alpha."""
    x = np.asarray(x, dtype=float)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    a, b = float(alpha), float(beta)
    p1 = 0.5 * (a - b + (a + b + 2.0) * x)
    for k in range(2, n + 1):
        s = 2.0 * k + a + b
        c1 = 2.0 * k * (k + a + b) * (s - 2.0)
        c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b)
        c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s
        p0, p1 = p1, (c2 * p1 - c3 * p0) / c1
    return p1


def jhat(n, alpha, x):
    """Jacobi P_n^(alpha,0) normalised: int ((1-x)/2)^alpha jhat^2 dx = 1."""
    return jacobi(n, alpha, 0.0, x) * np.sqrt((2 * n + alpha + 1) / 2.0)


def jhat_d(n, alpha, x):
    """Derivative of jhat: d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)."""
    if n == 0:
        return np.zeros_like(np.asarray(x, dtype=float))
    return 0.5 * (n + alpha + 1) * jacobi(n - 1, alpha + 1, 1.0, x) * np.sqrt((2 * n + alpha + 1) / 2.0)


def _warped(k, n, alpha, x):
    """g(x) = ((1-x)/2)^k jhat_n^alpha(x) and g'(x)."""
    x = np.asarray(x, dtype=float)
    h = (1.0 - x) / 2.0
    P, dP = jhat(n, alpha, x), jhat_d(n, alpha, x)
    g = h ** k * P
    dg = h ** k * dP
    if k > 0:
        dg = dg - 0.5 * k * h ** (k - 1) * P
    return g, dg


def _factors(etype, p, q, r, a, b, c):
    """1D factors (fa, fb, fc) and derivatives of mode (p, q, r)."""
    fa, da = _warped(0, p, 0, a)
    if etype in (HEX, PYR):
        fb, db = _warped(0, q, 0, b)
    else:
        fb, db = _warped(p, q, 2 * p + 1, b)
    if etype in (HEX, PRISM):
        fc, dc = _warped(0, r, 0, c)
    elif etype == TET:
        fc, dc = _warped(p + q, r, 2 * p + 2 * q + 2, c)
    else:
        m = max(p, q)
        fc, dc = _warped(m, r, 2 * m + 2, c)
    return fa, fb, fc, da, db, dc


def eval_basis_abc(etype, N, a, b, c, grad=False):
    """phi at collapsed points: [npts, nM]; with grad also d phi/d(a,b,c): [3, npts, nM]."""
    a, b, c = (np.atleast_1d(np.asarray(v, dtype=float)) for v in (a, b, c))
    ml = modes(etype, N)
    phi = np.empty((a.size, len(ml)))
    dabc = np.empty((3, a.size, len(ml))) if grad else None
    for i, (p, q, r) in enumerate(ml):
        fa, fb, fc, da, db, dc = _factors(etype, p, q, r, a, b, c)
        phi[:, i] = fa * fb * fc
        if grad:
            dabc[0, :, i] = da * fb * fc
            dabc[1, :, i] = fa * db * fc
            dabc[2, :, i] = fa * fb * dc
    return (phi, dabc) if grad else phi


def eval_basis(etype, N, pts, grad=False):
    """phi at reference points pts [npts, 3]; with grad, grad_xi phi [3, npts, nM]
    by the chain rule through the collapse: grad_xi = Jc^{-T} grad_abc."""
    pts = np.atleast_2d(np.asarray(pts, dtype=float))
    a, b, c = collapse(etype, pts[:, 0], pts[:, 1], pts[:, 2])
    if not grad:
        return eval_basis_abc(etype, N, a, b, c)
    phi, dabc = eval_basis_abc(etype, N, a, b, c, grad=True)
    Jc = collapse_jacobian(etype, a, b, c)              # [npts, 3(xi), 3(abc)]
    # grad_abc phi = Jc^T grad_xi phi  ->  grad_xi = solve(Jc^T, grad_abc)
    JT = np.transpose(Jc, (0, 2, 1))
    g = np.linalg.solve(JT, np.transpose(dabc, (1, 0, 2)))  # [npts, 3, nM]
    return phi, np.transpose(g, (1, 0, 2))
