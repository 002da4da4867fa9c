"""Collapsed Gauss-Legendre volume and face rules (Sec. 2, Duffy transform).

Volume: n = N+1 Gauss-Legendre points in each collapsed coordinate (a, b, c);
the weight of point (a_i, b_j, c_k) is w_i w_j w_k det(d(xi,eta,zeta)/d(a,b,c)),
i.e. the Duffy Jacobian (1-b)/2 (prism), ((1-b)/2)((1-c)/2)^2 (tet) or
((1-c)/2)^2 (pyramid).

Faces: a quadrilateral face carries the n x n Gauss-Legendre tensor rule in its
own parameters (s, t); a triangular face the n x n collapsed rule
s = (1+alpha)(1-beta)/2 - 1, t = beta with weight w_i w_j (1-beta_j)/2.  The
face parametrisation is the local vertex order of elements.FACES.

Parity: pinned by exact integration of monomials against closed forms
(tests/test_oracle_quadrature.py).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss

from .elements import FACES, REF_VERTS, collapse_jacobian, uncollapse


def gauss_legendre(n):
    return leggauss(n)


def volume_rule(etype, N):
    """Points [n^3, 3] in reference coordinates and weights [n^3]."""
    x, w = gauss_legendre(N + 1)
    A, B, C = np.meshgrid(x, x, x, indexing="ij")
    WA, WB, WC = np.meshgrid(w, w, w, indexing="ij")
    a, b, c = A.ravel(), B.ravel(), C.ravel()
    det = np.linalg.det(collapse_jacobian(etype, a, b, c))
    xi, eta, zeta = uncollapse(etype, a, b, c)
    return np.stack([xi, eta, zeta], axis=1), (WA * WB * WC).ravel() * det


def face_param_rule(nverts, N):
    """(s, t) points [n^2, 2] and weights [n^2] on the face's parameter domain."""
    x, w = gauss_legendre(N + 1)
    S, T = np.meshgrid(x, x, indexing="ij")
    WS, WT = np.meshgrid(w, w, indexing="ij")
    if nverts == 4:
        return np.stack([S.ravel(), T.ravel()], axis=1), (WS * WT).ravel()
    al, be = S.ravel(), T.ravel()
    s = (1 + al) * (1 - be) / 2 - 1
    return np.stack([s, be], axis=1), (WS * WT).ravel() * (1 - be) / 2


def face_map(corners, st):
    """x(s, t) = c0 + (s+1)/2 (c1-c0) + (t+1)/2 (c2-c0) for corners [k, 3]."""
    c0, c1, c2 = corners[0], corners[1], corners[2]
    return c0 + 0.5 * (st[:, :1] + 1) * (c1 - c0) + 0.5 * (st[:, 1:2] + 1) * (c2 - c0)


def face_rule(etype, lf, N):
    """Reference-element points [n^2, 3] of local face lf, parameter weights [n^2],
    and the reference tangents d xi/ds, d xi/dt."""
    fv = FACES[etype][lf]
    corners = REF_VERTS[etype][fv]
    st, w = face_param_rule(len(fv), N)
    pts = face_map(corners, st)
    ts = 0.5 * (corners[1] - corners[0])
    tt = 0.5 * (corners[2] - corners[0])
    return pts, w, ts, tt
