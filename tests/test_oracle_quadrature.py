"""Pins of the oracle's collapsed Gauss-Legendre rules (Sec. 2, Duffy transform)
against closed-form monomial integrals over each reference element.

Closed forms, with x = (xi+1)/2, y = (eta+1)/2, z = (zeta+1)/2:
  hex      int xi^a eta^b zeta^c        = prod (1 + (-1)^k)/(k + 1)
  tet      int x^a y^b z^c              = 8 a! b! c! / (a+b+c+3)!   (Dirichlet)
  prism    int x^a y^b zeta^c           = 4 a! b!/(a+b+2)! (1+(-1)^c)/(c+1)
  pyramid  int x^a y^b z^c              = 8 c! (a+b+2)! / ((a+1)(b+1)(a+b+c+3)!)
Exactness degrees with n = N+1 points per direction: hex 2N+1 per direction,
prism 2N in (xi, eta) and 2N+1 in zeta, tet and pyramid 2N-1 in total degree.
"""
import itertools
from math import factorial

import numpy as np
import pytest

from oracle.elements import HEX, PRISM, PYR, TET, REF_VOLUME, FACES, REF_VERTS
from oracle.quadrature import volume_rule, face_rule, gauss_legendre


def exact(etype, a, b, c):
    if etype == HEX:
        f = lambda k: (1 + (-1) ** k) / (k + 1)
        return f(a) * f(b) * f(c)
    if etype == TET:
        return 8.0 * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
    if etype == PRISM:
        return 4.0 * factorial(a) * factorial(b) / factorial(a + b + 2) * (1 + (-1) ** c) / (c + 1)
    if etype == PYR:
        return 8.0 * factorial(c) * factorial(a + b + 2) / ((a + 1) * (b + 1) * factorial(a + b + c + 3))
    raise ValueError


def integrand(etype, pts, a, b, c):
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    if etype == HEX:
        return xi ** a * eta ** b * zeta ** c
    if etype == PRISM:
        return ((xi + 1) / 2) ** a * ((eta + 1) / 2) ** b * zeta ** c
    return ((xi + 1) / 2) ** a * ((eta + 1) / 2) ** b * ((zeta + 1) / 2) ** c


def exact_set(etype, N):
    for a, b, c in itertools.product(range(2 * N + 2), repeat=3):
        if etype == HEX:
            yield a, b, c
        elif etype == PRISM and a + b <= 2 * N:
            yield a, b, c
        elif etype in (TET, PYR) and a + b + c <= 2 * N - 1:
            yield a, b, c


@pytest.mark.parametrize("etype", [HEX, PRISM, PYR, TET])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_volume_rule_exact(etype, N):
    pts, w = volume_rule(etype, N)
    assert pts.shape == ((N + 1) ** 3, 3)
    assert abs(w.sum() - REF_VOLUME[etype]) < 1e-14 * REF_VOLUME[etype]
    worst = 0.0
    for a, b, c in exact_set(etype, N):
        f = integrand(etype, pts, a, b, c)
        got = w @ f
        ref = exact(etype, a, b, c)
        worst = max(worst, abs(got - ref) / (np.abs(w) @ np.abs(f)))
    assert worst < 1e-13


@pytest.mark.parametrize("etype", [PRISM, PYR, TET])
def test_volume_rule_not_exact_beyond(etype):
    """Sanity that the pin has teeth: one degree beyond the stated exactness fails."""
    N = 2
    pts, w = volume_rule(etype, N)
    a, b, c = (0, 0, 2 * N) if etype in (TET, PYR) else (2 * N + 1, 0, 0)
    got = w @ integrand(etype, pts, a, b, c)
    assert abs(got - exact(etype, a, b, c)) > 1e-8


def test_gauss_legendre_closed_form():
    x, w = gauss_legendre(2)
    assert np.allclose(np.sort(x), [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    x, w = gauss_legendre(3)
    assert np.allclose(np.sort(x), [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w[np.argsort(x)], [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("etype", [HEX, PRISM, PYR, TET])
def test_face_rules_area_and_points(etype):
    """Face weights sum to the reference face area; the points lie on the face plane."""
    N = 3
    for lf, fv in enumerate(FACES[etype]):
        pts, w, ts, tt = face_rule(etype, lf, N)
        S = np.linalg.norm(np.cross(ts, tt))
        C = REF_VERTS[etype][fv]
        if len(fv) == 4:
            area = np.linalg.norm(np.cross(C[1] - C[0], C[2] - C[0]))
        else:
            area = 0.5 * np.linalg.norm(np.cross(C[1] - C[0], C[2] - C[0]))
        assert abs((w * S).sum() - area) < 1e-13
        nrm = np.cross(C[1] - C[0], C[2] - C[0])
        assert np.abs((pts - C[0]) @ nrm).max() < 1e-13
