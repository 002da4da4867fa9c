"""Pins of the oracle's orthonormal modal bases (reading of Sec. 2's test
functions): dimension, orthonormality under an exact rule, reproduction of the
polynomial space, finite-difference gradients, and the divergence theorem on
each reference element (which also pins the face parametrisations)."""
import itertools

import numpy as np
import pytest

from oracle.elements import (HEX, PRISM, PYR, TET, FACES, REF_VERTS, REF_VOLUME,
                             eval_basis, n_modes, collapse, uncollapse)
from oracle.quadrature import volume_rule, face_rule

TYPES = [HEX, PRISM, PYR, TET]


def dim_formula(etype, N):
    n = N + 1
    return {HEX: n ** 3, PRISM: n * n * (n + 1) // 2, PYR: n * (n + 1) * (2 * n + 1) // 6,
            TET: n * (n + 1) * (n + 2) // 6}[etype]


@pytest.mark.parametrize("etype", TYPES)
@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 5])
def test_dimension(etype, N):
    assert n_modes(etype, N) == dim_formula(etype, N)


@pytest.mark.parametrize("etype", TYPES)
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_orthonormal_exact_rule(etype, N):
    # N+3 points per collapsed direction integrate phi_i phi_j exactly
    pts, w = volume_rule(etype, N + 2)
    V = eval_basis(etype, N, pts)
    M = V.T @ (w[:, None] * V)
    assert np.abs(M - np.eye(M.shape[0])).max() < 1e-13


def space_monomials(etype, N):
    for a, b, c in itertools.product(range(N + 1), repeat=3):
        if etype == HEX or (etype == PRISM and a + b <= N) or (etype in (TET, PYR) and a + b + c <= N):
            yield a, b, c


@pytest.mark.parametrize("etype", TYPES)
@pytest.mark.parametrize("N", [1, 2, 3])
def test_reproduces_space(etype, N):
    pts, w = volume_rule(etype, N + 2)
    V = eval_basis(etype, N, pts)
    rng = np.random.default_rng(0)
    # random interior test points
    a, b, c = rng.uniform(-0.95, 0.95, size=(3, 20))
    tp = np.stack(uncollapse(etype, a, b, c), axis=1)
    Vt = eval_basis(etype, N, tp)
    for (i, j, k) in space_monomials(etype, N):
        f = lambda P: P[:, 0] ** i * P[:, 1] ** j * P[:, 2] ** k
        coef = V.T @ (w * f(pts))
        assert np.abs(Vt @ coef - f(tp)).max() < 1e-12


def test_n0_is_cell_average():
    for t in TYPES:
        pts, w = volume_rule(t, 0)
        V = eval_basis(t, 0, pts)
        assert np.allclose(V, 1.0 / np.sqrt(REF_VOLUME[t]), atol=1e-15)


@pytest.mark.parametrize("etype", TYPES)
def test_gradient_finite_difference(etype):
    N = 3
    rng = np.random.default_rng(1)
    a, b, c = rng.uniform(-0.8, 0.8, size=(3, 12))
    P = np.stack(uncollapse(etype, a, b, c), axis=1)
    _, G = eval_basis(etype, N, P, grad=True)
    h = 1e-5
    for k in range(3):
        dP = np.zeros(3)
        dP[k] = h
        fd = (eval_basis(etype, N, P + dP) - eval_basis(etype, N, P - dP)) / (2 * h)
        assert np.abs(fd - G[k]).max() < 1e-6 * max(1.0, np.abs(G[k]).max())


@pytest.mark.parametrize("etype", TYPES)
@pytest.mark.parametrize("N", [1, 3, 4])
def test_divergence_theorem(etype, N):
    """int grad phi_i = sum_faces int phi_i n dS on the reference element."""
    pts, w = volume_rule(etype, N + 2)
    _, G = eval_basis(etype, N, pts, grad=True)
    lhs = np.einsum("q,kqi->ki", w, G)
    rhs = np.zeros_like(lhs)
    centre = REF_VERTS[etype].mean(0)
    for lf, fv in enumerate(FACES[etype]):
        fp, fw, ts, tt = face_rule(etype, lf, N + 2)
        cr = np.cross(ts, tt)
        S = np.linalg.norm(cr)
        n = cr / S
        if np.dot(n, REF_VERTS[etype][fv].mean(0) - centre) < 0:
            n = -n
        phi = eval_basis(etype, N, fp)
        rhs += np.outer(n, (fw * S) @ phi)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_collapse_roundtrip():
    rng = np.random.default_rng(2)
    a, b, c = rng.uniform(-0.99, 0.99, size=(3, 50))
    for t in TYPES:
        x = uncollapse(t, a, b, c)
        a2, b2, c2 = collapse(t, *x)
        assert np.allclose([a2, b2, c2], [a, b, c], atol=1e-13)
