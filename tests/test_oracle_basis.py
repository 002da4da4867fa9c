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


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_hex_scaled_nodal_basis_is_orthogonal(N):
    """On the hexahedron the n-point rule (n = N + 1) integrates every product
    of two modes exactly and V is square, so O = W^{1/2} V is an orthogonal
    matrix: storing W^{1/2} V Q instead of Q is an exact change of basis
    whose inverse is its transpose (what lets the hexahedra be stored in
    nodal values with cotangents transforming like states).  A prism has
    fewer modes than points, so no such square transform exists there."""
    pts, w = volume_rule(HEX, N)
    V = eval_basis(HEX, N, pts)
    assert V.shape == (len(w), len(w))
    O = np.sqrt(w)[:, None] * V
    eye = np.eye(len(w))
    assert np.abs(O.T @ O - eye).max() < 1e-13
    assert np.abs(O @ O.T - eye).max() < 1e-13
    # V M^{-1} V^T = W^{-1}: the projected residual is a pointwise scale
    assert np.abs(V @ V.T - np.diag(1.0 / w)).max() < 1e-12 * (1.0 / w).max()
    pts_p, w_p = volume_rule(PRISM, N)
    assert eval_basis(PRISM, N, pts_p).shape[1] < len(w_p)


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


def test_jacobi_against_exact_sum():
    """P_n^(a,b) from the recurrence vs its explicit finite sum
    sum_s C(n+a, n-s) C(n+b, s) ((x-1)/2)^s ((x+1)/2)^(n-s) evaluated with 50
    significant digits (mpmath), for the orders and weights the bases use."""
    mp = pytest.importorskip("mpmath")
    from oracle.elements import jacobi
    mp.mp.dps = 50
    xs = np.linspace(-0.99, 0.99, 23)
    worst = 0.0
    for n in range(0, 7):
        for a in range(0, 15):
            for b in (0, 1):
                got = jacobi(n, a, b, xs)
                for x, g in zip(xs, got):
                    X = mp.mpf(float(x))
                    ref = sum(mp.binomial(n + a, n - s) * mp.binomial(n + b, s) * ((X - 1) / 2) ** s * ((X + 1) / 2) ** (n - s)
                              for s in range(n + 1))
                    worst = max(worst, abs(g - float(ref)) / max(1.0, abs(float(ref))))
    assert worst < 2e-14


def test_neighbour_points_are_face_points():
    """The neighbour's reference coordinates of the owner's face points, found
    by inverting its affine map, form the neighbour's own face point set when
    the face rule is symmetric (quadrilaterals; triangles sharing the collapse
    vertex) and always lie on the neighbour's face."""
    import dg_inputs as di
    from oracle.mesh import from_box
    from oracle.quadrature import face_rule
    for kind, m in (("mixed", 3), ("kuhn", 2)):
        box = di.reorder_vertices(di.box_mesh(m, kind, seed=1), seed=4)
        mesh = from_box(box, 3)
        for f, (e0, l0, e1, l1) in enumerate(mesh.faces):
            _, ref1, _, _ = mesh.face_geometry(f)
            fv = FACES[mesh.etype[e1]][l1]
            C = REF_VERTS[mesh.etype[e1]][fv]
            nrm = np.cross(C[1] - C[0], C[2] - C[0])
            assert np.abs((ref1 - C[0]) @ nrm).max() < 1e-14
            if len(fv) == 4:
                own, _, _, _ = face_rule(mesh.etype[e1], l1, 3)
                d = np.abs(ref1[:, None, :] - own[None, :, :]).sum(-1).min(1)
                assert d.max() < 1e-14
