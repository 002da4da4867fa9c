"""Pins of the curved-element oracle (pointwise J in Eq. 1 and in the
projection of Algorithm 1, vertex-interpolated element maps):

  * on affine meshes it reproduces the affine oracle (projection and RHS);
  * the perturbed meshes still tile the periodic box exactly: sum of
    w_q J_q over all elements = (2 pi)^3;
  * divergence theorem on every element with the face rule's points, normals
    and weights: sum_p (w S n)_p = 0 and sum_p x_d (w S n_d')_p = delta Vol;
  * free-stream preservation and discrete conservation on randomly
    perturbed meshes of every kind;
  * the projection preserves integrals (1^T W J V M^{-1} V^T W J q = 1^T W J q)
    and reproduces the element maps, which lie in every type's modal space;
  * the Newton-inverted neighbour points are the owner's physical points;
  * Algorithm 1 cross-check with Lagrange test functions on the collapsed grid;
  * L2 convergence of order about N+1 under a smooth deformation of the box.
"""
import math

import numpy as np
import pytest

import dg_inputs as di
from oracle.curved import CurvedOracle, curved_from_box
from oracle.dg import Oracle
from oracle.elements import collapse, collapse_jacobian, eval_basis
from oracle.euler import physical_flux, riemann
from oracle.mesh import from_box
from oracle.quadrature import gauss_legendre, volume_rule

U_CONST = np.array([1.2, 0.3, -0.2, 0.1, 3.0])


def curved(kind, m, N, amp=0.1, smooth=False, seed=1, flux="lf"):
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=seed), amp, smooth=smooth)
    return CurvedOracle(curved_from_box(box, N), flux=flux)


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("kuhn", 2, 3), ("hex", 2, 4), ("pyramid", 2, 3)])
def test_affine_limit(kind, m, N):
    box = di.box_mesh(m, kind, seed=1)
    oc, oa = CurvedOracle(curved_from_box(box, N)), Oracle(from_box(box, N))
    Q = oa.project(lambda x: di.perturbed_tgv_state(x, seed=3))
    Qc = oc.project(lambda x: di.perturbed_tgv_state(x, seed=3))
    assert np.abs(Qc - Q).max() < 1e-14 * np.abs(Q).max()
    R, Rc = oa.rhs(Q), oc.rhs(Q)
    for e in range(0, oa.mesh.n_elems, 2):
        vol = oa.apply_minv(e, oa.volume_term(Q, e))
        sl = slice(oa.mesh.dof_off[e], oa.mesh.dof_off[e + 1])
        assert np.abs(Rc[sl] - R[sl]).max() < 1e-13 * np.abs(vol).max()


@pytest.mark.parametrize("kind,m,N", [("hex", 2, 1), ("hex", 2, 3), ("prism", 2, 3), ("pyramid", 2, 1),
                                      ("pyramid", 2, 3), ("mixed", 3, 3), ("kuhn", 2, 2), ("four", 4, 2)])
def test_geometry_identities(kind, m, N):
    o = curved(kind, m, N)
    mesh = o.mesh
    vols = np.array([o.volume(e) for e in range(mesh.n_elems)])
    assert abs(vols.sum() / (2 * np.pi) ** 3 - 1) < 1e-14
    for e in range(mesh.n_elems):
        tot, mom = np.zeros(3), np.zeros((3, 3))
        for f, side in mesh.elem_faces[e]:
            e0, _, e1, _ = mesh.faces[f]
            ref0, ref1, wS, nrm = mesh.face_geometry(f)
            x = mesh.to_physical(e0, ref0) if side == 0 else mesh.to_physical(e1, ref1)
            a = (wS * nrm) * (1 if side == 0 else -1)
            tot += a.sum(1)
            mom += np.einsum("pd,ep->de", x, a)
        assert np.abs(tot).max() < 1e-14 * vols[e] ** (2 / 3) * 10
        assert np.abs(mom - vols[e] * np.eye(3)).max() < 1e-14 * vols[e] * 10


@pytest.mark.parametrize("kind,m,N", [("hex", 2, 1), ("hex", 2, 3), ("prism", 2, 1), ("prism", 2, 3),
                                      ("pyramid", 2, 1), ("pyramid", 2, 3), ("mixed", 3, 3), ("kuhn", 2, 2),
                                      ("four", 4, 2)])
@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_free_stream(kind, m, N, flux):
    o = curved(kind, m, N, flux=flux)
    Q = o.project(lambda x: np.tile(U_CONST[:, None], (1, x.shape[0])))
    worst = 0.0
    for e in range(o.mesh.n_elems):
        vol = o.volume_term(Q, e)
        worst = max(worst, np.abs(vol - o.surface_term(Q, e)).max() / np.abs(vol).max())
    assert worst < 1e-13


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("kuhn", 2, 2), ("four", 4, 2), ("pyramid", 2, 2)])
def test_conservation(kind, m, N):
    o = curved(kind, m, N)
    R = o.rhs(o.project(di.tgv_state))
    tot = sum(o.integrate(R, e) for e in range(o.mesh.n_elems))
    scale = max(np.abs(o.integrate(np.abs(R), e)).max() for e in range(o.mesh.n_elems))
    assert np.abs(tot).max() < 1e-13 * scale * o.mesh.n_elems


@pytest.mark.parametrize("kind,m,N", [("mixed", 2, 1), ("mixed", 2, 3), ("four", 4, 2)])
def test_projection_integrals_and_maps(kind, m, N):
    o = curved(kind, m, N)
    mesh = o.mesh
    # integrals of the projected TGV state equal the quadrature integrals
    Q = o.project(di.tgv_state)
    for e in range(mesh.n_elems):
        op = o.ops[mesh.etype[e]]
        direct = di.tgv_state(o.quad_points(e)) @ (op.w * o.Jq[e])
        assert np.abs(o.integrate(Q, e) - direct).max() < 1e-13 * np.abs(direct).max()
    # the element map (relative to the element's first vertex) is in the space
    for e in range(mesh.n_elems):
        op = o.ops[mesh.etype[e]]
        x = mesh.to_physical_rel(e, op.pts).T                     # [3, nQ]
        c = o.apply_minv(e, (x * (op.w * o.Jq[e])) @ op.V)
        pts = np.array([[-0.3, -0.4, -0.1], [0.1, -0.8, 0.2], [-0.9, -0.2, -0.5]])
        assert np.abs(c @ eval_basis(mesh.etype[e], N, pts).T - mesh.to_physical_rel(e, pts).T).max() < 1e-13 * 2 * np.pi


def test_neighbour_points_match():
    o = curved("four", 4, 3)
    mesh = o.mesh
    for f in range(0, len(mesh.faces), 5):
        e0, l0, e1, l1 = mesh.faces[f]
        ref0, ref1, _, _ = mesh.face_geometry(f)
        x0 = mesh.to_physical(e0, ref0)
        x1 = mesh.to_physical(e1, ref1)
        d = (x0 - x1) / mesh.period
        assert np.abs(d - np.rint(d)).max() < 1e-14 * 10


def lagrange(nodes, x):
    x = np.asarray(x, dtype=float)[:, None]
    n = len(nodes)
    L = np.ones((x.shape[0], n))
    dL = np.zeros((x.shape[0], n))
    for i in range(n):
        for j in range(n):
            if j == i:
                continue
            term = (x[:, 0] - nodes[j]) / (nodes[i] - nodes[j])
            dL[:, i] = dL[:, i] * term + L[:, i] / (nodes[i] - nodes[j])
            L[:, i] = L[:, i] * term
    return L, dL


def nodal_residual(o, Q, e):
    """Eq. 1 tested with the tensor Lagrange functions of the collapsed grid
    (Algorithm 1's nodal form) with pointwise metrics, mapped back by V^T."""
    m = o.mesh
    t, N = m.etype[e], m.N
    x, _ = gauss_legendre(N + 1)
    op = o.ops[t]
    a, b, c = collapse(t, *op.pts.T)
    n = N + 1
    (La, dLa), (Lb, dLb), (Lc, dLc) = lagrange(x, a), lagrange(x, b), lagrange(x, c)
    dabc = np.stack([np.einsum("qi,qj,qk->qijk", dLa, Lb, Lc),
                     np.einsum("qi,qj,qk->qijk", La, dLb, Lc),
                     np.einsum("qi,qj,qk->qijk", La, Lb, dLc)]).reshape(3, len(a), n ** 3)
    Jc = collapse_jacobian(t, a, b, c)
    gxi = np.linalg.solve(np.transpose(Jc, (0, 2, 1)), np.transpose(dabc, (1, 0, 2)))  # [q, 3(xi), m]
    Jq, G = m.volume_geometry(e, op.pts)
    gx = np.einsum("qkd,qkm->dqm", G, gxi)
    U = m.block(Q, e) @ op.V.T
    F = physical_flux(U, o.gamma)
    vol = np.einsum("dqm,dvq->vm", gx, (op.w * Jq) * F)
    surf = np.zeros_like(vol)
    for f, side in m.elem_faces[e]:
        e0, _, e1, _ = m.faces[f]
        ref0, ref1, wS, nrm = m.face_geometry(f)
        UL = m.block(Q, e0) @ eval_basis(m.etype[e0], N, ref0).T
        UR = m.block(Q, e1) @ eval_basis(m.etype[e1], N, ref1).T
        Fh = wS * riemann(o.flux, UL, UR, nrm, o.gamma)
        ref = ref0 if side == 0 else ref1
        fa, fb, fc = collapse(t, *ref.T)
        ellf = np.einsum("pi,pj,pk->pijk", lagrange(x, fa)[0], lagrange(x, fb)[0],
                         lagrange(x, fc)[0]).reshape(len(fa), n ** 3)
        surf += (Fh @ ellf) if side == 0 else -(Fh @ ellf)
    return (vol - surf) @ op.V


@pytest.mark.parametrize("kind,m,N", [("mixed", 2, 3), ("four", 4, 2)])
def test_algorithm1_nodal_equivalence(kind, m, N):
    o = curved(kind, m, N)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    for e in range(0, o.mesh.n_elems, 3):
        modal = o.volume_term(Q, e) - o.surface_term(Q, e)
        assert np.abs(modal - nodal_residual(o, Q, e)).max() < 1e-12 * np.abs(modal).max()


def l2_density_error(o, Q, t):
    err, rules = 0.0, {}
    for e in range(o.mesh.n_elems):
        et = o.mesh.etype[e]
        if et not in rules:
            pts, w = volume_rule(et, o.mesh.N + 3)
            rules[et] = (pts, w, eval_basis(et, o.mesh.N, pts))
        pts, w, V = rules[et]
        Jq, _ = o.mesh.volume_geometry(e, pts)
        rho_h = (o.mesh.block(Q, e) @ V.T)[0]
        rho = di.advected_density_state(o.mesh.to_physical(e, pts), t=t)[0]
        err += (w * Jq) @ (rho_h - rho) ** 2
    return math.sqrt(err)


@pytest.mark.parametrize("kind,N,margin", [("hex", 3, 0.4), ("prism", 3, 0.2), ("pyramid", 3, 0.2),
                                           ("mixed", 3, 0.1)])
def test_convergence_order_smooth_deformation(kind, N, margin):
    """Density error after 5 LSERK steps on 2^3 and 4^3 cube meshes under the
    same smooth deformation of the box (measured rates 3.2-3.8 at N = 3)."""
    T, errs = 0.1, []
    for m in (2, 4):
        o = curved(kind, m, N, amp=0.15, smooth=True)
        Q = o.run(o.project(di.advected_density_state), T / 5, 5)
        errs.append(l2_density_error(o, Q, T))
    rate = math.log2(errs[0] / errs[1])
    assert rate > N + margin, (errs, rate)


def test_perturbed_meshes_are_curved():
    """The perturbation really makes hex, prism and pyramid maps non-affine
    (J varies inside the element), while tetrahedra keep a constant J."""
    o = curved("four", 4, 2)
    spread = {}
    for e in range(o.mesh.n_elems):
        t = int(o.mesh.etype[e])
        spread[t] = max(spread.get(t, 0.0), np.ptp(o.Jq[e]) / o.Jq[e].mean())
    assert spread[0] > 1e-2 and spread[1] > 1e-2 and spread[2] > 1e-2
    assert spread[3] < 1e-13


@pytest.mark.parametrize("kind,m,N,flux", [("mixed", 2, 2, "lf"), ("four", 4, 1, "lf"), ("pyramid", 2, 2, "roe")])
def test_adjoint_dot_product(kind, m, N, flux):
    """<J v, w> = <v, J^T w> with J v by a complex step through the curved
    residual (exact to rounding) and J^T w from rhs_vjp."""
    from oracle.adjoint import rhs_jvp
    o = curved(kind, m, N, flux=flux)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    scale = np.abs(Q).max()
    v = di.random_vector(Q.size, seed=21) * scale
    w = di.random_vector(Q.size, seed=22)
    lhs = rhs_jvp(o, Q, v) @ w
    rhs = v @ o.rhs_vjp(Q, w)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_rk_adjoint_dot_product():
    from oracle.adjoint import rk_jvp, rk_vjp
    o = curved("mixed", 2, 2)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    v = di.random_vector(Q.size, seed=23) * np.abs(Q).max()
    w = di.random_vector(Q.size, seed=24)
    lhs = rk_jvp(o, Q, 1e-3, 2, v) @ w
    rhs = v @ rk_vjp(o, Q, 1e-3, 2, w)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


# ---------------------------------------------------------------- Navier-Stokes on curved elements
NS_MU, NS_PR = 0.05, 0.72


def curved_ns(kind, m, N, amp=0.1, mu=NS_MU, flux="lf", reorder=None):
    from oracle.curved import CurvedNSOracle
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=1), amp)
    if reorder is not None:
        box = di.reorder_vertices(box, seed=reorder)
    return CurvedNSOracle(curved_from_box(box, N), flux=flux, mu=mu, Pr=NS_PR)


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("four", 4, 2)])
def test_ns_affine_limit(kind, m, N):
    from oracle.curved import CurvedNSOracle
    from oracle.navier_stokes import NSOracle
    box = di.box_mesh(m, kind, seed=1)
    oc = CurvedNSOracle(curved_from_box(box, N), mu=NS_MU, Pr=NS_PR)
    oa = NSOracle(from_box(box, N), mu=NS_MU, Pr=NS_PR)
    Q = oa.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    R, Rc = oa.rhs(Q), oc.rhs(Q)
    G = oa.lifted_gradient(Q)
    for e in range(0, oa.mesh.n_elems, 2):
        vol = oa.apply_minv(e, oa.ns_volume_term(Q, e, G))
        sl = slice(oa.mesh.dof_off[e], oa.mesh.dof_off[e + 1])
        assert np.abs(Rc[sl] - R[sl]).max() < 1e-13 * np.abs(vol).max()


def test_ns_mu_zero_is_curved_euler():
    o = curved_ns("mixed", 3, 3, mu=0.0)
    oe = curved("mixed", 3, 3)
    Q = oe.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    assert np.abs(o.rhs(Q) - oe.rhs(Q)).max() <= 1e-14 * np.abs(oe.rhs(Q)).max()


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("four", 4, 2), ("pyramid", 2, 2)])
def test_ns_free_stream_and_conservation(kind, m, N):
    o = curved_ns(kind, m, N)
    Qf = o.project(lambda x: np.tile(U_CONST[:, None], (1, x.shape[0])))
    assert np.abs(o.rhs(Qf)).max() < 1e-12
    R = o.rhs(o.project(di.tgv_state))
    tot = sum(o.integrate(R, e) for e in range(o.mesh.n_elems))
    scale = max(np.abs(o.integrate(np.abs(R), e)).max() for e in range(o.mesh.n_elems))
    assert np.abs(tot).max() < 1e-13 * scale * o.mesh.n_elems


# a primitive state linear in x (rho, u, v, w, p) and its constant gradient
LIN = np.array([[1.0, 0.10, -0.05, 0.02],
                [0.3, 0.20, 0.10, -0.10],
                [-0.2, 0.05, 0.15, 0.07],
                [0.1, -0.12, 0.04, 0.09],
                [70.0, 1.0, -2.0, 0.5]])


def lin_state(x, gamma=1.4):
    rho, u, v, w, p = LIN[:, :1] + LIN[:, 1:] @ x.T
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)])


@pytest.mark.parametrize("kind,N", [("hex", 3), ("mixed", 3), ("prism", 3), ("pyramid", 3)])
def test_ns_lifting_exact_for_linear_W(kind, N):
    """The curved element maps lie in every type's modal space, so at N = 3
    the conservative state of a W linear in x (cubic in x) is represented
    exactly; BR1 lifting then returns grad W on elements away from the
    periodic seam (where the non-periodic W jumps)."""
    m = 4
    o = curved_ns(kind, m, N)
    Q = o.project(lin_state)
    h = 2 * np.pi / m
    idx = np.floor((o.mesh.centroid + np.pi) / h).astype(int)
    elems = np.nonzero(np.all((idx >= 1) & (idx <= m - 2), axis=1))[0]
    assert len(elems) > 0
    G = o.lifted_gradient(Q, elems)
    exact = LIN[:, 1:].T
    wmax = np.abs(LIN[:, 0]) + np.pi * np.abs(LIN[:, 1:]).sum(axis=1)
    for e in elems:
        gq = G[e] @ o.ops[o.mesh.etype[e]].V.T
        err = np.abs(gq - exact[:, :, None]).max(axis=(0, 2))
        assert np.all(err < 5e-12 * wmax), (e, err)


@pytest.mark.parametrize("kind,m,N,flux", [("mixed", 2, 2, "lf"), ("four", 4, 1, "roe")])
def test_ns_adjoint_dot_product(kind, m, N, flux):
    from oracle.adjoint import rhs_jvp
    o = curved_ns(kind, m, N, flux=flux)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    v = di.random_vector(Q.size, seed=25) * np.abs(Q).max()
    w = di.random_vector(Q.size, seed=26)
    lhs = rhs_jvp(o, Q, v) @ w
    rhs = v @ o.rhs_vjp(Q, w)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
