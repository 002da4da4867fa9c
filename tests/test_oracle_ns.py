"""Pins of the oracle's Navier-Stokes residual with BR1 lifting.

  * BR1 lifting reproduces the exact gradient of a primitive state W that is
    linear or quadratic in x (and whose conservative state lies in the modal
    space): by Gauss's theorem the lifted gradient is the projection of grad W
    whenever W is continuous across the element's faces, so on elements away
    from the periodic seam (where a non-periodic polynomial jumps) G = grad W
    to rounding;
  * exact residual of a polynomial state: with rho = 1, u linear and p
    quadratic every flux is a polynomial of degree <= 3, the quadrature is
    exact at N = 4, and the DG residual on elements two layers away from the
    seam equals the L2 projection of the strong-form residual
    -div(F_e - F_v), computed here symbolically (sympy) from the textbook
    Navier-Stokes-Fourier fluxes -- an independent route to the viscous
    stress, the heat flux and every sign;
  * mu = 0 reduces the residual to the Euler residual;
  * free-stream preservation and discrete conservation on periodic meshes.
"""
import math

import numpy as np
import pytest

import dg_inputs as di
from oracle.dg import Oracle
from oracle.mesh import from_box
from oracle.navier_stokes import NSOracle

GAMMA, MU, PR = 1.4, 0.05, 0.72


def make(kind, m, N, seed=1, mu=MU, flux="lf", reorder=None):
    box = di.box_mesh(m, kind, seed=seed)
    if reorder is not None:
        box = di.reorder_vertices(box, seed=reorder)
    return NSOracle(from_box(box, N), flux=flux, gamma=GAMMA, mu=mu, Pr=PR)


def interior(o, m, layers):
    """Elements whose cube lies at least `layers` cubes away from the seam."""
    h = 2 * math.pi / m
    idx = np.floor((o.mesh.centroid + math.pi) / h).astype(int)
    ok = np.all((idx >= layers) & (idx <= m - 1 - layers), axis=1)
    return np.nonzero(ok)[0]


def conservative(rho, u, v, w, p):
    return np.stack([rho, rho * u, rho * v, rho * w, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v + w * w)])


# a linear primitive state (rho, u, v, w, p) and its constant gradient
LIN = np.array([[1.0, 0.10, -0.05, 0.02],      # rho = c0 + c . x
                [0.3, 0.20, 0.10, -0.10],
                [-0.2, 0.05, 0.15, 0.07],
                [0.1, -0.12, 0.04, 0.09],
                [70.0, 1.0, -2.0, 0.5]])


def lin_state(x):
    W = LIN[:, :1] + LIN[:, 1:] @ x.T
    return conservative(*W)


@pytest.mark.parametrize("kind,N,reorder", [("mixed", 3, None), ("kuhn", 3, 5), ("mixed", 4, 3), ("prism", 3, None)])
def test_lifting_exact_for_linear_W(kind, N, reorder):
    m = 4
    o = make(kind, m, N, reorder=reorder)
    Q = o.project(lin_state)
    elems = interior(o, m, 1)
    assert len(elems) > 0
    G = o.lifted_gradient(Q, elems)
    exact = LIN[:, 1:].T                                   # [3(d), 5]
    # rounding of W_v (size |W_v|) through a derivative: tolerance per component
    wmax = np.abs(LIN[:, 0]) + math.pi * np.abs(LIN[:, 1:]).sum(axis=1)
    for e in elems:
        gq = G[e] @ o.ops[o.mesh.etype[e]].V.T              # [3, 5, nQ]
        err = np.abs(gq - exact[:, :, None]).max(axis=(0, 2))
        assert np.all(err < 5e-12 * wmax), (e, err)


def test_lifting_exact_for_quadratic_p():
    m, N = 4, 3
    o = make("mixed", m, N, seed=2)
    c = np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.25])        # p = 70 + quadratic form

    def state(x):
        X, Y, Z = x.T
        p = 70 + c[0] * X * X + c[1] * Y * Y + c[2] * Z * Z + c[3] * X * Y + c[4] * Y * Z + c[5] * X * Z
        one = np.ones_like(X)
        return conservative(one, 0.3 + 0.1 * Y, -0.2 + 0.05 * Z, 0.1 * one + 0.02 * X, p)

    Q = o.project(state)
    elems = interior(o, m, 1)
    G = o.lifted_gradient(Q, elems)
    for e in elems:
        op = o.ops[o.mesh.etype[e]]
        X, Y, Z = o.quad_points(e).T
        gp = np.stack([2 * c[0] * X + c[3] * Y + c[5] * Z, 2 * c[1] * Y + c[3] * X + c[4] * Z,
                       2 * c[2] * Z + c[4] * Y + c[5] * X])
        gq = G[e] @ op.V.T
        assert np.abs(gq[:, 4] - gp).max() < 5e-12 * 80.0       # |p| <= 80
        assert np.abs(gq[:, 0]).max() < 1e-11
        assert np.abs(gq[1, 1] - 0.1).max() < 1e-11 and np.abs(gq[2, 2] - 0.05).max() < 1e-11
        assert np.abs(gq[0, 3] - 0.02).max() < 1e-11


def strong_residual(which):
    """State and -div(F_e - F_v) of a polynomial state (rho = 1), derived
    symbolically (sympy) from the textbook Navier-Stokes-Fourier fluxes:
    returns (state(x[P,3]) -> [5, P], residual(x[P,3]) -> [5, P]).
      'linear':  u linear in x, y, z; p quadratic (every flux of degree <= 3);
      'shear':   u = (f(x), h(z), g(x)) quadratic, p = p0 + c y^2 + d x (fluxes
                 of degree <= 6 in each coordinate separately)."""
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z")
    xs = (X, Y, Z)
    R = sp.Rational
    rho = sp.Integer(1)
    if which == "linear":
        u = (R(3, 10) + R(1, 5) * X - R(1, 10) * Y + R(1, 20) * Z,
             -R(1, 5) + R(1, 10) * X + R(3, 20) * Y - R(1, 10) * Z,
             R(1, 10) - R(1, 20) * X + R(1, 25) * Y + R(1, 8) * Z)
        p = 70 + R(3, 10) * X ** 2 - R(1, 5) * Y ** 2 + R(1, 2) * Z ** 2 \
            + R(1, 10) * X * Y - R(2, 5) * Y * Z + R(1, 4) * X * Z + X - Z
    else:
        u = (R(1, 5) + R(1, 10) * X - R(1, 20) * X ** 2,
             R(-1, 10) + R(1, 8) * Z + R(1, 16) * Z ** 2,
             R(3, 10) - R(1, 10) * X + R(1, 12) * X ** 2)
        p = 70 + R(2, 5) * Y ** 2 - R(1, 2) * X
    g, mu, Pr = R(7, 5), R(1, 20), R(18, 25)
    E = p / (g - 1) + rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / 2
    U = [rho, rho * u[0], rho * u[1], rho * u[2], E]
    div = sum(sp.diff(u[i], xs[i]) for i in range(3))
    tau = [[mu * (sp.diff(u[i], xs[j]) + sp.diff(u[j], xs[i])) - (R(2, 3) * mu * div if i == j else 0)
            for j in range(3)] for i in range(3)]
    kappa = mu * g / ((g - 1) * Pr)
    qh = [-kappa * sp.diff(p / rho, xs[d]) for d in range(3)]
    res = []
    for v in range(5):
        tot = 0
        for d in range(3):
            if v == 0:
                Fe, Fv = rho * u[d], 0
            elif v < 4:
                Fe = rho * u[v - 1] * u[d] + (p if v - 1 == d else 0)
                Fv = tau[v - 1][d]
            else:
                Fe = (E + p) * u[d]
                Fv = sum(u[i] * tau[i][d] for i in range(3)) - qh[d]
            tot += sp.diff(Fe - Fv, xs[d])
        res.append(sp.expand(-tot))
    fns = [sp.lambdify((X, Y, Z), r, "numpy") for r in res]
    state_fns = [sp.lambdify((X, Y, Z), s, "numpy") for s in U]

    def ev(fs, x):
        return np.stack([np.broadcast_to(np.asarray(f(*x.T), dtype=float), (x.shape[0],)) for f in fs])

    return (lambda x: ev(state_fns, x)), (lambda x: ev(fns, x))


def check_exact(o, m, which):
    state, resid = strong_residual(which)
    Q = o.project(state)
    elems = interior(o, m, 2)
    assert len(elems) > 0
    R = o.rhs(Q, elems)
    Rex = o.project(resid)
    for e in elems:
        a, b = o.mesh.block(R, e), o.mesh.block(Rex, e)
        assert np.abs(a - b).max() < 1e-11 * max(1.0, np.abs(b).max()), (e, np.abs(a - b).max())


@pytest.mark.parametrize("kind,reorder", [("mixed", None), ("kuhn", 7), ("mixed", 4)])
@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_polynomial_state_exact_residual(kind, reorder, flux):
    """Linear velocity (constant stress: pins the viscous work and the heat
    flux) on every element type; the quadrature is exact at N = 4."""
    m, N = 6, 4
    o = make(kind, m, N, seed=3, flux=flux, reorder=reorder)
    assert o.mu == MU and o.Pr == PR
    check_exact(o, m, "linear")


@pytest.mark.parametrize("reorder", [None, 9])
def test_shear_state_exact_residual_hex(reorder):
    """Quadratic velocity (linear stress: pins every stress component in the
    momentum equations, diagonal and off-diagonal); on hexahedra the tensor
    Gauss rule with N + 1 = 6 points integrates each coordinate to degree 11,
    enough for these fluxes."""
    m, N = 6, 5
    o = make("hex", m, N, seed=3, reorder=reorder)
    check_exact(o, m, "shear")


def test_viscous_stress_invariants():
    """Stokes stress: symmetric and trace-free, zero for a rigid rotation and a
    uniform translation, mu * shear rate for a simple shear; heat flux zero
    for uniform p / rho."""
    from oracle.navier_stokes import viscous_flux
    rng = np.random.default_rng(5)
    U = conservative(np.array([1.3]), np.array([0.2]), np.array([-0.1]), np.array([0.3]), np.array([60.0]))
    g = rng.uniform(-1, 1, (3, 5, 1))
    F = viscous_flux(U, g, GAMMA, MU, PR)
    tau = F[:, 1:4, 0]                                     # tau[d, i] = F_v[d][1 + i]
    np.testing.assert_allclose(tau, tau.T, rtol=0, atol=1e-16)
    assert abs(np.trace(tau)) < 1e-16
    rot = np.zeros((3, 5, 1))
    A = np.array([[0, 0.3, -0.2], [-0.3, 0, 0.1], [0.2, -0.1, 0]])
    rot[:, 1:4, 0] = A                                     # du_i/dx_d antisymmetric
    assert np.abs(viscous_flux(U, rot, GAMMA, MU, PR)[:, 1:4]).max() < 1e-17
    shear = np.zeros((3, 5, 1))
    shear[1, 1, 0] = 0.7                                   # du/dy
    F = viscous_flux(U, shear, GAMMA, MU, PR)
    assert abs(F[1, 1, 0] - MU * 0.7) < 1e-17 and abs(F[0, 2, 0] - MU * 0.7) < 1e-17
    heat = np.zeros((3, 5, 1))
    heat[:, 0, 0] = [0.1, 0.2, -0.3]
    heat[:, 4, 0] = (60.0 / 1.3) * heat[:, 0, 0]           # grad p = (p/rho) grad rho
    assert np.abs(viscous_flux(U, heat, GAMMA, MU, PR)[:, 4]).max() < 1e-15
    assert np.all(viscous_flux(U, rot * 0, GAMMA, MU, PR)[:, 0] == 0)


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("kuhn", 2, 2)])
def test_mu_zero_is_euler(kind, m, N):
    o = make(kind, m, N, mu=0.0)
    e = Oracle(o.mesh, flux="lf", gamma=GAMMA)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=4, amp=0.05))
    np.testing.assert_allclose(o.rhs(Q), e.rhs(Q), rtol=0, atol=1e-14 * np.abs(e.rhs(Q)).max())


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("kuhn", 2, 3), ("mixed", 2, 4)])
def test_ns_free_stream(kind, m, N):
    o = make(kind, m, N)
    U0 = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    Q = o.project(lambda x: np.tile(U0[:, None], (1, x.shape[0])))
    R = o.rhs(Q)
    scale = max(abs(o.volume_term(Q, e)).max() for e in range(o.mesh.n_elems))
    assert np.abs(R).max() * min(o.mesh.J) < 1e-13 * scale


@pytest.mark.parametrize("kind,m,N,flux", [("mixed", 3, 3, "lf"), ("kuhn", 2, 2, "roe"), ("mixed", 2, 4, "lf")])
def test_ns_conservation(kind, m, N, flux):
    o = make(kind, m, N, flux=flux)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=6, amp=0.05))
    R = o.rhs(Q)
    total = sum(o.integrate(R, e) for e in range(o.mesh.n_elems))
    scale = sum(np.abs(o.integrate(R, e)) for e in range(o.mesh.n_elems))
    assert np.all(np.abs(total) < 1e-12 * scale), (total, scale)


# ---------------------------------------------------------------- adjoint
def ns_jvp(o, Q, V):
    """J(Q) V by one complex step through the NS residual (brute force route)."""
    h = 1e-30
    return o.rhs(np.asarray(Q, dtype=float) + 1j * h * np.asarray(V)).imag / h


@pytest.mark.parametrize("kind,m,N,flux,reorder", [("hex", 2, 1, "lf", None), ("prism", 2, 1, "roe", 3)])
def test_ns_vjp_dense_jacobian(kind, m, N, flux, reorder):
    """Transpose of the Jacobian assembled column by column with complex steps."""
    o = make(kind, m, N, flux=flux, reorder=reorder)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=5, amp=0.05))
    n = len(Q)
    J = np.stack([ns_jvp(o, Q, np.eye(n)[j]) for j in range(n)], axis=1)
    w = di.random_vector(n, seed=9)
    ref = J.T @ w
    got = o.rhs_vjp(Q, w)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("kind,m,N,flux,reorder", [("mixed", 2, 3, "lf", None), ("kuhn", 2, 2, "roe", 7),
                                                    ("mixed", 2, 2, "lf", 5)])
def test_ns_vjp_dot(kind, m, N, flux, reorder):
    o = make(kind, m, N, flux=flux, reorder=reorder)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=6, amp=0.05))
    w = di.random_vector(len(Q), seed=10)
    vjp = o.rhs_vjp(Q, w)
    for s in range(3):
        v = di.random_vector(len(Q), seed=20 + s)
        a, b = np.dot(w, ns_jvp(o, Q, v)), np.dot(vjp, v)
        assert abs(a - b) < 1e-11 * (np.abs(w).sum() * np.abs(ns_jvp(o, Q, v)).max()), (a, b)


def test_ns_rk_vjp_dot():
    from oracle.adjoint import rk_jvp, rk_vjp
    o = make("mixed", 2, 2)
    Q = o.project(lambda x: di.perturbed_tgv_state(x, seed=7, amp=0.05))
    w = di.random_vector(len(Q), seed=11)
    v = di.random_vector(len(Q), seed=12)
    dt, K = 2e-3, 2
    a = np.dot(w, rk_jvp(o, Q, dt, K, v))
    b = np.dot(rk_vjp(o, Q, dt, K, w), v)
    assert abs(a - b) < 1e-11 * abs(a), (a, b)
