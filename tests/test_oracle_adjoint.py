"""Pins of the oracle adjoint (no counterpart in the paper): the hand-written
transposed residual against the dense Jacobian assembled by complex steps
through the oracle's forward residual (brute force), the dot-product test
<J v, w> = <v, J^T w>, central finite differences, and the reverse LSERK."""
import numpy as np
import pytest

import dg_inputs as di
from oracle.adjoint import rhs_jvp, rhs_vjp, rk_jvp, rk_vjp
from oracle.dg import Oracle
from oracle.mesh import from_box


def make(kind, m, N, flux="lf", seed=1):
    return Oracle(from_box(di.box_mesh(m, kind, seed=seed), N), flux=flux)


def state(o, seed=3):
    return o.project(lambda x: di.perturbed_tgv_state(x, seed=seed, amp=0.05))


@pytest.mark.parametrize("kind,N,ncols", [("hex", 1, None), ("kuhn", 1, 48), ("mixed", 2, 48)])
@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_vjp_equals_dense_jacobian(kind, N, ncols, flux):
    """Columns of J by complex steps (all of them, or a seeded subset)."""
    o = make(kind, 2, N, flux=flux)
    Q = state(o)
    n = Q.size
    cols = np.arange(n) if ncols is None else np.sort(
        np.random.default_rng(11).choice(n, size=ncols, replace=False))
    Jd = np.stack([rhs_jvp(o, Q, np.eye(n)[k]) for k in cols], axis=1)
    w = di.random_vector(n, seed=7)
    ref = Jd.T @ w
    assert np.abs(rhs_vjp(o, Q, w)[cols] - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("kind,m,N", [("mixed", 2, 2), ("mixed", 3, 1)])
@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_dot_product(kind, m, N, flux):
    o = make(kind, m, N, flux=flux)
    Q = state(o)
    for s in range(2):
        v = di.random_vector(Q.size, seed=10 + s)
        w = di.random_vector(Q.size, seed=20 + s)
        a = w @ rhs_jvp(o, Q, v)
        b = v @ rhs_vjp(o, Q, w)
        assert abs(a - b) < 1e-11 * abs(a)


@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_jvp_central_difference(flux):
    """Central differences with the perturbation scaled per variable (h small
    enough not to cross the kinks of max and |.|)."""
    o = make("mixed", 2, 2, flux=flux)
    Q = state(o)
    scale = np.concatenate([np.repeat(np.abs(o.mesh.block(Q, e)).max(1), o.mesh.nM[e])
                            for e in range(o.mesh.n_elems)])
    v = di.random_vector(Q.size, seed=5) * scale
    h = 1e-7
    fd = (o.rhs(Q + h * v) - o.rhs(Q - h * v)) / (2 * h)
    jv = rhs_jvp(o, Q, v)
    assert np.abs(fd - jv).max() < 1e-6 * np.abs(jv).max()


def test_rk_vjp_dot_product():
    o = make("mixed", 2, 2)
    Q0 = state(o)
    v = di.random_vector(Q0.size, seed=31)
    w = di.random_vector(Q0.size, seed=32)
    dt, K = 2e-3, 2
    a = w @ rk_jvp(o, Q0, dt, K, v)
    b = v @ rk_vjp(o, Q0, dt, K, w)
    assert abs(a - b) < 1e-11 * abs(a)


def test_abs_kink_reading():
    """At u.n = 0 exactly (w = 0 on z-faces of the TGV) the Roe adjoint uses
    d|x|/dx = 0, which central differences reproduce."""
    from oracle.euler import rabs
    x = np.array([0.0, 1.0, -2.0]) + 1j * 1e-30
    assert np.allclose(rabs(x).imag / 1e-30, [0.0, 1.0, -1.0])
