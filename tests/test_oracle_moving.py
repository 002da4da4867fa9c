"""Pins of the moving-mesh oracle (oracle/moving.py): reduction to the static
curved oracle at zero velocity, the geometric conservation law (the residual
of a constant state is the time derivative of its moments, and a constant
state stays constant through LSERK steps -- while the same steps with the
Jacobian at the stage time drift), conservation of int J q, and convergence
to the advected density wave on a mesh in motion."""
import math

import numpy as np
import pytest

import dg_inputs as di
from oracle.curved import CurvedOracle, curved_from_box
from oracle.dg import LSERK_A, LSERK_B
from oracle.elements import eval_basis
from oracle.moving import LSERK_C, MovingOracle
from oracle.quadrature import volume_rule

CONST = np.array([1.2, 0.3, -0.2, 0.1, 3.0])


def moving(kind, m, N, amp=0.3, seed=1):
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=seed), 0.1)
    return MovingOracle(box, N, di.vertex_velocities(box.xyz, amp)), box


def constant(mo):
    return mo.project(lambda x: np.repeat(CONST[:, None], len(x), axis=1), 0.0)


def test_zero_velocity_is_the_static_curved_oracle():
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    N = 2
    mo = MovingOracle(box, N, np.zeros_like(box.xyz))
    co = CurvedOracle(curved_from_box(box, N))
    Q = co.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    np.testing.assert_array_equal(mo.rhs(Q, 0.0), co.rhs(Q))
    a, b = mo.run(Q, 0.0, 1e-3, 2), co.run(Q, 1e-3, 2)
    assert np.abs(a - b).max() < 1e-14 * np.abs(b).max()


@pytest.mark.parametrize("kind,N", [("hex", 2), ("prism", 3), ("pyramid", 2), ("mixed", 1), ("mixed", 3)])
def test_geometric_conservation(kind, N):
    mo, _ = moving(kind, 2, N)
    Q = constant(mo)
    # semi-discrete: the residual of a constant state is d/dt of its moments
    # M(t) Q (a cubic in t: the four-point difference is exact)
    h = 0.1
    W = lambda t: mo.weighted(Q, t)
    dm = (-W(2 * h) + 8 * W(h) - 8 * W(-h) + W(-2 * h)) / (12 * h)
    assert np.abs(mo.rate(Q, 0.0) - dm).max() < 1e-13 * np.abs(W(0.0)).max()
    # fully discrete: steps keep the constant to rounding
    Q2 = mo.run(Q, 0.0, 0.05, 2)
    assert np.abs(Q2 - Q).max() < 1e-13 * np.abs(Q).max()


def test_stage_time_jacobian_drifts():
    """The discrete GCL is what keeps the constant: the same step with the
    Jacobian taken at the stage time moves it by O(dt^5)."""
    mo, _ = moving("pyramid", 2, 2)
    Q = constant(mo)
    t, dt = 0.0, 0.1
    Ut = mo.weighted(Q, t)
    K = np.zeros_like(Ut)
    for s in range(5):
        ts = t + LSERK_C[s] * dt
        K = LSERK_A[s] * K + dt * mo.rate(mo.unweighted(Ut, ts), ts)
        Ut = Ut + LSERK_B[s] * K
    drift = np.abs(mo.unweighted(Ut, t + dt) - Q).max()
    assert drift > 1e-8, drift


def _stage_values_of_powers(t, dt):
    """The 2N-storage recursion of the scheme on dy_k/dt = k t^(k-1),
    y_k(t) = t^k: the largest deviation of the stage values from t_s^k and
    of the end values from (t + dt)^k, each relative to max(1, |t|)^k."""
    y = np.array([1.0, t, t * t, t ** 3])
    K = np.zeros(4)
    worst = 0.0
    for s in range(5):
        ts = t + LSERK_C[s] * dt
        sc = max(1.0, abs(ts)) ** np.arange(4)
        if s > 0:
            worst = max(worst, np.max(np.abs(y - ts ** np.arange(4)) / sc))
        K = LSERK_A[s] * K + dt * np.array([0.0, 1.0, 2.0 * ts, 3.0 * ts * ts])
        y = y + LSERK_B[s] * K
    te = t + dt
    end = np.max(np.abs(y - te ** np.arange(4)) / max(1.0, abs(te)) ** np.arange(4))
    return worst, end


@pytest.mark.parametrize("t", [0.0, 0.01, 2.5])
def test_stage_values_of_the_powers_of_t(t):
    """The scheme is fourth order, so its step integrates the cubic
    polynomials t^k exactly up to the accuracy of its published coefficient
    rationals (the end values are the powers of t + dt to about 1e-15 at
    dt <= 1e-3); its internal stages are low order, so the stage values miss
    t_s^k by O(dt^2).  A step may therefore carry M Q into the next step,
    and a stage's factor may stand in for one of M(t_s), only at small dt --
    the library checks both per step (1e-14 and 1e-6)."""
    for dt in (6.6e-4, 1e-3):
        worst, end = _stage_values_of_powers(t, dt)
        assert end < 1e-14, (dt, end)
        assert 1e-10 < worst < 1e-6, (dt, worst)
    worst, end = _stage_values_of_powers(t, 0.01)
    assert worst > 1e-6 and end > 1e-14
    # the stage deviation shrinks like dt^2
    w1, _ = _stage_values_of_powers(t, 1e-3)
    w2, _ = _stage_values_of_powers(t, 5e-4)
    assert 3.5 < w1 / w2 < 4.5


def test_conservation_in_motion():
    mo, _ = moving("mixed", 2, 2)
    Q = mo.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1), 0.0)
    before = mo.integral(Q, 0.0)
    after = mo.integral(mo.run(Q, 0.0, 0.02, 2), 0.04)
    assert np.abs(after - before).max() < 1e-13 * np.abs(before).max()


def test_convergence_on_a_moving_mesh():
    """The advected density wave is exact in physical space: on a mixed mesh
    in motion (N = 2, 2^3 -> 4^3 cubes, two steps) the density error
    converges at the static mesh's rate (above N + 0.2)."""
    N, T, errs = 2, 0.04, []
    for m in (2, 4):
        box = di.perturb_vertices(di.box_mesh(m, "mixed", seed=1), 0.05, smooth=True)
        mo = MovingOracle(box, N, di.vertex_velocities(box.xyz, 0.5))
        Q = mo.run(mo.project(di.advected_density_state, 0.0), 0.0, T / 2, 2)
        o = mo.at(T)
        err = 0.0
        for e in range(o.mesh.n_elems):
            et = o.mesh.etype[e]
            pts, w = volume_rule(et, N + 3)
            Jq, _ = o.mesh.volume_geometry(e, pts)
            rho_h = (o.mesh.block(Q, e) @ eval_basis(et, N, pts).T)[0]
            rho = di.advected_density_state(o.mesh.to_physical(e, pts), t=T)[0]
            err += (w * Jq) @ (rho_h - rho) ** 2
        errs.append(math.sqrt(err))
    assert math.log2(errs[0] / errs[1]) > N + 0.2, errs


# ---------------------------------------------------------------- Navier-Stokes (m7)
def test_ns_zero_velocity_is_the_static_curved_ns_oracle():
    from oracle.curved import CurvedNSOracle
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    N, mu = 2, 0.05
    mo = MovingOracle(box, N, np.zeros_like(box.xyz), mu=mu)
    co = CurvedNSOracle(curved_from_box(box, N), mu=mu, Pr=0.72)
    Q = co.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    R, Rref = mo.rhs(Q, 0.0), co.rhs(Q)
    assert np.abs(R - Rref).max() <= 1e-14 * np.abs(Rref).max()


def test_ns_with_zero_viscosity_is_the_euler_moving_oracle():
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 0.3)
    a = MovingOracle(box, 2, vel, mu=0.0)
    b = MovingOracle(box, 2, vel)
    Q = b.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1), 0.0)
    np.testing.assert_array_equal(a.rate(Q, 0.07), b.rate(Q, 0.07))


def test_ns_free_stream_and_conservation_in_motion():
    """The viscous terms vanish on a constant state, so the discrete GCL keeps
    it constant through LSERK steps in motion; the Navier-Stokes residual
    conserves int J q (central viscous face flux)."""
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    mo = MovingOracle(box, 2, di.vertex_velocities(box.xyz, 0.3), mu=0.05)
    Qc = constant(mo)
    Q2 = mo.run(Qc, 0.0, 0.05, 2)
    assert np.abs(Q2 - Qc).max() < 1e-13 * np.abs(Qc).max()
    Q = mo.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1), 0.0)
    before = mo.integral(Q, 0.0)
    after = mo.integral(mo.run(Q, 0.0, 0.02, 2), 0.04)
    assert np.abs(after - before).max() < 1e-13 * np.abs(before).max()
