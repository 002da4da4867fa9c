"""Time-varying geometry: the moving-mesh (arbitrary Lagrangian-Eulerian)
form of Eq. 1 with the projection of Algorithm 1 solved afresh at every
stage, because the Jacobian changes with time (Sec. 2: the mesh may move;
Algorithm 1 notes that the projection then cannot be precomputed).

Readings (the paper prints no moving-mesh scheme; shared with the library):
  * m1 motion: every mesh vertex moves at a constant velocity,
    x_v(t) = x_v + t u_v, with u_v the same for periodic images; every
    element is the vertex interpolant of its reference element at every time
    (the curved-element reading), so dx/dxi is linear in t, J(t) a cubic and
    the contravariant metric J dxi/dx a quadratic in t at every point.
  * m2 weak form in the moving frame: for every test function phi_i,
      d/dt int J q phi_i dxi + oint (F.n - (xdot.n) q)* phi_i dS
        - int J (dxi/dx)(F(q) - q xdot) . grad_xi phi_i dxi = 0,
    xdot = sum_v N_v(xi) u_v the mesh velocity.
  * m3 surface flux: Lax-Friedrichs in the moving frame,
      (F(U-).n - s U- + F(U+).n - s U+)/2 - lam (U+ - U-)/2,
      s = xdot.n at the face point, lam = max(|u-.n - s| + c-, |u+.n - s| + c+).
  * m4 modal time stepping with a time-dependent J (Algorithm 1): the
    evolved unknown is the mass-weighted modal vector Ut = M Q,
    M = V^T diag(w J) V per element; at every stage the projection
    Q = M^{-1} Ut is solved afresh (Cholesky), the residual of m2 evaluated at
    the stage time t_s = t_n + c_s dt (the published c_s of LSERK(5,4)) and Ut
    advanced by the LSERK stage.
  * m5 geometric conservation: the Jacobian in the stage's mass matrix is the
    LSERK stage value of J, i.e. dJ/dt = div_xi(J dxi/dx xdot) integrated by
    the same stages as the solution (a discrete geometric conservation law).
    J(t) is a cubic in t at every point, so the stage value is
    J^_s = sum_k y_k,s J_k with J(t) = sum_k J_k t^k and y_k,s the LSERK stage
    value of t^k; it equals J(t) at every step's end.  With it a constant
    state stays constant to rounding: the residual of a constant state is
    exactly the time derivative of its moments int phi_i J dxi (the collapsed
    rule integrates those polynomial integrands exactly), so every stage's
    Ut is exactly M^_s times the constant.  (With the Jacobian at the stage
    time t_s instead, a constant state drifts by O(dt^5) per step.)
  * m6 hexahedra, prisms and pyramids (the types whose maps the motion
    bends); LF surface flux.
  * m7 Navier-Stokes (BR1) on a moving mesh: the lifted gradient of W is a
    physical-space gradient, so the lifting is the static curved one on the
    geometry of the stage time (the BR1 reading of the Navier-Stokes
    oracle); the viscous flux and its central face flux are unchanged; only
    the convective flux moves to the moving frame (volume F(q) - q xdot,
    face the moving-frame LF flux of m3).

Parity: pinned by tests/test_oracle_moving.py -- zero velocity reduces to the
static curved oracle (Euler and Navier-Stokes); a constant state stays constant through LSERK steps on
a mesh in motion (m5); the total of int J q over the mesh is conserved; the
residual of a constant state equals the time derivative of the moments
int J phi_i (central difference in t); and the advected density wave, an
exact solution in physical space, converges on a moving mesh.
Test infrastructure only, like the rest of the oracle.
"""
from __future__ import annotations

import copy

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from .curved import CurvedNSOracle, CurvedOracle, curved_from_box, shape_functions
from .dg import LSERK_A, LSERK_B
from .elements import TET
from .euler import physical_flux, pressure, rabs, rmax
from .navier_stokes import viscous_flux

# Carpenter & Kennedy (1994), (5,4) "solution 3": the stage times
LSERK_C = np.array([0.0,
                    1432997174477.0 / 9575080441755.0,
                    2526269341429.0 / 6820363183857.0,
                    2006345519317.0 / 3224310063776.0,
                    2802321613138.0 / 2924317926251.0])


def ale_lax_friedrichs(UL, UR, n, s, gamma):
    """m3: LF flux in a frame moving with normal speed s."""
    n = np.asarray(n)

    def side(U):
        F = physical_flux(U, gamma)
        Fn = sum(F[d] * n[d] for d in range(3)) - s * U
        un = (U[1] * n[0] + U[2] * n[1] + U[3] * n[2]) / U[0]
        c = np.sqrt(gamma * pressure(U, gamma) / U[0])
        return Fn, rabs(un - s) + c
    FL, lL = side(UL)
    FR, lR = side(UR)
    lam = rmax(lL, lR)
    return 0.5 * (FL + FR) - 0.5 * lam * (UR - UL)


class MovingOracle:
    """Eq. 1 in the moving frame on a box whose vertices move at the constant
    velocities `vel` [n_vertices, 3] (readings m1-m7).  States are modal
    coefficients Q in caller layout at a given time; the LSERK steps evolve
    the mass-weighted Ut = M(t) Q internally.  mu = None: the Euler
    equations; a viscosity mu (and Prandtl number Pr): Navier-Stokes (m7)."""

    def __init__(self, box, N, vel, flux="lf", gamma=1.4, mu=None, Pr=0.72):
        if flux != "lf":
            raise ValueError("the moving-mesh reading takes the LF flux")
        if np.any(np.asarray(box.etype) == TET):
            raise ValueError("the moving-mesh reading covers hexahedra, prisms and pyramids")
        self.box, self.N, self.gamma = box, int(N), gamma
        self.mu, self.Pr = mu, Pr
        self.vel = np.asarray(vel, dtype=float)
        self._at = {}
        base = self.at(0.0)
        self.mesh = base.mesh          # connectivity and layout (the same at every time)

    def at(self, t):
        """The curved oracle of the mesh at time t (cached)."""
        t = float(t)
        if t not in self._at:
            b = copy.copy(self.box)
            b.xyz = np.asarray(self.box.xyz, dtype=float) + t * self.vel
            cm = curved_from_box(b, self.N)
            if self.mu is None:
                self._at[t] = CurvedOracle(cm, flux="lf", gamma=self.gamma)
            else:
                self._at[t] = CurvedNSOracle(cm, flux="lf", gamma=self.gamma, mu=self.mu, Pr=self.Pr)
        return self._at[t]

    def mesh_velocity(self, o, e, ref):
        """xdot at reference points of element e: [3, P]."""
        m = o.mesh
        return (shape_functions(m.etype[e], np.atleast_2d(ref)) @ self.vel[m.verts[e]]).T

    # ------------------------------------------------------------ residual (m2, m3)
    def rate(self, Q, t, elems=None):
        """vol - surf at time t: the time derivative of Ut = M(t) Q (with
        elems, only those elements' blocks, from the faces they touch)."""
        o = self.at(t)
        m = o.mesh
        R = np.zeros_like(np.asarray(Q, dtype=float))
        elems = list(range(m.n_elems)) if elems is None else list(elems)
        faces1 = sorted({f for e in elems for f, _ in m.elem_faces[e]})
        G = None
        if self.mu is not None:
            # m7: the BR1 lifted gradient on the geometry of time t, for the
            # elements whose traces the faces need
            lift_elems = sorted({x for f in faces1 for x in (m.faces[f][0], m.faces[f][2])})
            faces2 = sorted({f for e in lift_elems for f, _ in m.elem_faces[e]})
            wstar = {f: o.face_wstar(Q, f) for f in faces2}
            G = {e: o.lifting(Q, e, wstar) for e in lift_elems}
        fluxes = {}
        for f in faces1:
            e0, l0, e1, _ = m.faces[f]
            phi0, phi1, wS, nrm = o.face_data(f)
            ref0 = m.face_geometry(f)[0]
            s = np.einsum("dp,dp->p", self.mesh_velocity(o, e0, ref0), nrm)
            UL, UR = m.block(Q, e0) @ phi0.T, m.block(Q, e1) @ phi1.T
            Fs = ale_lax_friedrichs(UL, UR, nrm, s, self.gamma)
            if G is not None:
                Fv = 0.5 * (viscous_flux(UL, G[e0] @ phi0.T, self.gamma, self.mu, self.Pr)
                            + viscous_flux(UR, G[e1] @ phi1.T, self.gamma, self.mu, self.Pr))
                Fs = Fs - np.einsum("dp,dvp->vp", nrm, Fv)
            fluxes[f] = wS * Fs
        for e in elems:
            op = o.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T                                   # [5, nQ]
            F = physical_flux(U, self.gamma)                             # [3(d), 5, nQ]
            F = F - self.mesh_velocity(o, e, op.pts)[:, None, :] * U[None]
            if G is not None:
                F = F - viscous_flux(U, G[e] @ op.V.T, self.gamma, self.mu, self.Pr)
            Fc = np.einsum("qkd,dvq->kvq", o.dxi_dx[e], F)
            vol = np.einsum("kqi,kvq->vi", op.G, (op.w * o.Jq[e]) * Fc)
            R[m.dof_off[e]:m.dof_off[e + 1]] = (vol - o.surface_term(Q, e, fluxes)).ravel()
        return R

    # ------------------------------------------------------------ mass matrix (m4, m5)
    def jacobian(self, e, t, y=None, h=None):
        """J at the volume points of element e: J(t), or with stage values y
        (y_k standing for t^k) J^ = sum_k y_k J_k of the cubic J(t) =
        sum_k J_k t^k, written as the combination of J at the four times
        t + c_s h (s = 0..3, the first LSERK stage times of the step from t)
        that reproduces every cubic, so only values of J are needed."""
        if y is None:
            return self.at(t).Jq[e]
        taus = t + h * LSERK_C[:4]
        coef = np.linalg.solve(np.vander(taus, 4, increasing=True).T, np.asarray(y, dtype=float))
        return sum(c * self.at(tau).Jq[e] for c, tau in zip(coef, taus))

    def mass(self, e, t, y=None, h=None):
        op = self.at(t).ops[self.mesh.etype[e]]
        return op.V.T @ ((op.w * self.jacobian(e, t, y, h))[:, None] * op.V)

    def weighted(self, Q, t, y=None, h=None):
        """Ut = M Q per element, M with J(t) (or J^ of the stage values y of
        the step from t of length h)."""
        m = self.mesh
        out = np.zeros_like(Q)
        for e in range(m.n_elems):
            out[m.dof_off[e]:m.dof_off[e + 1]] = (m.block(Q, e) @ self.mass(e, t, y, h)).ravel()
        return out

    def unweighted(self, Ut, t, y=None, h=None, elems=None):
        """Q = M^{-1} Ut per element (Cholesky), M as in weighted (with elems,
        only those elements)."""
        m = self.mesh
        out = np.zeros_like(Ut)
        for e in (range(m.n_elems) if elems is None else elems):
            c = cho_factor(self.mass(e, t, y, h))
            out[m.dof_off[e]:m.dof_off[e + 1]] = cho_solve(c, m.block(Ut, e).T).T.ravel()
        return out

    def rhs(self, Q, t, elems=None):
        """M(t)^{-1} (vol - surf) (what the library's dg_rhs returns on a mesh
        in motion); with elems, only those elements' blocks."""
        return self.unweighted(self.rate(Q, t, elems), t, elems=elems)

    def project(self, fn, t):
        return self.at(t).project(fn)

    def lserk_step(self, Q, t, dt):
        """One LSERK(5,4) step of Ut from t to t + dt (m4, m5): the stage value
        y_k of t^k runs through the same 2N-storage recursion as Ut."""
        Ut = self.weighted(Q, t)
        K = np.zeros_like(Ut)
        y = np.array([t ** k for k in range(4)])
        Ky = np.zeros(4)
        for s in range(5):
            ts = t + LSERK_C[s] * dt
            Q_s = self.unweighted(Ut, t, y=y, h=dt)
            K = LSERK_A[s] * K + dt * self.rate(Q_s, ts)
            Ut = Ut + LSERK_B[s] * K
            Ky = LSERK_A[s] * Ky + dt * np.array([k * ts ** (k - 1) if k else 0.0 for k in range(4)])
            y = y + LSERK_B[s] * Ky
        return self.unweighted(Ut, t, y=y, h=dt)

    def run(self, Q, t, dt, nsteps):
        for k in range(nsteps):
            Q = self.lserk_step(Q, t + k * dt, dt)
        return Q

    def integral(self, Q, t):
        """int J q over the mesh at time t: [5]."""
        o = self.at(t)
        return sum(o.integrate(Q, e) for e in range(o.mesh.n_elems))

