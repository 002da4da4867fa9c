"""Modal DG right-hand side, projection (Algorithm 1) and LSERK(5,4).

For element e of type T with modal coefficients Q_e [5, nM] the weak form of
Eq. 1 reads M_e dQ_e/dt = vol_e - surf_e with
  vol_e[:, i]  = sum_q w_q J_e sum_d (d phi_i / d x_d)(xi_q) F_d(U_q)
  surf_e[:, i] = sum_faces sum_p (w S)_p phi_i(x_p) (F.n)*_p      (owner side)
               = - sum_p (w S)_p phi_i(x_p) (F.n)*_p                (neighbour)
  M_e          = J_e V^T W V                                        (Algorithm 1)
U_q is the modal expansion evaluated directly at the quadrature point.  The
flux (F.n)* is evaluated once per face point, at the owner's points, with the
owner's outward normal.  R_e = M_e^{-1}(vol_e - surf_e) by a Cholesky solve.

Projection (Algorithm 1): Q = M^{-1} V^T W J q for values q at the volume
points.  Time integration: LSERK(5,4) of Carpenter & Kennedy (1994), 2N-storage,
K <- A_s K + dt R(Q); Q <- Q + B_s K, K = 0 at the start of every step.

The residual is assembled element by element ('gather' form): an element's
face terms are computed from its own faces, so any subset of elements can be
evaluated alone (used for sampled checks on large meshes).

Parity: pinned by free-stream preservation, discrete conservation, convergence
order, and the nodal Algorithm-1 cross-check (tests/test_oracle_dg.py).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from .elements import eval_basis
from .euler import physical_flux, riemann
from .quadrature import volume_rule

# Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage RK, "solution 3".
LSERK_A = np.array([0.0,
                    -567301805773.0 / 1357537059087.0,
                    -2404267990393.0 / 2016746695238.0,
                    -3550918686646.0 / 2091501179385.0,
                    -1275806237668.0 / 842570457699.0])
LSERK_B = np.array([1432997174477.0 / 9575080441755.0,
                    5161836677717.0 / 13612068292357.0,
                    1720146321549.0 / 2090206949498.0,
                    3134564353537.0 / 4481467310338.0,
                    2277821191437.0 / 14882151754819.0])


class TypeOps:
    """Per-(type, N) volume tables: V [nQ, nM], grad_xi V [3, nQ, nM], w [nQ], M_ref."""

    def __init__(self, etype, N):
        self.pts, self.w = volume_rule(etype, N)
        self.V, self.G = eval_basis(etype, N, self.pts, grad=True)
        self.Mref = self.V.T @ (self.w[:, None] * self.V)
        self.chol = cho_factor(self.Mref)


class Oracle:
    def __init__(self, mesh, flux="lf", gamma=1.4):
        self.mesh = mesh
        self.flux = flux
        self.gamma = gamma
        self.ops = {t: TypeOps(t, mesh.N) for t in sorted(set(mesh.etype.tolist()))}
        self._face_cache = {}

    # ------------------------------------------------------------ helpers
    def face_data(self, f):
        if f not in self._face_cache:
            m = self.mesh
            e0, l0, e1, l1 = m.faces[f]
            ref0, ref1, wS, nrm = m.face_geometry(f)
            phi0 = eval_basis(m.etype[e0], m.N, ref0)
            phi1 = eval_basis(m.etype[e1], m.N, ref1)
            self._face_cache[f] = (phi0, phi1, wS, nrm)
        return self._face_cache[f]

    def face_flux(self, Q, f):
        """(w S)_p (F.n)*_p at the owner's points of face f: [5, n^2]."""
        m = self.mesh
        e0, _, e1, _ = m.faces[f]
        phi0, phi1, wS, nrm = self.face_data(f)
        UL = m.block(Q, e0) @ phi0.T
        UR = m.block(Q, e1) @ phi1.T
        return wS * riemann(self.flux, UL, UR, nrm, self.gamma)

    def volume_term(self, Q, e):
        m = self.mesh
        op = self.ops[m.etype[e]]
        U = m.block(Q, e) @ op.V.T                       # [5, nQ]
        F = physical_flux(U, self.gamma)                 # [3(d), 5, nQ]
        g = m.dxi_dx[e]                                  # [3(k), 3(d)]
        Fc = np.einsum("kd,dvq->kvq", g, F)             # sum_d dxi_k/dx_d F_d
        return m.J[e] * np.einsum("kqi,kvq->vi", op.G, op.w * Fc)

    def surface_term(self, Q, e, fluxes=None):
        m = self.mesh
        s = np.zeros((5, m.nM[e]), dtype=Q.dtype)
        for f, side in m.elem_faces[e]:
            phi0, phi1, _, _ = self.face_data(f)
            Fh = fluxes[f] if fluxes is not None else self.face_flux(Q, f)
            s = s + (Fh @ phi0 if side == 0 else -(Fh @ phi1))
        return s

    def apply_minv(self, e, r):
        op = self.ops[self.mesh.etype[e]]
        if np.iscomplexobj(r):
            return (cho_solve(op.chol, r.real.T).T + 1j * cho_solve(op.chol, r.imag.T).T) / self.mesh.J[e]
        return cho_solve(op.chol, r.T).T / self.mesh.J[e]

    # ------------------------------------------------------------ public
    def rhs(self, Q, elems=None):
        """R in caller layout; with elems, only those elements' blocks are filled."""
        m = self.mesh
        Q = np.asarray(Q)
        R = np.zeros_like(Q)
        elems = range(m.n_elems) if elems is None else elems
        needed = sorted({f for e in elems for f, _ in m.elem_faces[e]})
        fluxes = {f: self.face_flux(Q, f) for f in needed}
        for e in elems:
            r = self.volume_term(Q, e) - self.surface_term(Q, e, fluxes)
            R[m.dof_off[e]:m.dof_off[e + 1]] = self.apply_minv(e, r).ravel()
        return R

    def quad_points(self, e):
        op = self.ops[self.mesh.etype[e]]
        return self.mesh.to_physical(e, op.pts)

    def project(self, values_at_points):
        """Algorithm 1 projection Q = M^{-1} V^T W J q; values_at_points(x[nQ,3]) -> [5, nQ]."""
        m = self.mesh
        Q = np.zeros(m.n_dof())
        for e in range(m.n_elems):
            op = self.ops[m.etype[e]]
            q = values_at_points(self.quad_points(e))
            r = m.J[e] * (q * op.w) @ op.V
            Q[m.dof_off[e]:m.dof_off[e + 1]] = self.apply_minv(e, r).ravel()
        return Q

    def evaluate(self, Q, e, ref_pts):
        return self.mesh.block(Q, e) @ eval_basis(self.mesh.etype[e], self.mesh.N, ref_pts).T

    def integrate(self, Q, e):
        """int_e U dx by the volume rule: [5]."""
        op = self.ops[self.mesh.etype[e]]
        return self.mesh.J[e] * (self.mesh.block(Q, e) @ op.V.T) @ op.w

    def lserk_step(self, Q, dt, stages_out=None):
        K = np.zeros_like(Q)
        for s in range(5):
            if stages_out is not None:
                stages_out.append(Q.copy())
            K = LSERK_A[s] * K + dt * self.rhs(Q)
            Q = Q + LSERK_B[s] * K
        return Q

    def run(self, Q, dt, nsteps):
        for _ in range(nsteps):
            Q = self.lserk_step(Q, dt)
        return Q
