"""Curved (non-affine) elements for the oracle: pointwise J in Eq. 1 and in
the projection of Algorithm 1.

Sec. 2 writes the weak form on elements mapped by x = chi(xi) with a
pointwise Jacobian J and contravariant metric terms, and notes with
Algorithm 1 that the projection M^{-1} V^T W J cannot be formed once per
element type when J varies.  The affine oracle (oracle.mesh, oracle.dg) covers
the case J = const per element; this module drops that restriction.

Element maps (a reading: the paper names no geometry representation beyond
x = chi(xi)).  Each element is the vertex interpolant of its reference element,
x = sum_v N_v(xi) X_v, with
  hex      N_v = prod_d (1 + r_vd xi_d) / 2            (trilinear; r_v = reference vertex)
  prism    N_i = l_i(xi, eta) (1 - zeta)/2,  N_{i+3} = l_i(xi, eta) (1 + zeta)/2,
           l_0 = -(xi + eta)/2, l_1 = (1 + xi)/2, l_2 = (1 + eta)/2
  pyramid  N_v = (1 + r_v0 a)/2 (1 + r_v1 b)/2 (1 - c)/2 for the base, N_4 = (1 + c)/2,
           in the collapsed coordinates (a, b, c) of the pyramid
  tet      barycentric (affine)
so quadrilateral faces are bilinear and triangular faces planar, and two
elements that share a face's vertices share the face exactly.  d x / d xi is
taken by complex-step differentiation of the map (exact to rounding).

Per volume point q of element e: J_q = |det dx/dxi| and dxi/dx = (dx/dxi)^{-1};
the volume term is sum_q w_q J_q sum_d (d phi_i / d x_d)(xi_q) F_d(U_q), the
mass matrix M_e = V^T diag(w_q J_q) V (dense for every type), and the
projection Q = M_e^{-1} V^T W J q (Algorithm 1, J pointwise).

Faces: the owner's face points as in the affine case; at each point the area
vector is w_p |t_s x t_t| |det F| F^{-T} N (Nanson's formula with the
reference outward unit normal N and reference tangents t_s, t_t of the face
parametrisation, F = dx/dxi at the point); (w S)_p is its length and the
normal its direction.  The neighbour's reference coordinates of each owner
face point are found by Newton's method on the neighbour's map.

The adjoint (rhs_vjp) is the transpose of each of these steps.
CurvedNSOracle carries the Navier-Stokes residual with BR1 lifting of
oracle.navier_stokes onto curved elements (pointwise metric and normals).

Parity: pinned by reduction to the affine oracle on affine meshes, the
divergence theorem on every element, the total volume of the box, free-stream
preservation, conservation, reproduction of the element maps by the
projection, convergence of order about N+1 under a smooth deformation, and
for the adjoint the dot-product test against complex-step directional
derivatives of the residual and of K LSERK steps
(tests/test_oracle_curved.py).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_factor, cho_solve

from .dg import Oracle
from .elements import FACES, HEX, PRISM, PYR, REF_VERTS, TET, eval_basis, n_modes
from .euler import physical_flux, riemann
from .mesh import OracleMesh
from .navier_stokes import NSOracle, _cs, primitive, viscous_flux
from .quadrature import face_rule

H_CS = 1e-30


def shape_functions(etype, pts):
    """N_v at reference points pts [P, 3] (real or complex): [P, nv]."""
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    R = REF_VERTS[etype]
    if etype == HEX:
        return np.stack([(1 + R[v, 0] * xi) * (1 + R[v, 1] * eta) * (1 + R[v, 2] * zeta) / 8
                         for v in range(8)], axis=1)
    if etype == PRISM:
        lam = [-(xi + eta) / 2, (1 + xi) / 2, (1 + eta) / 2]
        return np.stack([lam[i] * (1 - zeta) / 2 for i in range(3)] +
                        [lam[i] * (1 + zeta) / 2 for i in range(3)], axis=1)
    if etype == TET:
        return np.stack([-(1 + xi + eta + zeta) / 2, (1 + xi) / 2, (1 + eta) / 2, (1 + zeta) / 2], axis=1)
    if etype == PYR:
        a = 2 * (1 + xi) / (1 - zeta) - 1
        b = 2 * (1 + eta) / (1 - zeta) - 1
        base = [(1 + R[v, 0] * a) / 2 * (1 + R[v, 1] * b) / 2 * (1 - zeta) / 2 for v in range(4)]
        return np.stack(base + [(1 + zeta) / 2], axis=1)
    raise ValueError(etype)


class CurvedOracleMesh(OracleMesh):
    """OracleMesh without the affine restriction (element maps as above)."""

    def __init__(self, xyz, etype, elem_vert_off, elem_verts, period, N):
        self.xyz = np.asarray(xyz, dtype=float)
        self.etype = np.asarray(etype, dtype=np.int64)
        self.N = int(N)
        self.period = None if period is None else np.asarray(period, dtype=float)
        off = np.asarray(elem_vert_off)
        ev = np.asarray(elem_verts)
        E = self.etype.size
        self.n_elems = E
        self.verts = [ev[off[e]:off[e + 1]] for e in range(E)]
        for e in range(E):
            if self.verts[e].size != REF_VERTS[self.etype[e]].shape[0]:
                raise ValueError(f"element {e}: wrong vertex count")
        self.nM = np.array([n_modes(t, N) for t in self.etype])
        self.dof_off = np.zeros(E + 1, dtype=np.int64)
        self.dof_off[1:] = np.cumsum(5 * self.nM)
        self.centroid = np.array([self.xyz[v].mean(0) for v in self.verts])
        self._match_faces()

    # ------------------------------------------------------------ maps
    def _rel(self, e):
        """Vertex positions relative to the element's first vertex."""
        X = self.xyz[self.verts[e]]
        return X - X[0]

    def to_physical_rel(self, e, ref):
        """chi_e(ref) - X_{v0}: [P, 3] (real or complex ref)."""
        ref = np.atleast_2d(ref)
        return shape_functions(self.etype[e], ref) @ self._rel(e)

    def to_physical(self, e, ref):
        return self.xyz[self.verts[e][0]] + self.to_physical_rel(e, ref)

    def jacobian(self, e, ref):
        """F = dx/dxi at reference points: [P, 3(x_d), 3(xi_k)]."""
        ref = np.atleast_2d(np.asarray(ref, dtype=float))
        cols = []
        for k in range(3):
            d = np.zeros(3, dtype=complex)
            d[k] = 1j * H_CS
            cols.append(self.to_physical_rel(e, ref + d).imag / H_CS)
        return np.stack(cols, axis=2)

    def volume_geometry(self, e, pts):
        """J_q = |det F| and dxi/dx = F^{-1} at the volume points."""
        F = self.jacobian(e, pts)
        det = np.linalg.det(F)
        if not (np.all(det > 0) or np.all(det < 0)):
            raise ValueError(f"element {e} is inverted or degenerate at a quadrature point")
        return np.abs(det), np.linalg.inv(F)

    def to_reference(self, e, x_rel, guess):
        """Newton's method for chi_e(xi) - X_{v0} = x_rel, per row."""
        xi = np.array(guess, dtype=float)
        for _ in range(60):
            r = self.to_physical_rel(e, xi) - x_rel
            F = self.jacobian(e, xi)
            step = np.linalg.solve(F, r[..., None])[..., 0]
            xi = xi - step
            if np.abs(step).max() < 1e-15:
                break
        return xi

    def face_geometry(self, f):
        """Owner reference points, neighbour reference points of the same
        physical points, (w S)_p and outward unit normals [3, P]."""
        e0, l0, e1, l1 = self.faces[f]
        t0 = self.etype[e0]
        ref0, w, ts, tt = face_rule(t0, l0, self.N)
        # reference outward unit normal of the face
        nr = np.cross(ts, tt)
        nr = nr / np.linalg.norm(nr)
        cen = REF_VERTS[t0][FACES[t0][l0]].mean(0) - REF_VERTS[t0].mean(0)
        if np.dot(nr, cen) < 0:
            nr = -nr
        F = self.jacobian(e0, ref0)
        det = np.abs(np.linalg.det(F))
        area = (w * np.linalg.norm(np.cross(ts, tt)) * det)[:, None] * \
            np.einsum("pkd,k->pd", np.linalg.inv(F), nr)        # |det F| F^{-T} N, scaled
        wS = np.linalg.norm(area, axis=1)
        nrm = (area / wS[:, None]).T
        shift = np.zeros(3)
        if self.period is not None:
            d = self.face_centroid(e0, l0) - self.face_centroid(e1, l1)
            shift = np.rint(d / self.period) * self.period
        x_rel = (self.xyz[self.verts[e0][0]] - shift - self.xyz[self.verts[e1][0]]) + \
            self.to_physical_rel(e0, ref0)
        t1 = self.etype[e1]
        guess = np.tile(REF_VERTS[t1][FACES[t1][l1]].mean(0), (ref0.shape[0], 1))
        ref1 = self.to_reference(e1, x_rel, guess)
        return ref0, ref1, wS, nrm


def curved_from_box(box, N):
    return CurvedOracleMesh(box.xyz, box.etype, box.elem_vert_off, box.elem_verts, box.period, N)


class _PerElement:
    """e -> field(e), computed on first use (large meshes are checked on
    sampled elements only)."""

    def __init__(self, fill):
        self._fill = fill
        self._vals = {}

    def __getitem__(self, e):
        e = int(e)
        if e not in self._vals:
            self._fill(e)
        return self._vals[e]


class CurvedOracle(Oracle):
    """Oracle (Eq. 1, Algorithm 1, LSERK) on a CurvedOracleMesh.  Per
    element: Jq [nQ], dxi_dx [nQ, 3(xi_k), 3(x_d)] and the Cholesky factor of
    M_e = V^T diag(w J) V."""

    def __init__(self, mesh, flux="lf", gamma=1.4):
        super().__init__(mesh, flux=flux, gamma=gamma)
        self.Jq = _PerElement(self._element_geometry)
        self.dxi_dx = _PerElement(self._element_geometry)
        self.chol = _PerElement(self._element_geometry)

    def _element_geometry(self, e):
        op = self.ops[self.mesh.etype[e]]
        Jq, G = self.mesh.volume_geometry(e, op.pts)
        self.Jq._vals[e] = Jq
        self.dxi_dx._vals[e] = G
        self.chol._vals[e] = cho_factor(op.V.T @ ((op.w * Jq)[:, None] * op.V))

    def face_data(self, f):
        if f not in self._face_cache:
            m = self.mesh
            e0, l0, e1, l1 = m.faces[f]
            ref0, ref1, wS, nrm = m.face_geometry(f)
            phi0 = eval_basis(m.etype[e0], m.N, ref0)
            phi1 = eval_basis(m.etype[e1], m.N, ref1)
            self._face_cache[f] = (phi0, phi1, wS, nrm)
        return self._face_cache[f]

    def volume_term(self, Q, e):
        m = self.mesh
        op = self.ops[m.etype[e]]
        U = m.block(Q, e) @ op.V.T                       # [5, nQ]
        F = physical_flux(U, self.gamma)                 # [3(d), 5, nQ]
        Fc = np.einsum("qkd,dvq->kvq", self.dxi_dx[e], F)
        return np.einsum("kqi,kvq->vi", op.G, (op.w * self.Jq[e]) * Fc)

    def apply_minv(self, e, r):
        c = self.chol[e]
        if np.iscomplexobj(r):
            return cho_solve(c, r.real.T).T + 1j * cho_solve(c, r.imag.T).T
        return cho_solve(c, r.T).T

    def project(self, values_at_points):
        m = self.mesh
        Q = np.zeros(m.n_dof())
        for e in range(m.n_elems):
            op = self.ops[m.etype[e]]
            q = values_at_points(self.quad_points(e))
            r = (q * (op.w * self.Jq[e])) @ op.V
            Q[m.dof_off[e]:m.dof_off[e + 1]] = self.apply_minv(e, r).ravel()
        return Q

    def integrate(self, Q, e):
        op = self.ops[self.mesh.etype[e]]
        return (self.mesh.block(Q, e) @ op.V.T) @ (op.w * self.Jq[e])

    def rhs_vjp(self, Q, Rbar):
        """(dR/dQ)^T Rbar: the transpose of every step of rhs on curved
        elements, with the pointwise metric in the volume term:
          rbar_e = M_e^{-1} Rbar_e (M_e symmetric)
          Fbar_d[v, q] = w_q J_q sum_k (dxi_k/dx_d)(q) sum_i (dphi_i/dxi_k)(q) rbar[v, i]
          Ubar[:, q] = sum_d (dF_d/dU)^T Fbar_d[:, q];  Qbar_e += Ubar V
        and the face part of oracle.adjoint with per-point w S and normals."""
        from .adjoint import cs_jacobian, face_vjp
        m = self.mesh
        Q = np.asarray(Q, dtype=float)
        Qbar = np.zeros_like(Q)
        rbar = {e: self.apply_minv(e, m.block(Rbar, e)) for e in range(m.n_elems)}
        for e in range(m.n_elems):
            op = self.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T
            Fbar = (op.w * self.Jq[e]) * np.einsum("qkd,kqi,vi->dvq", self.dxi_dx[e], op.G, rbar[e])
            JF = cs_jacobian(lambda X: physical_flux(X, self.gamma), U)
            Ubar = np.einsum("dvuq,dvq->uq", JF, Fbar)
            Qbar[m.dof_off[e]:m.dof_off[e + 1]] += (Ubar @ op.V).ravel()
        face_vjp(self, Q, rbar, Qbar)
        return Qbar

    def volume(self, e):
        op = self.ops[self.mesh.etype[e]]
        return float(op.w @ self.Jq[e])


class CurvedNSOracle(NSOracle, CurvedOracle):
    """Navier-Stokes residual with BR1 lifting (oracle.navier_stokes) on a
    CurvedOracleMesh: the lifting's volume term and the total flux use the
    pointwise metric, w_q J_q as the volume weight, and the face terms the
    per-point normals (the lifting face term multiplies W* by the normal at
    each face point before testing, the central viscous flux takes its normal
    component per point); M_e^{-1} is the curved element's dense inverse."""

    def lifting(self, Q, e, wstar):
        m = self.mesh
        op = self.ops[m.etype[e]]
        W = primitive(m.block(Q, e) @ op.V.T, self.gamma)               # [5, nQ]
        gx = np.einsum("qkd,kqi->dqi", self.dxi_dx[e], op.G)             # d phi_i / d x_d at q
        vol = np.einsum("dqi,vq->dvi", gx, (op.w * self.Jq[e]) * W)
        surf = np.zeros_like(vol)
        for f, side in m.elem_faces[e]:
            phi0, phi1, _, nrm = self.face_data(f)
            phi, sgn = (phi0, 1.0) if side == 0 else (phi1, -1.0)
            for d in range(3):
                surf[d] = surf[d] + sgn * ((nrm[d] * wstar[f]) @ phi)
        return np.stack([self.apply_minv(e, surf[d] - vol[d]) for d in range(3)])

    def ns_face_flux(self, Q, f, G):
        m = self.mesh
        e0, _, e1, _ = m.faces[f]
        phi0, phi1, wS, nrm = self.face_data(f)
        UL = m.block(Q, e0) @ phi0.T
        UR = m.block(Q, e1) @ phi1.T
        gL = G[e0] @ phi0.T
        gR = G[e1] @ phi1.T
        Fv = 0.5 * (viscous_flux(UL, gL, self.gamma, self.mu, self.Pr)
                    + viscous_flux(UR, gR, self.gamma, self.mu, self.Pr))
        Fvn = np.einsum("dp,dvp->vp", nrm, Fv)
        return wS * (riemann(self.flux, UL, UR, nrm, self.gamma) - Fvn)

    def ns_volume_term(self, Q, e, G):
        m = self.mesh
        op = self.ops[m.etype[e]]
        U = m.block(Q, e) @ op.V.T
        gradW = G[e] @ op.V.T
        F = physical_flux(U, self.gamma) - viscous_flux(U, gradW, self.gamma, self.mu, self.Pr)
        Fc = np.einsum("qkd,dvq->kvq", self.dxi_dx[e], F)
        return np.einsum("kqi,kvq->vi", op.G, (op.w * self.Jq[e]) * Fc)

    def rhs_vjp(self, Q, Rbar):
        """Qbar = (dR/dQ)^T Rbar: the steps of NSOracle.rhs_vjp with the
        pointwise metric and per-point normals."""
        m = self.mesh
        gam, mu, Pr = self.gamma, self.mu, self.Pr
        Q = np.asarray(Q, dtype=float)
        Qbar = np.zeros_like(Q)
        E, F = m.n_elems, len(m.faces)
        wstar = {f: self.face_wstar(Q, f) for f in range(F)}
        G = {e: self.lifting(Q, e, wstar) for e in range(E)}
        rbar = {e: self.apply_minv(e, m.block(Rbar, e)) for e in range(E)}
        Gbar = {e: np.zeros((3, 5, m.nM[e])) for e in range(E)}
        Wsbar = {f: np.zeros_like(wstar[f]) for f in range(F)}

        def add(e, vals):
            Qbar[m.dof_off[e]:m.dof_off[e + 1]] += vals.ravel()

        def vf_u(g):
            return lambda X: viscous_flux(X, g, gam, mu, Pr)

        def vf_g(U):
            return lambda Y: viscous_flux(U, Y, gam, mu, Pr)

        for e in range(E):
            op = self.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T
            gW = G[e] @ op.V.T
            Fbar = (op.w * self.Jq[e]) * np.einsum("qkd,kqi,vi->dvq", self.dxi_dx[e], op.G, rbar[e])
            JU = _cs(lambda X: physical_flux(X, gam), U) - _cs(vf_u(gW), U)
            JG = _cs(vf_g(U), gW)
            add(e, np.einsum("dvuq,dvq->uq", JU, Fbar) @ op.V)
            Gbar[e] += -np.einsum("dvxyq,dvq->xyq", JG, Fbar) @ op.V
        for f, (e0, _, e1, _) in enumerate(m.faces):
            phi0, phi1, wS, nrm = self.face_data(f)
            UL, UR = m.block(Q, e0) @ phi0.T, m.block(Q, e1) @ phi1.T
            gL, gR = G[e0] @ phi0.T, G[e1] @ phi1.T
            Fsbar = wS * (-(rbar[e0] @ phi0.T) + rbar[e1] @ phi1.T)
            JL = _cs(lambda X: riemann(self.flux, X, UR, nrm, gam), UL)
            JR = _cs(lambda X: riemann(self.flux, UL, X, nrm, gam), UR)
            Fvbar = -0.5 * nrm[:, None, :] * Fsbar[None]                         # [3, 5, P]
            ULbar = np.einsum("vup,vp->up", JL, Fsbar) + np.einsum("dvup,dvp->up", _cs(vf_u(gL), UL), Fvbar)
            URbar = np.einsum("vup,vp->up", JR, Fsbar) + np.einsum("dvup,dvp->up", _cs(vf_u(gR), UR), Fvbar)
            add(e0, ULbar @ phi0)
            add(e1, URbar @ phi1)
            Gbar[e0] += np.einsum("dvxyp,dvp->xyp", _cs(vf_g(UL), gL), Fvbar) @ phi0
            Gbar[e1] += np.einsum("dvxyp,dvp->xyp", _cs(vf_g(UR), gR), Fvbar) @ phi1
        for e in range(E):
            op = self.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T
            sbar = np.stack([self.apply_minv(e, Gbar[e][d]) for d in range(3)])
            gx = np.einsum("qkd,kqi->dqi", self.dxi_dx[e], op.G)
            Wbar = -(op.w * self.Jq[e]) * np.einsum("dqi,dvi->vq", gx, sbar)
            JW = _cs(lambda X: primitive(X, gam), U)
            add(e, np.einsum("wuq,wq->uq", JW, Wbar) @ op.V)
            for f, side in m.elem_faces[e]:
                phi0, phi1, _, nrm = self.face_data(f)
                phi, sgn = (phi0, 1.0) if side == 0 else (phi1, -1.0)
                for d in range(3):
                    Wsbar[f] += sgn * nrm[d] * (sbar[d] @ phi.T)
        for f, (e0, _, e1, _) in enumerate(m.faces):
            phi0, phi1, wS, _ = self.face_data(f)
            UL, UR = m.block(Q, e0) @ phi0.T, m.block(Q, e1) @ phi1.T
            a = 0.5 * wS * Wsbar[f]
            add(e0, np.einsum("wup,wp->up", _cs(lambda X: primitive(X, gam), UL), a) @ phi0)
            add(e1, np.einsum("wup,wp->up", _cs(lambda X: primitive(X, gam), UR), a) @ phi1)
        return Qbar


__all__ = ["CurvedOracle", "CurvedNSOracle", "CurvedOracleMesh", "curved_from_box", "shape_functions", "HEX", "PRISM", "PYR", "TET"]
