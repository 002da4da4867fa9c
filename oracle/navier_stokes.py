"""Navier-Stokes right-hand side with BR1 lifting (test infrastructure only).

The paper's weak form (Eq. 1) carries a flux F(q, grad q) that depends on the
solution gradient: its solver integrates the compressible Navier-Stokes-
Fourier equations (Sec. 2) and its benchmark is the viscous Taylor-Green
vortex at Re = 1600 (Sec. 4).  The paper does not print the viscous
discretisation; the reading taken here is the first Bassi-Rebay scheme
(BR1) on the primitive variables W = (rho, u, v, w, p):

  lifting, per element e, direction d and component v of W:
    int_e G_d phi J dxi = sum_faces int_f phi W* n_d dS - int_e W dphi/dx_d J dxi
    W* = (W- + W+)/2 at every face point,  n the element's outward normal,
  i.e. G_e = M_e^{-1} (surf_d - vol_d) with the mass matrix of Algorithm 1;
  G is the lifted gradient of W in the element's modal space.

  viscous flux (Stokes hypothesis, constant mu, Fourier heat flux):
    tau = mu (grad u + grad u^T - 2/3 div u I)
    q   = -kappa grad(p / rho),   kappa = mu gamma / ((gamma - 1) Pr)
    F_v[d] = (0, tau_{x d}, tau_{y d}, tau_{z d}, sum_i u_i tau_{i d} - q_d)
  with grad W taken from the lifted G (grad(p/rho) = (grad p - (p/rho) grad rho)/rho).

  residual: the Euler residual of the oracle's Eq. 1 with F -> F_e - F_v in the
  volume term and (F.n)* -> (F_e.n)* - (F_v(U-, G-) + F_v(U+, G+)).n / 2 at
  the faces (central viscous flux).  Both sides' U and G are evaluated at the
  owner's face points, the neighbour by its own expansion at those physical
  points, exactly as the inviscid face term.

Works on real or complex arrays (complex-step differentiation).  With mu = 0
the residual is the Euler residual.

Adjoint (rhs_vjp): the plain transpose of every step above, in reverse
order -- projection, volume flux (inviscid and viscous, with the viscous
flux's dependence on both U and the lifted gradient), face flux (Riemann and
central viscous parts), then the lifting (mass solve, volume and face terms)
and the face values W*; the pointwise Jacobians come from complex steps
through the functions of this module and oracle.euler.

Parity: pinned by exact lifting of linear W, exact residuals of polynomial
states against a symbolic strong-form residual, reduction to Euler at mu = 0,
free-stream preservation and conservation; the adjoint by the dense Jacobian
from complex steps through rhs (brute force) and the dot-product test
(tests/test_oracle_ns.py).
"""
from __future__ import annotations

import numpy as np

from .dg import Oracle
from .euler import physical_flux, riemann

H_CS = 1e-30


def _cs(fun, X):
    """Jacobian of fun at X by complex steps: X [*shape_in, P] -> [*shape_out, *shape_in, P]."""
    shape_in = X.shape[:-1]
    cols = []
    for idx in np.ndindex(*shape_in):
        dX = np.zeros(X.shape, dtype=complex)
        dX[idx] = 1.0
        cols.append(fun(X + 1j * H_CS * dX).imag / H_CS)
    out = np.stack(cols, axis=-2)                                 # [*out, prod(in), P]
    return out.reshape(out.shape[:-2] + shape_in + out.shape[-1:])


def primitive(U, gamma):
    rho, mx, my, mz, E = U
    u, v, w = mx / rho, my / rho, mz / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w))
    return np.stack([rho, u, v, w, p])


def viscous_flux(U, gradW, gamma, mu, Pr):
    """F_v[d] for d = x, y, z: [3, 5, ...]; gradW[d, v] = dW_v/dx_d."""
    W = primitive(U, gamma)
    rho, p = W[0], W[4]
    vel = W[1:4]
    du = gradW[:, 1:4]                      # du[d, i] = d u_i / d x_d
    div = du[0, 0] + du[1, 1] + du[2, 2]
    kappa = mu * gamma / ((gamma - 1.0) * Pr)
    F = []
    for d in range(3):
        tau = [mu * (du[d, i] + du[i, d]) - (2.0 / 3.0 * mu * div if i == d else 0.0) for i in range(3)]
        dT = (gradW[d, 4] - (p / rho) * gradW[d, 0]) / rho      # d(p/rho)/dx_d
        energy = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * dT
        F.append(np.stack([np.zeros_like(rho), tau[0], tau[1], tau[2], energy]))
    return np.stack(F)


class NSOracle(Oracle):
    def __init__(self, mesh, flux="lf", gamma=1.4, mu=1.0 / 1600.0, Pr=0.72):
        super().__init__(mesh, flux=flux, gamma=gamma)
        self.mu = mu
        self.Pr = Pr

    # ------------------------------------------------------------ lifting
    def face_wstar(self, Q, f):
        """(w S)_p W*_p at the owner's points of face f: [5, n^2]."""
        m = self.mesh
        e0, _, e1, _ = m.faces[f]
        phi0, phi1, wS, _ = self.face_data(f)
        WL = primitive(m.block(Q, e0) @ phi0.T, self.gamma)
        WR = primitive(m.block(Q, e1) @ phi1.T, self.gamma)
        return wS * 0.5 * (WL + WR)

    def lifting(self, Q, e, wstar):
        """Modal lifted gradient G_e [3(d), 5, nM]."""
        m = self.mesh
        op = self.ops[m.etype[e]]
        W = primitive(m.block(Q, e) @ op.V.T, self.gamma)         # [5, nQ]
        gx = np.einsum("kd,kqi->dqi", m.dxi_dx[e], op.G)           # d phi_i / d x_d at q
        vol = m.J[e] * np.einsum("dqi,vq->dvi", gx, op.w * W)
        surf = np.zeros_like(vol)
        for f, side in m.elem_faces[e]:
            phi0, phi1, _, nrm = self.face_data(f)
            phi, sgn = (phi0, 1.0) if side == 0 else (phi1, -1.0)
            Ws = wstar[f] @ phi                                   # [5, nM]
            for d in range(3):
                surf[d] = surf[d] + sgn * nrm[d] * Ws
        return np.stack([self.apply_minv(e, surf[d] - vol[d]) for d in range(3)])

    # ------------------------------------------------------------ residual
    def ns_face_flux(self, Q, f, G):
        m = self.mesh
        e0, _, e1, _ = m.faces[f]
        phi0, phi1, wS, nrm = self.face_data(f)
        UL = m.block(Q, e0) @ phi0.T
        UR = m.block(Q, e1) @ phi1.T
        gL = G[e0] @ phi0.T                                        # [3, 5, n^2]
        gR = G[e1] @ phi1.T
        Fv = 0.5 * (viscous_flux(UL, gL, self.gamma, self.mu, self.Pr)
                    + viscous_flux(UR, gR, self.gamma, self.mu, self.Pr))
        Fvn = np.einsum("d,dvp->vp", nrm, Fv)
        return wS * (riemann(self.flux, UL, UR, nrm, self.gamma) - Fvn)

    def ns_volume_term(self, Q, e, G):
        m = self.mesh
        op = self.ops[m.etype[e]]
        U = m.block(Q, e) @ op.V.T
        gradW = G[e] @ op.V.T                                      # [3, 5, nQ]
        F = physical_flux(U, self.gamma) - viscous_flux(U, gradW, self.gamma, self.mu, self.Pr)
        Fc = np.einsum("kd,dvq->kvq", m.dxi_dx[e], F)
        return m.J[e] * np.einsum("kqi,kvq->vi", op.G, op.w * Fc)

    def rhs(self, Q, elems=None):
        """R in caller layout; with elems, only those elements' blocks are filled."""
        m = self.mesh
        Q = np.asarray(Q)
        R = np.zeros_like(Q)
        elems = list(range(m.n_elems)) if elems is None else list(elems)
        faces1 = sorted({f for e in elems for f, _ in m.elem_faces[e]})
        lift_elems = sorted({x for f in faces1 for x in (m.faces[f][0], m.faces[f][2])})
        faces2 = sorted({f for e in lift_elems for f, _ in m.elem_faces[e]})
        wstar = {f: self.face_wstar(Q, f) for f in faces2}
        G = {e: self.lifting(Q, e, wstar) for e in lift_elems}
        fluxes = {f: self.ns_face_flux(Q, f, G) for f in faces1}
        for e in elems:
            r = self.ns_volume_term(Q, e, G) - self.surface_term(Q, e, fluxes)
            R[m.dof_off[e]:m.dof_off[e + 1]] = self.apply_minv(e, r).ravel()
        return R

    def rhs_vjp(self, Q, Rbar):
        """Qbar = (dR/dQ)^T Rbar (caller layout), every step transposed."""
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

        # volume: total flux F_e(U) - F_v(U, grad W)
        for e in range(E):
            op = self.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T
            gW = G[e] @ op.V.T
            Fbar = m.J[e] * op.w * np.einsum("kd,kqi,vi->dvq", m.dxi_dx[e], op.G, rbar[e])
            JU = _cs(lambda X: physical_flux(X, gam), U) - _cs(vf_u(gW), U)     # [3, 5, 5, nQ]
            JG = _cs(vf_g(U), gW)                                               # [3, 5, 3, 5, nQ]
            add(e, np.einsum("dvuq,dvq->uq", JU, Fbar) @ op.V)
            Gbar[e] += -np.einsum("dvxyq,dvq->xyq", JG, Fbar) @ op.V
        # faces: Riemann flux minus the central viscous flux
        for f, (e0, _, e1, _) in enumerate(m.faces):
            phi0, phi1, wS, nrm = self.face_data(f)
            UL, UR = m.block(Q, e0) @ phi0.T, m.block(Q, e1) @ phi1.T
            gL, gR = G[e0] @ phi0.T, G[e1] @ phi1.T
            Fsbar = wS * (-(rbar[e0] @ phi0.T) + rbar[e1] @ phi1.T)
            JL = _cs(lambda X: riemann(self.flux, X, UR, nrm, gam), UL)
            JR = _cs(lambda X: riemann(self.flux, UL, X, nrm, gam), UR)
            Fvbar = -0.5 * nrm[:, None, None] * Fsbar[None]                    # [3, 5, P]
            ULbar = np.einsum("vup,vp->up", JL, Fsbar) + np.einsum("dvup,dvp->up", _cs(vf_u(gL), UL), Fvbar)
            URbar = np.einsum("vup,vp->up", JR, Fsbar) + np.einsum("dvup,dvp->up", _cs(vf_u(gR), UR), Fvbar)
            add(e0, ULbar @ phi0)
            add(e1, URbar @ phi1)
            Gbar[e0] += np.einsum("dvxyp,dvp->xyp", _cs(vf_g(UL), gL), Fvbar) @ phi0
            Gbar[e1] += np.einsum("dvxyp,dvp->xyp", _cs(vf_g(UR), gR), Fvbar) @ phi1
        # lifting: G_d = M^{-1}(surf_d - vol_d)
        for e in range(E):
            op = self.ops[m.etype[e]]
            U = m.block(Q, e) @ op.V.T
            sbar = np.stack([self.apply_minv(e, Gbar[e][d]) for d in range(3)])
            gx = np.einsum("kd,kqi->dqi", m.dxi_dx[e], op.G)
            Wbar = -m.J[e] * op.w * np.einsum("dqi,dvi->vq", gx, sbar)
            JW = _cs(lambda X: primitive(X, gam), U)                            # [5, 5, nQ]
            add(e, np.einsum("wuq,wq->uq", JW, Wbar) @ op.V)
            for f, side in m.elem_faces[e]:
                phi0, phi1, _, nrm = self.face_data(f)
                phi, sgn = (phi0, 1.0) if side == 0 else (phi1, -1.0)
                for d in range(3):
                    Wsbar[f] += sgn * nrm[d] * (sbar[d] @ phi.T)
        # face values W* = w S (W(U-) + W(U+)) / 2
        for f, (e0, _, e1, _) in enumerate(m.faces):
            phi0, phi1, wS, _ = self.face_data(f)
            UL, UR = m.block(Q, e0) @ phi0.T, m.block(Q, e1) @ phi1.T
            a = 0.5 * wS * Wsbar[f]
            add(e0, np.einsum("wup,wp->up", _cs(lambda X: primitive(X, gam), UL), a) @ phi0)
            add(e1, np.einsum("wup,wp->up", _cs(lambda X: primitive(X, gam), UR), a) @ phi1)
        return Qbar

    def lifted_gradient(self, Q, elems=None):
        """{e: G_e [3, 5, nM]} for the given elements (all by default)."""
        m = self.mesh
        elems = list(range(m.n_elems)) if elems is None else list(elems)
        faces = sorted({f for e in elems for f, _ in m.elem_faces[e]})
        wstar = {f: self.face_wstar(Q, f) for f in faces}
        return {e: self.lifting(Q, e, wstar) for e in elems}
