"""Adjoint of the modal DG right-hand side and of K LSERK steps.

The paper differentiates nothing; these are the vector-Jacobian products the
library exports, written as the plain transpose of each step of oracle.dg:

  rbar_e      = M_e^{-1} Rbar_e                         (M_e symmetric)
  volume      Fbar_d[v, q] = J_e w_q sum_k (dxi_k/dx_d) sum_i (dphi_i/dxi_k)(q) rbar[v, i]
              Ubar[:, q]   = sum_d (dF_d/dU)(U_q)^T Fbar_d[:, q];  Qbar_e += Ubar V
  faces       Fbar*_p = (w S)_p (-rbar_own Phi_own[p]^T + rbar_nb Phi_nb[p]^T)
              Ubar-_p = (dF*/dU-)^T Fbar*_p,  Ubar+_p = (dF*/dU+)^T Fbar*_p
              Qbar_own += Ubar- Phi_own,  Qbar_nb += Ubar+ Phi_nb
The 5x5 pointwise Jacobians are formed by complex-step differentiation of the
oracle's own flux functions (exact to rounding; |x| has derivative 0 at x = 0
and max takes the '-' side at ties).

Reverse LSERK (2N storage, K = 0 at every step start), per stage s = 5..1:
  Kbar += B_s Qbar;  Qbar += dt J(Q_{s-1})^T Kbar;  Kbar <- A_s Kbar.
All forward stage states are stored (no checkpointing: this is the plain
definition; the library's checkpointed recomputation must reproduce it).

Parity: pinned by the dense Jacobian assembled column by column with complex
steps through oracle.dg (brute force), the dot-product test, and central finite
differences (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

from .dg import LSERK_A, LSERK_B
from .euler import physical_flux, riemann

H_CS = 1e-30


def cs_jacobian(fun, U):
    """d fun / d U by complex steps: fun maps [5, P] -> [k, ..., P]; returns [k.., 5, P]."""
    cols = []
    for u in range(5):
        dU = np.zeros((5,) + U.shape[1:], dtype=complex)
        dU[u] = 1.0
        cols.append(fun(U + 1j * H_CS * dU).imag / H_CS)
    return np.stack(cols, axis=-2)


def rhs_vjp(o, Q, Rbar):
    m = o.mesh
    Q = np.asarray(Q, dtype=float)
    Qbar = np.zeros_like(Q)
    rbar = {}
    for e in range(m.n_elems):
        rbar[e] = o.apply_minv(e, m.block(Rbar, e))
    # volume
    for e in range(m.n_elems):
        op = o.ops[m.etype[e]]
        U = m.block(Q, e) @ op.V.T                                   # [5, nQ]
        g = m.dxi_dx[e]
        Fbar = m.J[e] * op.w * np.einsum("kd,kqi,vi->dvq", g, op.G, rbar[e])
        JF = cs_jacobian(lambda X: physical_flux(X, o.gamma), U)     # [3, 5(v), 5(u), nQ]
        Ubar = np.einsum("dvuq,dvq->uq", JF, Fbar)
        Qbar[m.dof_off[e]:m.dof_off[e + 1]] += (Ubar @ op.V).ravel()
    face_vjp(o, Q, rbar, Qbar)
    return Qbar


def face_vjp(o, Q, rbar, Qbar):
    """Face part of the transpose: adds to Qbar the cotangents of both
    traces of every face, given rbar_e = M_e^{-1} Rbar_e per element.  The
    face weights w S and the normals may be per point (curved owners)."""
    m = o.mesh
    for f, (e0, _, e1, _) in enumerate(m.faces):
        phi0, phi1, wS, nrm = o.face_data(f)
        UL = m.block(Q, e0) @ phi0.T
        UR = m.block(Q, e1) @ phi1.T
        Fs_bar = wS * (-(rbar[e0] @ phi0.T) + rbar[e1] @ phi1.T)     # [5, P]
        JL = cs_jacobian(lambda X: riemann(o.flux, X, UR, nrm, o.gamma), UL)
        JR = cs_jacobian(lambda X: riemann(o.flux, UL, X, nrm, o.gamma), UR)
        ULbar = np.einsum("vup,vp->up", JL, Fs_bar)
        URbar = np.einsum("vup,vp->up", JR, Fs_bar)
        Qbar[m.dof_off[e0]:m.dof_off[e0 + 1]] += (ULbar @ phi0).ravel()
        Qbar[m.dof_off[e1]:m.dof_off[e1 + 1]] += (URbar @ phi1).ravel()


def rhs_jvp(o, Q, V):
    """J(Q) V by one complex step through the oracle's own residual."""
    return o.rhs(np.asarray(Q, dtype=float) + 1j * H_CS * np.asarray(V)).imag / H_CS


def rk_forward(o, Q0, dt, nsteps):
    """Final state and the stage states Q_{s-1} of every stage, in order."""
    stages = []
    Q = np.asarray(Q0, dtype=float).copy()
    for _ in range(nsteps):
        Q = o.lserk_step(Q, dt, stages_out=stages)
    return Q, stages


def rk_vjp(o, Q0, dt, nsteps, QKbar):
    _, stages = rk_forward(o, Q0, dt, nsteps)
    Qbar = np.asarray(QKbar, dtype=float).copy()
    for step in reversed(range(nsteps)):
        Kbar = np.zeros_like(Qbar)
        for s in reversed(range(5)):
            Kbar = Kbar + LSERK_B[s] * Qbar
            Qs = stages[5 * step + s]
            Qbar = Qbar + dt * (o.rhs_vjp(Qs, Kbar) if hasattr(o, "rhs_vjp") else rhs_vjp(o, Qs, Kbar))
            Kbar = LSERK_A[s] * Kbar
    return Qbar


def rk_jvp(o, Q0, dt, nsteps, V):
    Q = np.asarray(Q0, dtype=float) + 1j * H_CS * np.asarray(V)
    for _ in range(nsteps):
        Q = o.lserk_step(Q, dt)
    return Q.imag / H_CS
