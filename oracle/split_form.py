"""Entropy-stable split form of the volume integral on hexahedra.

Sec. 2 of the paper stabilises the DGSEM by an entropy-stable formulation
built on a summation-by-parts property and the two-point flux of
Chandrashekar (2013); the construction on collapsed elements is deferred to
references that are not available here.  Readings taken (they are listed in
the design notes and shared with the library):

  * s1  Hexahedra only.  A hexahedron's n^3 Gauss-Legendre nodes (n = N+1,
        the volume rule of the weak form) carry the split form; prisms,
        pyramids and tetrahedra keep the weak form of Eq. 1 unchanged.
  * s2  Two-point flux: Chandrashekar's entropy-conservative and
        kinetic-energy-preserving flux for the entropy U = -rho s/(gamma-1),
        s = ln(p rho^-gamma), with the logarithmic mean
        ln-mean(a, b) = (a - b)/(ln a - ln b).
  * s3  Gauss nodes contain no face points, so the one-dimensional operator
        along each coordinate line is the hybridised SBP operator of the
        Gauss collocation method (Chan, Del Rey Fernandez and Carpenter,
        2019): with the 1D weights W, derivative D, Q = W D and the
        extrapolations E_-, E_+ to the line's two ends (signs s_-=-1,
        s_+=+1; Q + Q^T = sum_f s_f E_f^T E_f),
          r_i = - sum_j (Q - Q^T)_ij F#(u_i, u_j)
                - sum_f s_f E_f,i F#(u_i, u~_f)
                + sum_f s_f E_f,i sum_j E_f,j F#(u~_f, u_j),
        with F# contracted with the line direction's contravariant metric
        J dxi_l/dx (constant on an affine element) and each line's r scaled
        by the product of the two other directions' weights.  For the central
        flux F#(a, b) = (F(a) + F(b))/2 this equals the weak form's volume
        term Q^T F exactly (a pin below).
  * s4  Face states of a split-form hexahedron are entropy-projected: the
        entropy variables at the nodes, extended by their interpolating
        polynomial to the face point, mapped back to conservative variables,
        u~ = u(sum_q l_q(x) v(u_q)).  The numerical surface flux (LF, Roe,
        or the entropy-conservative F#.n with no dissipation, 'ec') is taken
        on these states.  With 'ec' the semi-discrete entropy rate
        sum_e sum_q w_q J v(u_q) . R_q vanishes on a periodic all-hex mesh;
        with LF it is not positive.
  * s5  Affine hexahedra only (constant metric).

Parity: pinned by tests/test_oracle_split_form.py -- the log mean against
50-digit values, consistency, symmetry and Tadmor's condition of the flux,
the entropy variables against the gradient of U, the reduction to the weak
form for the central flux, entropy conservation ('ec') and dissipation (LF)
on periodic hexahedral meshes, free stream and conservation on mixed meshes.
Test infrastructure only, like the rest of the oracle.
"""
from __future__ import annotations

import numpy as np

from .dg import Oracle
from .elements import HEX
from .euler import physical_flux, riemann
from .quadrature import gauss_legendre


def log_mean(a, b):
    """(a - b)/(ln a - ln b) for positive a, b (a where a == b).  With
    f = (a - b)/(a + b) and the identity ln(a/b) = 2 artanh(f): for |f| <= 1/2
    it is evaluated as ((a + b)/2) f/artanh(f) (no cancellation as b -> a),
    otherwise as (a - b)/ln(a/b) (artanh is ill-conditioned near |f| = 1)."""
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    f = (a - b) / (a + b)
    near = np.abs(f) <= 0.5
    safe = np.where(near & (f != 0.0), f, 0.5)
    ratio = np.where(f == 0.0, 1.0, safe / np.arctanh(safe))
    far = np.where(near, 1.0, (a - b) / np.log(np.where(near, 2.0, a / b)))
    return np.where(near, 0.5 * (a + b) * ratio, far)


def primitives(U, gamma):
    rho = U[0]
    vel = U[1:4] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * np.sum(vel * vel, axis=0))
    return rho, vel, p


def entropy(U, gamma):
    """Mathematical entropy U = -rho s/(gamma - 1), s = ln p - gamma ln rho."""
    rho, _, p = primitives(U, gamma)
    return -rho * (np.log(p) - gamma * np.log(rho)) / (gamma - 1.0)


def entropy_variables(U, gamma):
    """v = dU/du = ((gamma - s)/(gamma - 1) - rho |u|^2/(2p), rho u/p, -rho/p)."""
    rho, vel, p = primitives(U, gamma)
    s = np.log(p) - gamma * np.log(rho)
    v0 = (gamma - s) / (gamma - 1.0) - 0.5 * rho * np.sum(vel * vel, axis=0) / p
    return np.concatenate([v0[None], rho * vel / p, (-rho / p)[None]], axis=0)


def conservative_from_entropy(V, gamma):
    """The inverse map u(v): p/rho = -1/v4, u = -v_{1..3}/v4,
    s = gamma - (gamma - 1)(v0 + rho|u|^2/(2p)), rho = (-v4 e^s)^(-1/(gamma-1))."""
    v4 = V[4]
    vel = -V[1:4] / v4
    q = np.sum(V[1:4] * V[1:4], axis=0)
    s = gamma - (gamma - 1.0) * (V[0] - 0.5 * q / v4)
    rho = np.exp(-(s + np.log(-v4)) / (gamma - 1.0))
    p = -rho / v4
    E = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=0)
    return np.concatenate([rho[None], rho * vel, E[None]], axis=0)


def chandrashekar(UL, UR, m, gamma):
    """Chandrashekar's two-point flux F#(UL, UR) contracted with the vector m:
      F_rho = rho_ln (u_bar . m),  F_mom = p_hat m + u_bar F_rho,
      F_E = (1/(2 (gamma - 1) beta_ln) - |u|^2_bar / 2) F_rho + u_bar . F_mom,
    beta = rho/(2p), bars arithmetic means, _ln logarithmic means,
    p_hat = rho_bar/(2 beta_bar)."""
    m = np.asarray(m, dtype=float).reshape((3,) + (1,) * (np.ndim(UL) - 1))
    rL, uL, pL = primitives(UL, gamma)
    rR, uR, pR = primitives(UR, gamma)
    bL, bR = 0.5 * rL / pL, 0.5 * rR / pR
    rho_ln, beta_ln = log_mean(rL, rR), log_mean(bL, bR)
    ubar = 0.5 * (uL + uR)
    q2bar = 0.5 * (np.sum(uL * uL, axis=0) + np.sum(uR * uR, axis=0))
    p_hat = 0.5 * (rL + rR) / (bL + bR)
    Frho = rho_ln * np.sum(ubar * m, axis=0)
    Fmom = p_hat * m + ubar * Frho
    FE = (1.0 / (2.0 * (gamma - 1.0) * beta_ln) - 0.5 * q2bar) * Frho + np.sum(ubar * Fmom, axis=0)
    return np.concatenate([Frho[None], Fmom, FE[None]], axis=0)


def central(UL, UR, m, gamma):
    """(F(UL) + F(UR))/2 contracted with m (the two-point flux whose split form
    is the weak form)."""
    m = np.asarray(m, dtype=float)
    FL, FR = physical_flux(UL, gamma), physical_flux(UR, gamma)
    return 0.5 * sum((FL[d] + FR[d]) * m[d] for d in range(3))


def lagrange_values(x, pts):
    """l_j(pts) for the Lagrange basis on the nodes x, from the product form:
    [len(pts), n]."""
    pts = np.asarray(pts, dtype=float)
    n = len(x)
    L = np.ones((pts.size, n))
    for j in range(n):
        for k in range(n):
            if k != j:
                L[:, j] *= (pts - x[k]) / (x[j] - x[k])
    return L


def lagrange_1d(x):
    """Derivative matrix D_ij = l_j'(x_i) and end values E[-], E[+] (rows
    l_j(-1), l_j(+1)) of the Lagrange basis on the nodes x, from the product
    form of l_j."""
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                D[i, j] = sum(1.0 / (x[j] - x[k]) for k in range(n) if k != j)
            else:
                num = np.prod([x[i] - x[k] for k in range(n) if k not in (i, j)])
                den = np.prod([x[j] - x[k] for k in range(n) if k != j])
                D[i, j] = num / den
    E = np.zeros((2, n))
    for f, end in enumerate((-1.0, 1.0)):
        for j in range(n):
            E[f, j] = np.prod([(end - x[k]) / (x[j] - x[k]) for k in range(n) if k != j])
    return D, E


class SplitFormOracle(Oracle):
    """Oracle with the split-form volume term and entropy-projected traces on
    hexahedra (readings s1-s5); every other element as in Oracle.

    two_point: 'chandrashekar' (the method) or 'central' (whose split form is
    the weak form: a pin).  project: entropy-projected hexahedral traces (the
    method) or plain traces (with 'central' the weak form again).
    flux: 'lf', 'roe' or 'ec' (Chandrashekar F#.n, no dissipation)."""

    def __init__(self, mesh, flux="lf", gamma=1.4, two_point="chandrashekar", project=True):
        super().__init__(mesh, flux="lf" if flux == "ec" else flux, gamma=gamma)
        self.iflux = flux
        self.two_point = chandrashekar if two_point == "chandrashekar" else central
        self.project_traces = project
        n = mesh.N + 1
        x, w = gauss_legendre(n)
        self.x1, self.w1 = x, w
        self.D1, self.E1 = lagrange_1d(x)
        self.Q1 = w[:, None] * self.D1
        self._ref_cache = {}
        if HEX in self.ops:
            op = self.ops[HEX]
            # the oracle's hexahedral volume points are (xi_i, eta_j, zeta_k),
            # k fastest: check, so the tensor lines below are the right ones
            grid = np.stack(np.meshgrid(x, x, x, indexing="ij"), axis=-1).reshape(-1, 3)
            assert np.abs(op.pts - grid).max() < 1e-14

    # ------------------------------------------------------------ hexahedra
    def nodal_state(self, Q, e):
        return self.mesh.block(Q, e) @ self.ops[self.mesh.etype[e]].V.T      # [5, n^3]

    def split_volume_nodal(self, Q, e):
        """Nodal split-form volume term H [5, n^3] of hexahedron e (s3)."""
        m = self.mesh
        n = m.N + 1
        U = self.nodal_state(Q, e).reshape(5, n, n, n)
        metric = m.J[e] * m.dxi_dx[e]                                          # rows: J dxi_l/dx
        E, S = self.E1, self.Q1 - self.Q1.T
        sgn = (-1.0, 1.0)
        H = np.zeros((5, n, n, n))
        for l in range(3):
            Ul = np.moveaxis(U, 1 + l, 1)                                       # line index second
            Hl = np.zeros_like(Ul)
            for a in range(n):
                for b in range(n):
                    u = Ul[:, :, a, b]                                          # [5, n] along the line
                    if self.project_traces:
                        vt = entropy_variables(u, self.gamma) @ E.T            # [5, 2]
                        ut = conservative_from_entropy(vt, self.gamma)
                    else:
                        ut = u @ E.T
                    r = np.zeros((5, n))
                    for i in range(n):
                        for j in range(n):
                            if i != j:
                                r[:, i] -= S[i, j] * self.two_point(u[:, i], u[:, j], metric[l], self.gamma)
                        for f in range(2):
                            r[:, i] -= sgn[f] * E[f, i] * self.two_point(u[:, i], ut[:, f], metric[l], self.gamma)
                            acc = sum(E[f, j] * self.two_point(ut[:, f], u[:, j], metric[l], self.gamma)
                                      for j in range(n))
                            r[:, i] += sgn[f] * E[f, i] * acc
                    Hl[:, :, a, b] = self.w1[a] * self.w1[b] * r
            H += np.moveaxis(Hl, 1, 1 + l)
        return H.reshape(5, n ** 3)

    def volume_term(self, Q, e):
        if self.mesh.etype[e] != HEX:
            return super().volume_term(Q, e)
        # modal test functions: phi_i = sum_q phi_i(x_q) l_q, so vol = V^T H
        return self.split_volume_nodal(Q, e) @ self.ops[HEX].V

    def trace(self, Q, e, phi, ref):
        """The element's state at face points with reference coordinates ref
        [P, 3] and basis values phi [P, nM].  A split-form hexahedron gives
        u(v~), v~ the interpolant of the nodal entropy variables at the
        points, evaluated in its Lagrange form sum_q l_q(x) v_q (tensor
        products of 1D Lagrange polynomials on the Gauss nodes)."""
        if self.mesh.etype[e] != HEX or not self.project_traces:
            return self.mesh.block(Q, e) @ phi.T
        v = entropy_variables(self.nodal_state(Q, e), self.gamma)           # [5, n^3]
        n = self.mesh.N + 1
        La, Lb, Lc = (lagrange_values(self.x1, ref[:, d]) for d in range(3))
        ell = np.einsum("pi,pj,pk->pijk", La, Lb, Lc).reshape(len(ref), n ** 3)
        return conservative_from_entropy(v @ ell.T, self.gamma)

    def face_flux(self, Q, f):
        m = self.mesh
        e0, _, e1, _ = m.faces[f]
        phi0, phi1, wS, nrm = self.face_data(f)
        if f not in self._ref_cache:
            ref0, ref1, _, _ = m.face_geometry(f)
            self._ref_cache[f] = (ref0, ref1)
        ref0, ref1 = self._ref_cache[f]
        UL, UR = self.trace(Q, e0, phi0, ref0), self.trace(Q, e1, phi1, ref1)
        if self.iflux == "ec":
            return wS * chandrashekar(UL, UR, nrm, self.gamma)
        return wS * riemann(self.flux, UL, UR, nrm, self.gamma)

    # ------------------------------------------------------------ diagnostics
    def nodal_residual(self, R, e):
        """The residual of element e at its volume points, V R_e [5, n^3]."""
        return self.mesh.block(R, e) @ self.ops[self.mesh.etype[e]].V.T

    def entropy_rate(self, Q, R):
        """sum_e sum_q w_q J_e v(U_q) . R(x_q), the semi-discrete entropy
        production (exact for the hexahedra, whose rule integrates the
        product of two degree-N polynomials exactly), and the sum of the
        absolute values of its terms (its scale)."""
        total, scale = 0.0, 0.0
        for e in range(self.mesh.n_elems):
            op = self.ops[self.mesh.etype[e]]
            v = entropy_variables(self.nodal_state(Q, e), self.gamma)
            t = self.mesh.J[e] * op.w * np.sum(v * self.nodal_residual(R, e), axis=0)
            total += t.sum()
            scale += np.abs(t).sum()
        return total, scale
