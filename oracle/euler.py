"""Compressible Euler fluxes and the two Riemann solvers (LF, Roe).

Conservative variables U = (rho, rho u, rho v, rho w, E), p = (gamma-1)(E -
|m|^2/(2 rho)).  The paper's weak form (Eq. 1) leaves the numerical flux
(F.n)* unnamed; the two solvers below are the readings used throughout:

  LF:  F* = (F(U-) + F(U+)).n/2 - lambda (U+ - U-)/2,
       lambda = max(|u-.n| + c-, |u+.n| + c+),  c = sqrt(gamma p / rho).
  Roe: F* = (F(U-) + F(U+)).n/2 - sum_k |lambda_k| alpha_k r_k / 2 with the
       sqrt(rho)-weighted Roe average and no entropy fix.

All functions work on real or complex arrays (leading axis = variable).  For
complex input the non-analytic pieces (|.|, max) branch on the real part, so a
complex-step perturbation yields exact directional derivatives; |x| has
derivative 0 at x = 0, and at ties of max the '-' side wins (adjoint readings).

Parity: pinned by consistency, antisymmetry and the Roe property
(tests/test_oracle_euler.py).
"""
from __future__ import annotations

import numpy as np


def rabs(x):
    """|x|; on complex input the derivative carried by the imaginary part is
    sign(Re x), with sign(0) = 0 (the adjoint's reading at the kink)."""
    re = np.real(x)
    if not np.iscomplexobj(x):
        return np.abs(x)
    return np.where(re > 0, x, np.where(re < 0, -x, re + 0j))


def rmax(x, y):
    return np.where(np.real(x) >= np.real(y), x, y)


def pressure(U, gamma):
    rho, mx, my, mz, E = U
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)


def physical_flux(U, gamma):
    """F[d] for d = x, y, z: array [3, 5, ...]."""
    rho, mx, my, mz, E = U
    p = pressure(U, gamma)
    vel = (mx / rho, my / rho, mz / rho)
    F = []
    for d in range(3):
        ud = vel[d]
        F.append(np.stack([rho * ud,
                           mx * ud + (p if d == 0 else 0.0),
                           my * ud + (p if d == 1 else 0.0),
                           mz * ud + (p if d == 2 else 0.0),
                           (E + p) * ud]))
    return np.stack(F)


def normal_flux(U, n, gamma):
    F = physical_flux(U, gamma)
    n = np.asarray(n)
    return sum(F[d] * n[d] for d in range(3))


def lax_friedrichs(UL, UR, n, gamma):
    n = np.asarray(n)
    pL, pR = pressure(UL, gamma), pressure(UR, gamma)
    unL = (UL[1] * n[0] + UL[2] * n[1] + UL[3] * n[2]) / UL[0]
    unR = (UR[1] * n[0] + UR[2] * n[1] + UR[3] * n[2]) / UR[0]
    cL = np.sqrt(gamma * pL / UL[0])
    cR = np.sqrt(gamma * pR / UR[0])
    lam = rmax(rabs(unL) + cL, rabs(unR) + cR)
    return 0.5 * (normal_flux(UL, n, gamma) + normal_flux(UR, n, gamma)) - 0.5 * lam * (UR - UL)


def roe_dissipation(UL, UR, n, gamma, absfun=rabs):
    """sum_k absfun(lambda_k) alpha_k r_k for the Roe-averaged normal Jacobian."""
    n = np.asarray(n)
    rL, rR = UL[0], UR[0]
    uL = [UL[1 + d] / rL for d in range(3)]
    uR = [UR[1 + d] / rR for d in range(3)]
    pL, pR = pressure(UL, gamma), pressure(UR, gamma)
    HL, HR = (UL[4] + pL) / rL, (UR[4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    den = sL + sR
    u = [(sL * uL[d] + sR * uR[d]) / den for d in range(3)]
    H = (sL * HL + sR * HR) / den
    rho = sL * sR
    q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    c2 = (gamma - 1.0) * (H - 0.5 * q2)
    c = np.sqrt(c2)
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    drho = rR - rL
    dp = pR - pL
    du = [uR[d] - uL[d] for d in range(3)]
    dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2]
    a1 = (dp - rho * c * dun) / (2.0 * c2)
    a5 = (dp + rho * c * dun) / (2.0 * c2)
    a2 = drho - dp / c2
    l1, l2, l5 = absfun(un - c), absfun(un), absfun(un + c)
    dut = [du[d] - dun * n[d] for d in range(3)]
    out = []
    # wave 1 (u.n - c), wave 5 (u.n + c), entropy wave and shear waves (u.n)
    out.append(l1 * a1 + l5 * a5 + l2 * a2)
    for d in range(3):
        out.append(l1 * a1 * (u[d] - c * n[d]) + l5 * a5 * (u[d] + c * n[d])
                   + l2 * (a2 * u[d] + rho * dut[d]))
    ut_dut = u[0] * dut[0] + u[1] * dut[1] + u[2] * dut[2]
    out.append(l1 * a1 * (H - c * un) + l5 * a5 * (H + c * un)
               + l2 * (a2 * 0.5 * q2 + rho * ut_dut))
    return np.stack(out)


def roe(UL, UR, n, gamma):
    return 0.5 * (normal_flux(UL, n, gamma) + normal_flux(UR, n, gamma)) - 0.5 * roe_dissipation(UL, UR, n, gamma)


def riemann(kind, UL, UR, n, gamma):
    if kind == "lf":
        return lax_friedrichs(UL, UR, n, gamma)
    if kind == "roe":
        return roe(UL, UR, n, gamma)
    raise ValueError(kind)
