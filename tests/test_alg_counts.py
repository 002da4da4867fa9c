"""The per-point flop counts of alg_counts.json, derived by counting.

bench.py's roofline divides algorithmic flops by kernel time.  Its per-point
constants are frozen in alg_counts.json and derived here by running the
formulas on a value type that counts operations (+, -, *, / and sqrt one flop
each; abs, max, negation and comparisons none; an FMA two):
  * the oracle's own Euler flux and Riemann solvers (oracle/euler.py), the
    literal count of the plain CPU definitions (every directional flux formed,
    then dotted with the normal);
  * the arrangement the face kernel evaluates, transcribed below: the
    Lax-Friedrichs flux with the normal scaled by w S / 2 (one reciprocal and
    one square root per side, F_rho = m.n) and the Roe flux from the Euler
    normal fluxes of both sides, each times the face weight w S.
The test fails if the file and the counts disagree."""
import json
import math
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Op:
    """A value that counts the arithmetic done with it."""
    count = 0

    def _op(self, other=None):
        Op.count += 1
        return Op()

    __add__ = __radd__ = __sub__ = __rsub__ = __mul__ = __rmul__ = __truediv__ = __rtruediv__ = _op

    def __neg__(self):
        return Op()

    def __abs__(self):
        return Op()

    def sqrt(self):
        Op.count += 1
        return Op()

    @property
    def real(self):
        return 0.0

    def __ge__(self, other):
        return True


def ops(k):
    return np.array([Op() for _ in range(k)], dtype=object)


def counted(fn, *args):
    Op.count = 0
    fn(*args)
    return Op.count


def fma(a, b, c):
    return a * b + c


def fmax(a, b):
    return a


def sqrt(a):
    return a.sqrt()


def kernel_lf(UL, UR, n, wS, gamma):
    """The face kernel's Lax-Friedrichs arrangement (returns w S F*)."""
    h = 0.5 * wS
    s = [h * n[0], h * n[1], h * n[2]]
    gm1 = gamma - 1.0

    def side(U):
        r = 1.0 / U[0]
        ms = fma(U[1], s[0], fma(U[2], s[1], U[3] * s[2]))
        us = ms * r
        m2 = fma(U[1], U[1], fma(U[2], U[2], U[3] * U[3]))
        p = gm1 * fma(-0.5 * r, m2, U[4])
        F = [ms, fma(U[1], us, p * s[0]), fma(U[2], us, p * s[1]), fma(U[3], us, p * s[2]), (U[4] + p) * us]
        return F, fma(h, sqrt(gamma * p * r), abs(us))
    FL, lL = side(UL)
    FR, lR = side(UR)
    lam = fmax(lL, lR)
    return [fma(lam, UL[v] - UR[v], FL[v] + FR[v]) for v in range(5)]


def kernel_roe(UL, UR, n, wS, gamma):
    """The face kernel's Roe arrangement (returns w S F*)."""
    def normal_state(U):
        rinv = 1.0 / U[0]
        u, v, w = U[1] * rinv, U[2] * rinv, U[3] * rinv
        p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] * u + U[2] * v + U[3] * w))
        un = u * n[0] + v * n[1] + w * n[2]
        F = [U[0] * un, U[1] * un + p * n[0], U[2] * un + p * n[1], U[3] * un + p * n[2], (U[4] + p) * un]
        return F, p, rinv, (U[4] + p) * rinv
    FL, pL, rL, HL = normal_state(UL)
    FR, pR, rR, HR = normal_state(UR)
    sL, sR = sqrt(UL[0]), sqrt(UR[0])
    den = 1.0 / (sL + sR)
    uL = [UL[1] * rL, UL[2] * rL, UL[3] * rL]
    uR = [UR[1] * rR, UR[2] * rR, UR[3] * rR]
    u = [(sL * uL[d] + sR * uR[d]) * den for d in range(3)]
    H = (sL * HL + sR * HR) * den
    rho = sL * sR
    q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    c2 = (gamma - 1.0) * (H - 0.5 * q2)
    c = sqrt(c2)
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2]
    drho, dp = UR[0] - UL[0], pR - pL
    du = [uR[d] - uL[d] for d in range(3)]
    dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2]
    ic2 = 1.0 / c2
    a1 = 0.5 * (dp - rho * c * dun) * ic2
    a5 = 0.5 * (dp + rho * c * dun) * ic2
    a2 = drho - dp * ic2
    l1, l5, l2 = abs(un - c) * a1, abs(un + c) * a5, abs(un)
    dut = [du[d] - dun * n[d] for d in range(3)]
    D = [l1 + l5 + l2 * a2]
    for d in range(3):
        D.append(l1 * (u[d] - c * n[d]) + l5 * (u[d] + c * n[d]) + l2 * (a2 * u[d] + rho * dut[d]))
    udut = u[0] * dut[0] + u[1] * dut[1] + u[2] * dut[2]
    D.append(l1 * (H - c * un) + l5 * (H + c * un) + l2 * (a2 * 0.5 * q2 + rho * udut))
    return [wS * (0.5 * (FL[v] + FR[v]) - 0.5 * D[v]) for v in range(5)]


def log(a):
    return a.sqrt()          # one flop, like a square root


exp = log


def kernel_two_point_state(U, gm1):
    """The element kernel's two-point quantities of a state (split form)."""
    r = U[0]
    ri = 1.0 / r
    u, v, w = U[1] * ri, U[2] * ri, U[3] * ri
    q2 = fma(u, u, fma(v, v, w * w))
    p = gm1 * fma(-0.5 * r, q2, U[4])
    b = 0.5 * r / p
    return [r, u, v, w, b, log(r), log(b), q2]


def kernel_ln_mean_series(a, b):
    """The series branch of the logarithmic mean: the branch test,
    f = d/(a + b), u = f^2 and the degree-8 polynomial."""
    d, sm = a - b, a + b
    (d * d, 1e-2 * sm * sm)         # the branch test (a comparison)
    f = d / sm
    u = f * f
    g = Op()
    for _ in range(8):
        g = fma(g, u, Op())
    return 0.5 * sm * g


def kernel_two_point_flux(L, R, m, igm1):
    """The kernels' Chandrashekar flux F#(L, R).m from two-point quantities
    (series branch of both logarithmic means; one reciprocal of
    beta_L + beta_R serves 1/beta_ln and p_hat)."""
    rho_ln = kernel_ln_mean_series(L[0], R[0])
    db, sb = L[4] - R[4], L[4] + R[4]
    isb = 1.0 / sb
    (db * db, 1e-2 * sb * sb)         # the branch test (a comparison)
    u2 = (db * isb) * (db * isb)
    h = Op()
    for _ in range(7):
        h = fma(h, u2, Op())
    ib_ln = 2.0 * isb * h
    u, v, w = 0.5 * (L[1] + R[1]), 0.5 * (L[2] + R[2]), 0.5 * (L[3] + R[3])
    p_hat = 0.5 * (L[0] + R[0]) * isb
    q2 = 0.5 * (L[7] + R[7])
    F0 = rho_ln * fma(u, m[0], fma(v, m[1], w * m[2]))
    F = [F0, fma(p_hat, m[0], u * F0), fma(p_hat, m[1], v * F0), fma(p_hat, m[2], w * F0)]
    F.append(fma(fma(0.5 * igm1, ib_ln, -0.5 * q2), F0, fma(u, F[1], fma(v, F[2], w * F[3]))))
    return F


def kernel_entropy_variables(P, gamma, igm1):
    lnp = P[5] - 0.6931471805599453 - P[6]
    s = lnp - gamma * P[5]
    b2 = 2.0 * P[4]
    return [fma(gamma - s, igm1, -P[4] * P[7]), b2 * P[1], b2 * P[2], b2 * P[3], -b2]


def kernel_from_entropy_variables(v, gamma, igm1):
    b = -0.5 * v[4]
    iv4 = 1.0 / v[4]
    u, vv, w = -v[1] * iv4, -v[2] * iv4, -v[3] * iv4
    q2 = fma(u, u, fma(vv, vv, w * w))
    s = gamma - (gamma - 1.0) * fma(b, q2, v[0])
    lb = log(b)
    lr = -(s + 0.6931471805599453 + lb) * igm1
    r = exp(lr)
    p = 0.5 * r / b
    return [r, r * u, r * vv, r * w, fma(p, igm1, 0.5 * r * q2)], [r, u, vv, w, b, lr, lb, q2]


def derived_counts():
    from oracle import euler
    out = {
        "oracle_euler_flux_per_point": counted(euler.physical_flux, ops(5), 1.4),
        "oracle_lf_per_face_point": counted(euler.lax_friedrichs, ops(5), ops(5), ops(3), 1.4),
        "oracle_roe_per_face_point": counted(euler.roe, ops(5), ops(5), ops(3), 1.4),
        "kernel_lf_per_face_point": counted(kernel_lf, ops(5), ops(5), ops(3), Op(), 1.4),
        "kernel_roe_per_face_point": counted(kernel_roe, ops(5), ops(5), ops(3), Op(), 1.4),
    }
    # contravariant transform of the three directional fluxes with the 3x3
    # metric, per point: 3 x 5 outputs, each 3 products and 2 sums
    out["contravariant_transform_per_point"] = 3 * 5 * (3 + 2)
    out["f_F_per_point"] = out["oracle_euler_flux_per_point"] + out["contravariant_transform_per_point"]
    # split form (hexahedra), the kernels' arrangement; ln and exp count one flop
    out["split_two_point_state"] = counted(kernel_two_point_state, list(ops(5)), Op())
    out["split_two_point_flux"] = counted(kernel_two_point_flux, list(ops(8)), list(ops(8)), list(ops(3)), Op())
    out["split_entropy_variables"] = counted(kernel_entropy_variables, list(ops(8)), Op(), Op())
    out["split_from_entropy_variables"] = counted(kernel_from_entropy_variables, list(ops(5)), Op(), Op())
    return out


def test_counts_file_matches_the_formulas():
    with open(os.path.join(ROOT, "alg_counts.json")) as f:
        frozen = json.load(f)["per_point_flops"]
    assert frozen == derived_counts()


def test_counter_counts_a_known_formula():
    # (a + b) * c / d - sqrt(e): 4 binary operations and one square root
    a, b, c, d, e = ops(5)
    assert counted(lambda: (a + b) * c / d - sqrt(e)) == 5
    assert math.isclose(counted(fma, Op(), Op(), Op()), 2)


if __name__ == "__main__":
    import sys
    sys.path.insert(0, ROOT)
    print(json.dumps(derived_counts(), indent=1))
