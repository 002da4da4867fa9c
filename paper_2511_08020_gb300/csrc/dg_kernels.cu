// Kernels of the modal DG hot path; see dg_kernels.cuh for the phase layout.
#include <algorithm>
#include <cstdio>

#include "dg_kernels.cuh"

namespace dgk {

namespace {

__device__ __forceinline__ int sel3(int i, int j, int k, int w) { return w == 0 ? i : (w == 1 ? j : k); }

__device__ __forceinline__ bool finite_bits(double x) {
  // exponent field all ones <=> inf or nan (integer test, no FP64 pipe work)
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// ------------------------------------------------------------------ physics
// Euler normal flux F(U).n with u.n, p, 1/rho and c^2 as by-products.
struct NState {
  double F[5];
  double un, p, rinv, H;
};

__device__ __forceinline__ void normal_state(const double* U, const double* n, double gamma, NState& s) {
  s.rinv = 1.0 / U[0];
  double u = U[1] * s.rinv, v = U[2] * s.rinv, w = U[3] * s.rinv;
  s.p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] * u + U[2] * v + U[3] * w));
  s.un = u * n[0] + v * n[1] + w * n[2];
  s.F[0] = U[0] * s.un;
  s.F[1] = U[1] * s.un + s.p * n[0];
  s.F[2] = U[2] * s.un + s.p * n[1];
  s.F[3] = U[3] * s.un + s.p * n[2];
  s.F[4] = (U[4] + s.p) * s.un;
  s.H = (U[4] + s.p) * s.rinv;
}

// Lax-Friedrichs: F* = (F- + F+)/2 - lambda (U+ - U-)/2,
// lambda = max(|u-.n| + c-, |u+.n| + c+).
__device__ __forceinline__ void flux_lf(const double* UL, const double* UR, const double* n, double gamma, double* Fs) {
  NState L, R;
  normal_state(UL, n, gamma, L);
  normal_state(UR, n, gamma, R);
  double cL = sqrt(gamma * L.p * L.rinv), cR = sqrt(gamma * R.p * R.rinv);
  double lam = fmax(fabs(L.un) + cL, fabs(R.un) + cR);
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (L.F[v] + R.F[v]) - 0.5 * lam * (UR[v] - UL[v]);
}

// The Lax-Friedrichs flux above, already multiplied by the face weight
// wS = w S of the point, arranged for few FP64 instructions: with the scaled
// normal s = (wS/2) n,
//   wS F* = F_s(U-) + F_s(U+) + lam_s (U- - U+),
//   F_s(U) = (m.s, m (m.s)/rho + p s, (E + p)(m.s)/rho),
//   lam_s = max(|m-.s|/rho- + (wS/2) c-, |m+.s|/rho+ + (wS/2) c+),
// so rho F_0 = m.n needs no multiply, one reciprocal and one square root per
// side serve the flux and the wave speed, and the 1/2 and wS scales fold into
// the normal.
__device__ __forceinline__ void lf_side(const double* U, const double* s, double h, double gm1, double gamma,
                                        double* F, double& lam) {
  const double r = 1.0 / U[0];
  const double ms = fma(U[1], s[0], fma(U[2], s[1], U[3] * s[2]));
  const double us = ms * r;
  const double m2 = fma(U[1], U[1], fma(U[2], U[2], U[3] * U[3]));
  const double p = gm1 * fma(-0.5 * r, m2, U[4]);
  F[0] = ms;
  F[1] = fma(U[1], us, p * s[0]);
  F[2] = fma(U[2], us, p * s[1]);
  F[3] = fma(U[3], us, p * s[2]);
  F[4] = (U[4] + p) * us;
  lam = fma(h, sqrt(gamma * p * r), fabs(us));
}

__device__ __forceinline__ void moving_lf_side(const double* U, const double* s, double h, double sig, double gm1,
                                               double gamma, double* F, double& lam) {
  const double r = 1.0 / U[0];
  const double ms = fma(U[1], s[0], fma(U[2], s[1], U[3] * s[2]));
  const double us = ms * r;
  const double m2 = fma(U[1], U[1], fma(U[2], U[2], U[3] * U[3]));
  const double p = gm1 * fma(-0.5 * r, m2, U[4]);
  const double ur = us - sig;
  F[0] = fma(-sig, U[0], ms);
  F[1] = fma(U[1], ur, p * s[0]);
  F[2] = fma(U[2], ur, p * s[1]);
  F[3] = fma(U[3], ur, p * s[2]);
  F[4] = fma(U[4], ur, p * us);
  lam = fma(h, sqrt(gamma * p * r), fabs(ur));
}

__device__ __forceinline__ void flux_lf_scaled(const double* UL, const double* UR, const double* n, double wS,
                                               double gamma, double* Fs) {
  const double h = 0.5 * wS;
  const double s[3] = {h * n[0], h * n[1], h * n[2]};
  const double gm1 = gamma - 1.0;
  double FL[5], FR[5], lamL, lamR;
  lf_side(UL, s, h, gm1, gamma, FL, lamL);
  lf_side(UR, s, h, gm1, gamma, FR, lamR);
  const double lam = fmax(lamL, lamR);
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v] = fma(lam, UL[v] - UR[v], FL[v] + FR[v]);
}

// The same flux in a frame moving with normal speed sn = xdot.n at the point
// (moving meshes): F_s(U) - sig U with sig = (wS/2) sn, and the wave speed
// from the relative normal velocity, lam_s = max(|m.s/rho - sig| + (wS/2) c).
__device__ __forceinline__ void flux_lf_moving_scaled(const double* UL, const double* UR, const double* n, double wS,
                                                      double sn, double gamma, double* Fs) {
  const double h = 0.5 * wS;
  const double s[3] = {h * n[0], h * n[1], h * n[2]};
  const double sig = h * sn;
  const double gm1 = gamma - 1.0;
  double FL[5], FR[5], lamL, lamR;
  moving_lf_side(UL, s, h, sig, gm1, gamma, FL, lamL);
  moving_lf_side(UR, s, h, sig, gm1, gamma, FR, lamR);
  const double lam = fmax(lamL, lamR);
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v] = fma(lam, UL[v] - UR[v], FL[v] + FR[v]);
}

// Roe: F* = (F- + F+)/2 - sum_k |lambda_k| alpha_k r_k / 2 with
// sqrt(rho)-weighted averages of u and H, no entropy fix.
__device__ __forceinline__ void flux_roe(const double* UL, const double* UR, const double* n, double gamma, double* Fs) {
  NState L, R;
  normal_state(UL, n, gamma, L);
  normal_state(UR, n, gamma, R);
  double sL = sqrt(UL[0]), sR = sqrt(UR[0]);
  double den = 1.0 / (sL + sR);
  double uL[3] = {UL[1] * L.rinv, UL[2] * L.rinv, UL[3] * L.rinv};
  double uR[3] = {UR[1] * R.rinv, UR[2] * R.rinv, UR[3] * R.rinv};
  double u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = (sL * uL[d] + sR * uR[d]) * den;
  double H = (sL * L.H + sR * R.H) * den;
  double rho = sL * sR;
  double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  double c = sqrt(c2);
  double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  double drho = UR[0] - UL[0], dp = R.p - L.p;
  double du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  double dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  double ic2 = 1.0 / c2;
  double a1 = 0.5 * (dp - rho * c * dun) * ic2;
  double a5 = 0.5 * (dp + rho * c * dun) * ic2;
  double a2 = drho - dp * ic2;
  double l1 = fabs(un - c) * a1, l5 = fabs(un + c) * a5, l2 = fabs(un);
  double dut[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dut[d] = du[d] - dun * n[d];
  double D[5];
  D[0] = l1 + l5 + l2 * a2;
#pragma unroll
  for (int d = 0; d < 3; ++d) D[1 + d] = l1 * (u[d] - c * n[d]) + l5 * (u[d] + c * n[d]) + l2 * (a2 * u[d] + rho * dut[d]);
  double udut = u[0] * dut[0] + u[1] * dut[1] + u[2] * dut[2];
  D[4] = l1 * (H - c * un) + l5 * (H + c * un) + l2 * (a2 * 0.5 * q2 + rho * udut);
#pragma unroll
  for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (L.F[v] + R.F[v]) - 0.5 * D[v];
}

// ------------------------------------------------------------------ two-point flux (split form)
//
// Entropy-stable split form (Sec. 2: entropy-stable DGSEM with a
// summation-by-parts property and Chandrashekar's two-point flux) for the
// entropy U = -rho s/(gamma-1), s = ln(p rho^-gamma).  A state enters the
// two-point flux through kTP = 8 quantities: rho, u, v, w, beta = rho/(2p),
// ln rho, ln beta, |u|^2.
constexpr int kTP = 8;
constexpr double kLn2 = 0.69314718055994530942;

__device__ __forceinline__ void two_point_state(const double* U, double gm1, double* P) {
  const double r = U[0], ri = 1.0 / r;
  const double u = U[1] * ri, v = U[2] * ri, w = U[3] * ri;
  const double q2 = fma(u, u, fma(v, v, w * w));
  const double p = gm1 * fma(-0.5 * r, q2, U[4]);
  const double b = 0.5 * r / p;
  P[0] = r;
  P[1] = u;
  P[2] = v;
  P[3] = w;
  P[4] = b;
  P[5] = log(r);
  P[6] = log(b);
  P[7] = q2;
}

// Logarithmic mean (a - b)/(ln a - ln b) from the values and their logs.
// With f = (a - b)/(a + b) and u = f^2: for u < 1e-2 it is
// ((a + b)/2) f/artanh(f), the ratio from its Taylor series in u through u^7
// (f/artanh(f) = 1/(1 + u/3 + u^2/5 + ...); truncation below 2e-18), else the
// quotient of the differences (whose denominator is then at least 0.2).
__device__ __forceinline__ double ln_mean(double a, double b, double la, double lb) {
  const double d = a - b, sm = a + b;
  if (d * d < 1e-2 * sm * sm) {
    const double f = d / sm, u = f * f;
    double g = -5472607916.0 / 488462349375.0;
    g = fma(g, u, -25865068.0 / 1915538625.0);
    g = fma(g, u, -10719068.0 / 638512875.0);
    g = fma(g, u, -10196.0 / 467775.0);
    g = fma(g, u, -428.0 / 14175.0);
    g = fma(g, u, -44.0 / 945.0);
    g = fma(g, u, -4.0 / 45.0);
    g = fma(g, u, -1.0 / 3.0);
    g = fma(g, u, 1.0);
    return 0.5 * sm * g;
  }
  return d / (la - lb);
}

// Chandrashekar's two-point flux F#(L, R) contracted with m:
//   F_rho = rho_ln (u_bar . m),  F_mom = p_hat m + u_bar F_rho,
//   F_E = (1/(2 (gamma-1) beta_ln) - |u|^2_bar/2) F_rho + u_bar . F_mom,
// bars arithmetic means, _ln logarithmic means, p_hat = rho_bar/(2 beta_bar).
__device__ __forceinline__ void two_point_flux(const double* L, int sl, const double* R, int sr, const double* m,
                                               double igm1, double* F) {
  const double rho_ln = ln_mean(L[0], R[0], L[5 * sl], R[5 * sr]);
  // beta: one reciprocal of beta_L + beta_R serves p_hat and the series
  // branch of 1/beta_ln
  const double bL = L[4 * sl], bR = R[4 * sr];
  const double db = bL - bR, sb = bL + bR, isb = 1.0 / sb;
  double ib_ln;
  if (db * db < 1e-2 * sb * sb) {
    const double f = db * isb, u2 = f * f;
    double h = 1.0 / 15.0;
    h = fma(h, u2, 1.0 / 13.0);
    h = fma(h, u2, 1.0 / 11.0);
    h = fma(h, u2, 1.0 / 9.0);
    h = fma(h, u2, 1.0 / 7.0);
    h = fma(h, u2, 1.0 / 5.0);
    h = fma(h, u2, 1.0 / 3.0);
    h = fma(h, u2, 1.0);
    ib_ln = 2.0 * isb * h;
  } else {
    ib_ln = (L[6 * sl] - R[6 * sr]) / db;
  }
  const double u = 0.5 * (L[sl] + R[sr]), v = 0.5 * (L[2 * sl] + R[2 * sr]), w = 0.5 * (L[3 * sl] + R[3 * sr]);
  const double p_hat = 0.5 * (L[0] + R[0]) * isb;
  const double q2 = 0.5 * (L[7 * sl] + R[7 * sr]);
  const double F0 = rho_ln * fma(u, m[0], fma(v, m[1], w * m[2]));
  F[0] = F0;
  F[1] = fma(p_hat, m[0], u * F0);
  F[2] = fma(p_hat, m[1], v * F0);
  F[3] = fma(p_hat, m[2], w * F0);
  F[4] = fma(fma(0.5 * igm1, ib_ln, -0.5 * q2), F0, fma(u, F[1], fma(v, F[2], w * F[3])));
}

// Entropy variables v = ((gamma - s)/(gamma - 1) - beta |u|^2, 2 beta u, -2 beta)
// from the two-point quantities (s = ln p - gamma ln rho, ln p = ln rho - ln(2 beta)).
__device__ __forceinline__ void entropy_variables(const double* P, int sp, double gamma, double* v) {
  const double igm1 = 1.0 / (gamma - 1.0);
  const double lnp = P[5 * sp] - kLn2 - P[6 * sp];
  const double s = lnp - gamma * P[5 * sp];
  const double b2 = 2.0 * P[4 * sp];
  v[0] = fma(gamma - s, igm1, -P[4 * sp] * P[7 * sp]);
  v[1] = b2 * P[sp];
  v[2] = b2 * P[2 * sp];
  v[3] = b2 * P[3 * sp];
  v[4] = -b2;
}

// The inverse: conservative state U and its two-point quantities P from
// entropy variables: beta = -v4/2, u = -v_{1..3}/v4,
// s = gamma - (gamma - 1)(v0 + beta |u|^2), ln rho = -(s + ln(2 beta))/(gamma - 1).
__device__ __forceinline__ void from_entropy_variables(const double* v, double gamma, double* U, double* P) {
  const double igm1 = 1.0 / (gamma - 1.0);
  const double b = -0.5 * v[4];
  const double iv4 = 1.0 / v[4];
  const double u = -v[1] * iv4, vv = -v[2] * iv4, w = -v[3] * iv4;
  const double q2 = fma(u, u, fma(vv, vv, w * w));
  const double s = gamma - (gamma - 1.0) * fma(b, q2, v[0]);
  const double lb = log(b);
  const double lr = -(s + kLn2 + lb) * igm1;
  const double r = exp(lr);
  const double p = 0.5 * r / b;
  U[0] = r;
  U[1] = r * u;
  U[2] = r * vv;
  U[3] = r * w;
  U[4] = fma(p, igm1, 0.5 * r * q2);
  P[0] = r;
  P[1] = u;
  P[2] = vv;
  P[3] = w;
  P[4] = b;
  P[5] = lr;
  P[6] = lb;
  P[7] = q2;
}

// ------------------------------------------------------------------ viscous physics
//
// Navier-Stokes-Fourier fluxes with BR1 lifting of the primitive variables
// W = (rho, u, v, w, p): g[d * 5 + v] = dW_v / dx_d (the lifted gradient),
//   tau  = mu (grad u + grad u^T - 2/3 div u I)          (Stokes hypothesis)
//   F_v[d] = (0, tau_{x d}, tau_{y d}, tau_{z d}, u . tau_{. d} + kappa d(p/rho)/dx_d)
// with kappa = mu gamma / ((gamma - 1) Pr) (Fourier heat flux q = -kappa grad(p/rho)).

__device__ __forceinline__ void primitive(const double* U, double gm1, double* W) {
  const double r = 1.0 / U[0];
  W[0] = U[0];
  W[1] = U[1] * r;
  W[2] = U[2] * r;
  W[3] = U[3] * r;
  W[4] = gm1 * (U[4] - 0.5 * (U[1] * W[1] + U[2] * W[2] + U[3] * W[3]));
}

__device__ __forceinline__ void viscous_flux(const double* W, const double* g, double mu, double kappa,
                                             double Fv[3][5]) {
  const double div = g[1] + g[5 + 2] + g[10 + 3];
  const double rinv = 1.0 / W[0], Tr = W[4] * rinv;
  const double lam = (2.0 / 3.0) * mu * div;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i] = mu * (g[d * 5 + 1 + i] + g[i * 5 + 1 + d]) - (i == d ? lam : 0.0);
    const double dT = (g[d * 5 + 4] - Tr * g[d * 5]) * rinv;
    Fv[d][0] = 0.0;
    Fv[d][1] = tau[0];
    Fv[d][2] = tau[1];
    Fv[d][3] = tau[2];
    Fv[d][4] = W[1] * tau[0] + W[2] * tau[1] + W[3] * tau[2] + kappa * dT;
  }
}

// Reverse mode of viscous_flux: Fb[d][v] cotangent of F_v[d][v]; adds the
// cotangents of W (5) to Wb and of the gradient (15) to gb.
__device__ __forceinline__ void viscous_flux_vjp(const double* W, const double* g, double mu, double kappa,
                                                 const double Fb[3][5], double* Wb, double* gb) {
  const double div = g[1] + g[5 + 2] + g[10 + 3];
  const double rinv = 1.0 / W[0], Tr = W[4] * rinv;
  const double lam = (2.0 / 3.0) * mu * div;
  double lamb = 0.0, rinvb = 0.0, Trb = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double e = Fb[d][4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double tau = mu * (g[d * 5 + 1 + i] + g[i * 5 + 1 + d]) - (i == d ? lam : 0.0);
      const double taub = Fb[d][1 + i] + W[1 + i] * e;
      Wb[1 + i] += tau * e;
      gb[d * 5 + 1 + i] += mu * taub;
      gb[i * 5 + 1 + d] += mu * taub;
      if (i == d) lamb -= taub;
    }
    const double dTb = kappa * e;
    gb[d * 5 + 4] += dTb * rinv;
    gb[d * 5] -= Tr * rinv * dTb;
    Trb -= g[d * 5] * rinv * dTb;
    rinvb += (g[d * 5 + 4] - Tr * g[d * 5]) * dTb;
  }
  Wb[4] += rinv * Trb;
  rinvb += W[4] * Trb;
  Wb[0] -= rinv * rinv * rinvb;
  const double divb = (2.0 / 3.0) * mu * lamb;
  gb[1] += divb;
  gb[5 + 2] += divb;
  gb[10 + 3] += divb;
}

// Reverse mode of primitive: adds the cotangent of U to Ub.
__device__ __forceinline__ void primitive_vjp(const double* U, double gm1, const double* Wb, double* Ub) {
  const double r = 1.0 / U[0];
  const double hp = 0.5 * gm1 * Wb[4];
  double rb = 0.0;
  Ub[4] += gm1 * Wb[4];
#pragma unroll
  for (int i = 1; i <= 3; ++i) {
    const double Wi = U[i] * r;
    const double Wib = Wb[i] - hp * U[i];
    Ub[i] += r * Wib - hp * Wi;
    rb += U[i] * Wib;
  }
  Ub[0] += Wb[0] - r * r * rb;
}

// ------------------------------------------------------------------ adjoint physics
// Hand-written reverse mode of the functions above.  Readings at the kinks:
// d|x|/dx = sign(x) with sign(0) = 0; max(aL, aR) passes its cotangent to the
// left ('-') argument at ties.

__device__ __forceinline__ double sgn0(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// Cotangents of a side's normal-state quantities -> cotangent of U.
// Fb: cotangent of F(U).n; unb, pb, Hb: of u.n, p, H; ub: of u (3).
__device__ __forceinline__ void normal_state_vjp(const double* U, const double* n, double gamma, const NState& s,
                                                 const double* Fb, double unb, double pb, double Hb, double* ub,
                                                 double* Ub) {
  const double gm1 = gamma - 1.0;
  const double u[3] = {U[1] * s.rinv, U[2] * s.rinv, U[3] * s.rinv};
  // F[0] = rho un ; F[1+i] = m_i un + p n_i ; F[4] = (E + p) un
  Ub[0] += Fb[0] * s.un;
  unb += Fb[0] * U[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Ub[1 + i] += Fb[1 + i] * s.un;
    unb += Fb[1 + i] * U[1 + i];
    pb += Fb[1 + i] * n[i];
  }
  Ub[4] += Fb[4] * s.un;
  pb += Fb[4] * s.un;
  unb += Fb[4] * (U[4] + s.p);
  // H = (E + p) / rho
  Ub[4] += Hb * s.rinv;
  pb += Hb * s.rinv;
  Ub[0] -= Hb * s.H * s.rinv;
  // un = u.n
#pragma unroll
  for (int d = 0; d < 3; ++d) ub[d] += unb * n[d];
  // p = (gamma-1)(E - |m|^2 / (2 rho))
  Ub[4] += gm1 * pb;
  const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) Ub[1 + d] -= gm1 * u[d] * pb;
  Ub[0] += 0.5 * gm1 * q2 * pb;
  // u = m / rho
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Ub[1 + d] += ub[d] * s.rinv;
    Ub[0] -= ub[d] * u[d] * s.rinv;
  }
}

// Lax-Friedrichs: given Fsb = cotangent of F*, accumulate UbL, UbR.
__device__ __forceinline__ void flux_lf_vjp(const double* UL, const double* UR, const double* n, double gamma,
                                            const double* Fsb, double* UbL, double* UbR) {
  NState L, R;
  normal_state(UL, n, gamma, L);
  normal_state(UR, n, gamma, R);
  const double cL = sqrt(gamma * L.p * L.rinv), cR = sqrt(gamma * R.p * R.rinv);
  const double aL = fabs(L.un) + cL, aR = fabs(R.un) + cR;
  const double lam = aL >= aR ? aL : aR;
  double Fb[5], lamb = 0.0;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Fb[v] = 0.5 * Fsb[v];
    lamb -= 0.5 * Fsb[v] * (UR[v] - UL[v]);
    UbR[v] -= 0.5 * lam * Fsb[v];
    UbL[v] += 0.5 * lam * Fsb[v];
  }
  const double aLb = aL >= aR ? lamb : 0.0, aRb = aL >= aR ? 0.0 : lamb;
  // c = sqrt(gamma p / rho): dc = gamma dp / (2 c rho) - c drho / (2 rho)
  double ubL[3] = {0, 0, 0}, ubR[3] = {0, 0, 0};
  const double pbL = aLb * gamma * L.rinv / (2.0 * cL), pbR = aRb * gamma * R.rinv / (2.0 * cR);
  UbL[0] -= aLb * 0.5 * cL * L.rinv;
  UbR[0] -= aRb * 0.5 * cR * R.rinv;
  normal_state_vjp(UL, n, gamma, L, Fb, sgn0(L.un) * aLb, pbL, 0.0, ubL, UbL);
  normal_state_vjp(UR, n, gamma, R, Fb, sgn0(R.un) * aRb, pbR, 0.0, ubR, UbR);
}

// Roe: given Fsb = cotangent of F*, accumulate UbL, UbR (reverse of flux_roe).
__device__ __forceinline__ void flux_roe_vjp(const double* UL, const double* UR, const double* n, double gamma,
                                             const double* Fsb, double* UbL, double* UbR) {
  NState L, R;
  normal_state(UL, n, gamma, L);
  normal_state(UR, n, gamma, R);
  // forward recomputation
  const double sL = sqrt(UL[0]), sR = sqrt(UR[0]);
  const double den = 1.0 / (sL + sR);
  const double uL[3] = {UL[1] * L.rinv, UL[2] * L.rinv, UL[3] * L.rinv};
  const double uR[3] = {UR[1] * R.rinv, UR[2] * R.rinv, UR[3] * R.rinv};
  double u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = (sL * uL[d] + sR * uR[d]) * den;
  const double H = (sL * L.H + sR * R.H) * den;
  const double rho = sL * sR;
  const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double gm1 = gamma - 1.0;
  const double c2 = gm1 * (H - 0.5 * q2);
  const double c = sqrt(c2);
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  const double dp = R.p - L.p;
  const double du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  const double dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
  const double ic2 = 1.0 / c2;
  const double a1 = 0.5 * (dp - rho * c * dun) * ic2;
  const double a5 = 0.5 * (dp + rho * c * dun) * ic2;
  const double a2 = (UR[0] - UL[0]) - dp * ic2;
  const double e1 = fabs(un - c), e5 = fabs(un + c), l2 = fabs(un);
  const double l1 = e1 * a1, l5 = e5 * a5;
  double dut[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dut[d] = du[d] - dun * n[d];
  const double udut = u[0] * dut[0] + u[1] * dut[1] + u[2] * dut[2];
  // reverse
  double Db[5], FbL[5], FbR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Db[v] = -0.5 * Fsb[v];
    FbL[v] = FbR[v] = 0.5 * Fsb[v];
  }
  double l1b = 0, l5b = 0, l2b = 0, Hb = 0, cb = 0, unb = 0, a2b = 0, q2b = 0, rhob = 0, udutb = 0;
  double ub[3] = {0, 0, 0}, dutb[3] = {0, 0, 0};
  // D4
  l1b += Db[4] * (H - c * un);
  l5b += Db[4] * (H + c * un);
  l2b += Db[4] * (a2 * 0.5 * q2 + rho * udut);
  Hb += Db[4] * (l1 + l5);
  cb += Db[4] * (l5 - l1) * un;
  unb += Db[4] * (l5 - l1) * c;
  a2b += Db[4] * l2 * 0.5 * q2;
  q2b += Db[4] * l2 * a2 * 0.5;
  rhob += Db[4] * l2 * udut;
  udutb += Db[4] * l2 * rho;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ub[d] += udutb * dut[d];
    dutb[d] += udutb * u[d];
  }
  // D1..D3
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double b = Db[1 + d];
    l1b += b * (u[d] - c * n[d]);
    l5b += b * (u[d] + c * n[d]);
    l2b += b * (a2 * u[d] + rho * dut[d]);
    ub[d] += b * (l1 + l5 + l2 * a2);
    cb += b * (l5 - l1) * n[d];
    a2b += b * l2 * u[d];
    rhob += b * l2 * dut[d];
    dutb[d] += b * l2 * rho;
  }
  // D0
  l1b += Db[0];
  l5b += Db[0];
  l2b += Db[0] * a2;
  a2b += Db[0] * l2;
  // dut = du - dun n
  double dub[3], dunb = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dub[d] = dutb[d];
    dunb -= dutb[d] * n[d];
  }
  // eigenvalue magnitudes
  unb += sgn0(un) * l2b;
  const double s5 = sgn0(un + c), s1 = sgn0(un - c);
  unb += s5 * a5 * l5b + s1 * a1 * l1b;
  cb += s5 * a5 * l5b - s1 * a1 * l1b;
  const double a5b = e5 * l5b, a1b = e1 * l1b;
  // wave strengths
  double dpb = 0, ic2b = 0, drhob = a2b;
  dpb -= a2b * ic2;
  ic2b -= a2b * dp;
  dpb += 0.5 * ic2 * (a5b + a1b);
  rhob += 0.5 * ic2 * c * dun * (a5b - a1b);
  cb += 0.5 * ic2 * rho * dun * (a5b - a1b);
  dunb += 0.5 * ic2 * rho * c * (a5b - a1b);
  ic2b += 0.5 * (dp + rho * c * dun) * a5b + 0.5 * (dp - rho * c * dun) * a1b;
  double c2b = -ic2b * ic2 * ic2;
#pragma unroll
  for (int d = 0; d < 3; ++d) dub[d] += dunb * n[d];
  // un = u.n
#pragma unroll
  for (int d = 0; d < 3; ++d) ub[d] += unb * n[d];
  // c = sqrt(c2), c2 = (gamma-1)(H - q2/2), q2 = |u|^2
  c2b += cb / (2.0 * c);
  Hb += gm1 * c2b;
  q2b -= 0.5 * gm1 * c2b;
#pragma unroll
  for (int d = 0; d < 3; ++d) ub[d] += 2.0 * u[d] * q2b;
  // Roe averages
  double sLb = rhob * sR, sRb = rhob * sL, denb = 0.0;
  double HLb = Hb * sL * den, HRb = Hb * sR * den;
  sLb += Hb * L.H * den;
  sRb += Hb * R.H * den;
  denb += Hb * (sL * L.H + sR * R.H);
  double ubL[3], ubR[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sLb += ub[d] * uL[d] * den;
    sRb += ub[d] * uR[d] * den;
    ubL[d] = ub[d] * sL * den - dub[d];
    ubR[d] = ub[d] * sR * den + dub[d];
    denb += ub[d] * (sL * uL[d] + sR * uR[d]);
  }
  sLb -= denb * den * den;
  sRb -= denb * den * den;
  UbL[0] += sLb / (2.0 * sL) - drhob;
  UbR[0] += sRb / (2.0 * sR) + drhob;
  normal_state_vjp(UL, n, gamma, L, FbL, 0.0, -dpb, HLb, ubL, UbL);
  normal_state_vjp(UR, n, gamma, R, FbR, 0.0, dpb, HRb, ubR, UbR);
}

// Contravariant flux at a volume point (G_l = V_l U + p (0, M_l., V_l),
// V_l = M_l.u) in reverse: Gb[l][v] -> Ub[v].
__device__ __forceinline__ void contravariant_vjp(const double* U, const double M[3][3], double gamma,
                                                  const double Gb[3][5], double* Ub) {
  const double gm1 = gamma - 1.0;
  const double rinv = 1.0 / U[0];
  const double u[3] = {U[1] * rinv, U[2] * rinv, U[3] * rinv};
  const double p = gm1 * (U[4] - 0.5 * (U[1] * u[0] + U[2] * u[1] + U[3] * u[2]));
  const double Ep = U[4] + p;
  double pb = 0.0, ub[3] = {0, 0, 0};
#pragma unroll
  for (int v = 0; v < 5; ++v) Ub[v] = 0.0;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const double Vl = M[l][0] * u[0] + M[l][1] * u[1] + M[l][2] * u[2];
    const double Vb = Gb[l][0] * U[0] + Gb[l][1] * U[1] + Gb[l][2] * U[2] + Gb[l][3] * U[3] + Gb[l][4] * Ep;
    Ub[0] += Gb[l][0] * Vl;
    Ub[1] += Gb[l][1] * Vl;
    Ub[2] += Gb[l][2] * Vl;
    Ub[3] += Gb[l][3] * Vl;
    Ub[4] += Gb[l][4] * Vl;
    pb += Gb[l][1] * M[l][0] + Gb[l][2] * M[l][1] + Gb[l][3] * M[l][2] + Gb[l][4] * Vl;
#pragma unroll
    for (int d = 0; d < 3; ++d) ub[d] += Vb * M[l][d];
  }
  Ub[4] += gm1 * pb;
  const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int d = 0; d < 3; ++d) Ub[1 + d] += ub[d] * rinv - gm1 * u[d] * pb;
  Ub[0] += 0.5 * gm1 * q2 * pb - (ub[0] * u[0] + ub[1] * u[1] + ub[2] * u[2]) * rinv;
}

// ------------------------------------------------------------------ element phases
//
// Every pass gives one lane one output point and carries the 5 conservative
// variables in registers: one coefficient load feeds 5 independent FMA chains
// (instruction-level parallelism for the FP64 pipe) and the index arithmetic
// is done once per output.  Buffers are [var][point] with a var stride of nQ.

#define DG_FMA5(cf, src, stride, acc)            \
  do {                                           \
    const double _c = (cf);                      \
    const double* _s = (src);                    \
    acc[0] = fma(_c, _s[0], acc[0]);             \
    acc[1] = fma(_c, _s[(stride)], acc[1]);      \
    acc[2] = fma(_c, _s[2 * (stride)], acc[2]);  \
    acc[3] = fma(_c, _s[3 * (stride)], acc[3]);  \
    acc[4] = fma(_c, _s[4 * (stride)], acc[4]);  \
  } while (0)

// Modal -> nodal by the sum-factorised passes: sQ [5][nM] (modal
// coefficients) -> U in bufA [5][nQ]; bufB is scratch.
__device__ __forceinline__ void modal_to_nodal_passes(const Ctx& c, const TypeTab& T, const double* sQ, double* bufA,
                                                         double* bufB, int lane) {
  const int n = T.n, nM = T.nM, nQ = T.nQ, n2 = n * n;
  const double* dp = c.dpool;
  const int* ip = c.ipool;
  // c-pass: X[col][k] = sum_t C[col][t][k] Q[moff[col] + t], columns by decreasing length
  {
    const int cnt = T.ncols * n;
    for (int o = lane; o < cnt; o += blockDim.x) {
      int r = o / n, k = o - r * n;
      int col = ip[T.col_order + r];
      int len = ip[T.col_len + col];
      const double* C = dp + T.C + ip[T.col_coff + col] + k;
      const double* q = sQ + ip[T.col_moff + col];
      double acc[5] = {0, 0, 0, 0, 0};
      for (int t = 0; t < len; ++t) DG_FMA5(C[t * n], q + t, nM, acc);
      double* X = bufA + col * n + k;
#pragma unroll
      for (int v = 0; v < 5; ++v) X[v * nQ] = acc[v];
    }
  }
  __syncthreads();
  // b-pass: Y[p][j][k] = sum_t B[p][t][j] X[cbase[p] + t][k]
  for (int o = lane; o < nQ; o += blockDim.x) {
    int p = o / n2, jk = o - p * n2, j = jk / n, k = jk - j * n;
    int blen = ip[T.p_blen + p];
    const double* B = dp + T.B + ip[T.p_boff + p] + j;
    const double* X = bufA + ip[T.p_cbase + p] * n + k;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int t = 0; t < blen; ++t) DG_FMA5(B[t * n], X + t * n, nQ, acc);
#pragma unroll
    for (int v = 0; v < 5; ++v) bufB[v * nQ + o] = acc[v];
  }
  __syncthreads();
  // a-pass: U[i][j][k] = sum_p A[p][i] Y[p][j][k]
  for (int o = lane; o < nQ; o += blockDim.x) {
    int i = o / n2, jk = o - i * n2;
    const double* A = dp + T.A + i;
    const double* Y = bufB + jk;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int p = 0; p < n; ++p) DG_FMA5(A[p * n], Y + p * n2, nQ, acc);
#pragma unroll
    for (int v = 0; v < 5; ++v) bufA[v * nQ + o] = acc[v];
  }
  __syncthreads();
}

// Storage -> nodal: U = V Q in bufA [5][nQ] from a stored element block sQ.
// A hexahedron is stored as s = W^{1/2} V Q, so U = W^{-1/2} s pointwise;
// the other types hold modal coefficients.  sQ may alias bufB.
__device__ __noinline__ void modal_to_nodal(const Ctx& c, const TypeTab& T, const double* sQ, double* bufA,
                                            double* bufB, int lane) {
  if (T.type == HEX) {
    const int nQ = T.nQ;
    const double* rs = c.dpool + T.sqw + nQ;
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = sQ[w] * rs[w % nQ];
    __syncthreads();
    return;
  }
  modal_to_nodal_passes(c, T, sQ, bufA, bufB, lane);
}

// What the nodal->modal pass does with r = M_ref^{-1} V^T bufA of a mode
// (r = V^T bufA without the mass matrix when minv == false):
//   kStore: out[v nM + m] = scale r_v
//   kRk:    K <- a K + dt scale r (a == 0: K <- dt scale r), Q <- Q + b K,
//           and the new Q is also written to sQ when sQ != nullptr.
//   kAxpy:  out[v nM + m] += scale r_v
struct Epilogue {
  enum { kStore = 0, kRk = 1, kAxpy = 2 };
  int kind;
  bool minv;
  double scale;
  double* out;
  const double* Qi;
  double* Qo;
  double* K;
  double* sQ;
  double a, b, dt;
  // curved prism / pyramid: r = Md (V^T bufA) with the element's dense
  // inverse mass matrix Md [nM][nM] (symmetric) instead of minv and scale;
  // rbuf [5][nM] is shared scratch that no other argument aliases
  const double* Md = nullptr;
  double* rbuf = nullptr;
  // true: r is the modal result for a hexahedron too (the conversion to the
  // caller's layout); false: a hexahedron's r is in its scaled nodal storage
  bool modal = false;
};

// The epilogue of one mode given r_v (5 values).  Returns true if a
// non-finite state value was produced.
__device__ __forceinline__ bool epilogue_mode(const Epilogue& ep, int nM, int mode, const double* r) {
  bool bad = false;
  if (ep.kind == Epilogue::kStore) {
#pragma unroll
    for (int v = 0; v < 5; ++v) ep.out[v * nM + mode] = r[v];
  } else if (ep.kind == Epilogue::kAxpy) {
#pragma unroll
    for (int v = 0; v < 5; ++v) ep.out[v * nM + mode] += r[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int idx = v * nM + mode;
      const double R = r[v];
      const double k = (ep.a == 0.0) ? ep.dt * R : fma(ep.a, ep.K[idx], ep.dt * R);
      const double qn = fma(ep.b, k, ep.Qi[idx]);
      ep.K[idx] = k;
      ep.Qo[idx] = qn;
      if (ep.sQ) ep.sQ[idx] = qn;
      bad |= !finite_bits(qn);
    }
  }
  return bad;
}

// Nodal -> modal transpose: bufA [5][nQ] -> modal coefficients through `ep`;
// bufB is scratch.  Returns true if a non-finite state value was produced.
template <bool DENSE>
__device__ __noinline__ bool nodal_to_modal_t(const Ctx& c, const TypeTab& T, double* bufA, double* bufB, int lane,
                                              const Epilogue& ep) {
  const int n = T.n, nM = T.nM, nQ = T.nQ, n2 = n * n;
  const double* dp = c.dpool;
  const int* ip = c.ipool;
  if (!DENSE && T.type == HEX && !ep.modal) {
    // scaled nodal storage: W^{1/2} V M^{-1} V^T h = W^{-1/2} h (M = I)
    const double* rs = dp + T.sqw + nQ;
    bool bad = false;
    for (int q = lane; q < nQ; q += blockDim.x) {
      double acc[5];
      const double f = rs[q] * ep.scale;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = bufA[v * nQ + q] * f;
      bad |= epilogue_mode(ep, nM, q, acc);
    }
    __syncthreads();
    return bad;
  }
  for (int o = lane; o < nQ; o += blockDim.x) {
    int p = o / n2, jk = o - p * n2;
    const double* A = dp + T.A + p * n;
    const double* Hs = bufA + jk;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i) DG_FMA5(A[i], Hs + i * n2, nQ, acc);
#pragma unroll
    for (int v = 0; v < 5; ++v) bufB[v * nQ + o] = acc[v];
  }
  __syncthreads();
  {
    const int cnt = T.ncols * n;
    for (int o = lane; o < cnt; o += blockDim.x) {
      int col = o / n, k = o - col * n;
      int p = ip[T.col_p + col];
      int t = col - ip[T.p_cbase + p];
      const double* B = dp + T.B + ip[T.p_boff + p] + t * n;
      const double* Y = bufB + p * n2 + k;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int j = 0; j < n; ++j) DG_FMA5(B[j], Y + j * n, nQ, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufA[v * nQ + o] = acc[v];
    }
  }
  __syncthreads();
  bool bad = false;
  for (int mode = lane; mode < nM; mode += blockDim.x) {
    int col = ip[T.mode_col + mode];
    int t = mode - ip[T.col_moff + col];
    const double* C = dp + T.C + ip[T.col_coff + col] + t * n;
    const double* X = bufA + col * n;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < n; ++k) DG_FMA5(C[k], X + k, nQ, acc);
    if (DENSE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) ep.rbuf[v * nM + mode] = acc[v];
      continue;
    }
    const double mi = ep.minv ? dp[T.minv + mode] * ep.scale : ep.scale;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] *= mi;
    bad |= epilogue_mode(ep, nM, mode, acc);
  }
  if (DENSE) {
    // dense inverse mass matrix of a curved element (Algorithm 1 with a
    // pointwise J): lanes run over output modes, so the column reads of the
    // symmetric Md are coalesced and every load feeds 5 FMAs
    __syncthreads();
    for (int mode = lane; mode < nM; mode += blockDim.x) {
      const double* Mc = ep.Md + mode;
      double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int j = 0; j < nM; ++j) DG_FMA5(Mc[(size_t)j * nM], ep.rbuf + j, nM, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] *= ep.scale;
      bad |= epilogue_mode(ep, nM, mode, acc);
    }
  }
  __syncthreads();
  return bad;
}

// ANY: the launch may meet curved elements (their variants are compiled into
// the kernel only then, so affine launches keep the affine register budget).
template <bool ANY>
__device__ __forceinline__ bool nodal_to_modal(const Ctx& c, const TypeTab& T, double* bufA, double* bufB, int lane,
                                               const Epilogue& ep) {
  return (ANY && ep.Md) ? nodal_to_modal_t<true>(c, T, bufA, bufB, lane, ep)
                        : nodal_to_modal_t<false>(c, T, bufA, bufB, lane, ep);
}

// Values of the nodal field `src` [5][nQ] on the element's own face points,
// times `scale`, written to the face buffer `dst` at the element's side slots.
__device__ __forceinline__ void write_traces(const Ctx& c, const TypeTab& T, int64_t s, const double* src,
                                             double* dst, double scale, int lane, int ft_mult = 1,
                                             int64_t ft_add = 0) {
  const int n = T.n, nQ = T.nQ, n2 = n * n;
  const double* dp = c.dpool;
  const int cnt = T.nfaces * n2;
  const int64_t* ft = c.slot_ftoff + s * 6;
  for (int w = lane; w < cnt; w += blockDim.x) {
    int lf = w / n2, p = w - lf * n2;
    int ia = p % n, ib = p / n;
    const FaceDesc d = T.faces[lf];
    int sa = d.alpha == 0 ? n2 : (d.alpha == 1 ? n : 1);
    int sb = d.beta == 0 ? n2 : (d.beta == 1 ? n : 1);
    int sf = d.fixed == 0 ? n2 : (d.fixed == 1 ? n : 1);
    const double* e = dp + T.ext + d.end * n;
    const double* U = src + ia * sa + ib * sb;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < n; ++m) DG_FMA5(e[m], U + m * sf, nQ, acc);
    double* out = dst + ft_mult * ft[lf] + ft_add + p;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * n2] = scale * acc[v];
  }
}

// Structurally nonzero entries of d(a,b,c)_l / d(xi)_k per type: bit l*3+k.
// hex: diagonal; prism: a(xi, eta); pyramid: a(xi, zeta), b(eta, zeta);
// tet: a(xi, eta, zeta), b(eta, zeta); c = zeta for all.
__constant__ unsigned kMetricMask[4] = {0x111u, 0x113u, 0x135u, 0x137u};

// M = (w_q d(a,b,c)/d(xi)) (J dxi/dx) at volume point q, using each
// collapse's sparsity (hex: diagonal; prism, pyramid, tet: triangular).
__device__ __forceinline__ void point_metric(int type, const double* wa, const double* Jg, double M[3][3]) {
  switch (type) {
    case HEX: {
      double w0 = wa[0];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int d = 0; d < 3; ++d) M[l][d] = w0 * Jg[l * 3 + d];
      break;
    }
    case PRISM: {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        M[0][d] = wa[0] * Jg[d] + wa[1] * Jg[3 + d];
        M[1][d] = wa[4] * Jg[3 + d];
        M[2][d] = wa[8] * Jg[6 + d];
      }
      break;
    }
    case PYR: {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        M[0][d] = wa[0] * Jg[d] + wa[2] * Jg[6 + d];
        M[1][d] = wa[4] * Jg[3 + d] + wa[5] * Jg[6 + d];
        M[2][d] = wa[8] * Jg[6 + d];
      }
      break;
    }
    default: {  // TET
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        M[0][d] = wa[0] * Jg[d] + wa[1] * Jg[3 + d] + wa[2] * Jg[6 + d];
        M[1][d] = wa[4] * Jg[3 + d] + wa[5] * Jg[6 + d];
        M[2][d] = wa[8] * Jg[6 + d];
      }
      break;
    }
  }
}

// Forward phase of an affine hexahedron in the entropy-stable split form
// (hybridised Gauss SBP operator along every coordinate line):
//   r_i = - sum_j S_ij F#(u_i, u_j) - sum_f s_f E_f,i F#(u_i, u~_f)
//         + sum_f s_f E_f,i sum_j E_f,j F#(u~_f, u_j),
// S = W D - (W D)^T, E_f the extrapolation to the line's end f (s_- = -1,
// s_+ = +1), F# contracted with the line direction's metric J dxi_l/dx, u~_f
// the entropy-projected face state u(E_f v(u)); H_q = sum_l w_perp r_q^(l)
// with w_perp the product of the two other directions' weights.  For a
// central F# this is the weak form's H (sum_l D_l^T G_l).  The face states
// u~ are this element's traces (the face kernel takes the Riemann flux on
// them).  Every unordered node pair and every (face state, node) pair of a
// line is evaluated once per direction (F# is symmetric) into shared memory,
// then every node sums its line's terms.  sQ lives at the start of bufG;
// workspace: bufA [5 nQ] (nodal state, then entropy variables, then the
// accumulated H), bufG: [kTP][nQ] two-point quantities, [kTP][6 n^2] of the
// face states, then one direction's [n^2][n(n-1)/2][5] pair fluxes and
// [n^2][2][n][5] face-state fluxes.
__device__ __noinline__ void element_forward_split(const Ctx& c, const TypeTab& T, int64_t s, double* bufA,
                                                   double* bufG, int lane) {
  const int n = T.n, nQ = T.nQ, n2 = n * n, nF = 6 * n2;
  const double* dp = c.dpool;
  const double gamma = c.gamma, gm1 = gamma - 1.0, igm1 = 1.0 / gm1;
  modal_to_nodal(c, T, bufG, bufA, bufG, lane);
  double* P = bufG;
  double* Pf = P + kTP * nQ;
  double* Gs = Pf + kTP * nF;
  // nodal two-point quantities; the entropy variables overwrite U in place
  for (int q = lane; q < nQ; q += blockDim.x) {
    double U[5], Pq[kTP], v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = bufA[k * nQ + q];
    two_point_state(U, gm1, Pq);
#pragma unroll
    for (int k = 0; k < kTP; ++k) P[k * nQ + q] = Pq[k];
    entropy_variables(Pq, 1, gamma, v);
#pragma unroll
    for (int k = 0; k < 5; ++k) bufA[k * nQ + q] = v[k];
  }
  __syncthreads();
  // entropy-projected face states: extrapolate v along the face-normal
  // coordinate, map back; they are the element's traces
  const int64_t* ft = c.slot_ftoff + s * 6;
  for (int w = lane; w < nF; w += blockDim.x) {
    const int lf = w / n2, p = w - lf * n2;
    const int ia = p % n, ib = p / n;
    const FaceDesc d = T.faces[lf];
    const int sa = d.alpha == 0 ? n2 : (d.alpha == 1 ? n : 1);
    const int sb = d.beta == 0 ? n2 : (d.beta == 1 ? n : 1);
    const int sf = d.fixed == 0 ? n2 : (d.fixed == 1 ? n : 1);
    const double* e = dp + T.ext + d.end * n;
    const double* V = bufA + ia * sa + ib * sb;
    double vt[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < n; ++m) DG_FMA5(e[m], V + m * sf, nQ, vt);
    double U[5], Pp[kTP];
    from_entropy_variables(vt, gamma, U, Pp);
    double* out = c.T + ft[lf] + p;
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k * n2] = U[k];
#pragma unroll
    for (int k = 0; k < kTP; ++k) Pf[k * nF + w] = Pp[k];
  }
  __syncthreads();
  const ElemGeo& g = c.geo[s];
  const double* S = dp + T.sbp;
  const double* w1 = dp + T.w1;
  const double* E = dp + T.ext;
  const int np = n * (n - 1) / 2;         // unordered node pairs of a line
  double* Fp = Gs;                        // [n^2 lines][np][5] pair fluxes of one direction
  double* Ff = Fp + (size_t)n2 * np * 5;  // [n^2 lines][2 ends][n][5] face-state fluxes of one direction
  // the local face at the end `end` of coordinate l, and the index of a face
  // point from the two other coordinates' indices (x1 < x2 by coordinate)
  auto face_of = [&](int l, int end) {
    int lf = 0;
    for (int k = 0; k < 6; ++k)
      if (T.faces[k].fixed == l && T.faces[k].end == end) lf = k;
    return lf;
  };
  auto face_point = [&](int lf, int l, int x1, int x2) {
    const FaceDesc d = T.faces[lf];
    const int o1 = l == 0 ? 1 : 0;
    const int ia = d.alpha == o1 ? x1 : x2, ib = d.beta == o1 ? x1 : x2;
    return lf * n2 + ia + ib * n;
  };
  // H accumulates in bufA (the entropy variables are no longer needed)
  for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = 0.0;
  const int st[3] = {n2, n, 1};
#pragma unroll 1
  for (int l = 0; l < 3; ++l) {
    const int o1 = l == 0 ? 1 : 0, o2 = l == 2 ? 1 : 2;
    const double m[3] = {g.Jg[3 * l], g.Jg[3 * l + 1], g.Jg[3 * l + 2]};
    const int lf_end[2] = {face_of(l, 0), face_of(l, 1)};
    // every unordered node pair and every (face state, node) pair of every
    // line of this direction once (F# is symmetric)
    const int tasks = n2 * (np + 2 * n);
    for (int t = lane; t < tasks; t += blockDim.x) {
      double F[5];
      int line, k;
      if (t < n2 * np) {
        line = t / np;
        k = t - line * np;
        int i = 0, kk = k;
        while (kk >= n - 1 - i) {
          kk -= n - 1 - i;
          ++i;
        }
        const int j = i + 1 + kk;
        const int x1 = line / n, x2 = line - x1 * n;
        const int base = x1 * st[o1] + x2 * st[o2];
        two_point_flux(P + base + i * st[l], nQ, P + base + j * st[l], nQ, m, igm1, F);
        double* out = Fp + ((size_t)line * np + k) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v] = F[v];
      } else {
        const int u = t - n2 * np;
        line = u / (2 * n);
        const int rem = u - line * 2 * n, end = rem / n, j = rem - end * n;
        const int x1 = line / n, x2 = line - x1 * n;
        const int base = x1 * st[o1] + x2 * st[o2];
        two_point_flux(Pf + face_point(lf_end[end], l, x1, x2), nF, P + base + j * st[l], nQ, m, igm1, F);
        double* out = Ff + (((size_t)line * 2 + end) * n + j) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v] = F[v];
      }
    }
    __syncthreads();
    // per node: the line's terms of this direction
    for (int q = lane; q < nQ; q += blockDim.x) {
      const int idx[3] = {q / n2, (q / n) % n, q % n};
      const int x1 = idx[o1], x2 = idx[o2], ii = idx[l];
      const int line = x1 * n + x2;
      const double* Fl = Fp + (size_t)line * np * 5;
      double r[5] = {0, 0, 0, 0, 0};
      for (int j = 0; j < n; ++j) {
        if (j == ii) continue;
        const int i0 = ii < j ? ii : j, j0 = ii < j ? j : ii;
        const double* F = Fl + (i0 * (2 * n - i0 - 1) / 2 + (j0 - i0 - 1)) * 5;
        const double sij = -S[ii * n + j];
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = fma(sij, F[k], r[k]);
      }
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        const double* Fe = Ff + ((size_t)line * 2 + end) * n * 5;
        double G[5] = {0, 0, 0, 0, 0};
        for (int j = 0; j < n; ++j) {
          const double ej = E[end * n + j];
#pragma unroll
          for (int k = 0; k < 5; ++k) G[k] = fma(ej, Fe[j * 5 + k], G[k]);
        }
        const double se = (end ? 1.0 : -1.0) * E[end * n + ii];
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = fma(se, G[k] - Fe[ii * 5 + k], r[k]);
      }
      const double wp = w1[x1] * w1[x2];
#pragma unroll
      for (int k = 0; k < 5; ++k) bufA[k * nQ + q] = fma(wp, r[k], bufA[k * nQ + q]);
    }
    __syncthreads();
  }
  double* H = c.H + c.slot_hoff[s];
  for (int w = lane; w < 5 * nQ; w += blockDim.x) H[w] = bufA[w];
  __syncthreads();
}

// Forward phase of the element at slot s: nodal state, own-face traces and
// the nodal volume residual H.  sQ lives at the start of bufG.
template <bool CURVED>
__device__ __noinline__ void element_forward_t(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufG,
                                                  int lane) {
  const int n = T.n, nQ = T.nQ, n2 = n * n;
  const double* dp = c.dpool;
  modal_to_nodal(c, T, bufG, bufA, bufG, lane);
  write_traces(c, T, s, bufA, c.T, 1.0, lane);
  if (c.Usave) {
    // kept for the adjoint (reverse LSERK with stored stage data)
    double* Un = c.Usave + c.slot_hoff[s];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) Un[w] = bufA[w];
  }
  if (c.ns) {
    // Navier-Stokes: the volume residual needs the lifted gradient, which
    // needs the neighbours' traces; keep the nodal state for that phase.
    double* Un = c.Unod + c.slot_hoff[s];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) Un[w] = bufA[w];
    __syncthreads();
    return;
  }
  // contravariant fluxes G_l at the volume points (bufG, [3][5][nQ])
  const ElemGeo& g = c.geo[s];
  double Jg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Jg[k] = g.Jg[k];
  // a curved element reads its pointwise metric w (da/dxi)(J dxi/dx) instead
  const double* cm = CURVED ? c.cpool + c.slot_coff[s] : nullptr;
  // moving mesh: the mesh velocity at the volume points
  const double* xd = (CURVED && c.mpool) ? c.mpool + c.slot_moff[s] + 31 * nQ : nullptr;
  const double gm1 = c.gamma - 1.0;
  for (int q = lane; q < nQ; q += blockDim.x) {
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = bufA[v * nQ + q];
    double M[3][3];
    if (CURVED) {
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int d = 0; d < 3; ++d) M[l][d] = cm[(l * 3 + d) * nQ + q];
    } else {
      point_metric(T.type, dp + T.wA + q * 9, Jg, M);
    }
    double rinv = 1.0 / U[0];
    double u = U[1] * rinv, v = U[2] * rinv, w = U[3] * rinv;
    double p = gm1 * (U[4] - 0.5 * (U[1] * u + U[2] * v + U[3] * w));
    double Ep = U[4] + p;
    if (CURVED && xd) {
      // moving frame: (F(U) - U xdot) through the metric, W_l = M_l . xdot
      const double x0 = xd[q], x1 = xd[nQ + q], x2 = xd[2 * nQ + q];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double Vl = M[l][0] * u + M[l][1] * v + M[l][2] * w;
        const double Rl = Vl - (M[l][0] * x0 + M[l][1] * x1 + M[l][2] * x2);
        double* G = bufG + l * 5 * nQ + q;
        G[0] = Rl * U[0];
        G[nQ] = Rl * U[1] + p * M[l][0];
        G[2 * nQ] = Rl * U[2] + p * M[l][1];
        G[3 * nQ] = Rl * U[3] + p * M[l][2];
        G[4 * nQ] = Rl * U[4] + Vl * p;
      }
      continue;
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double Vl = M[l][0] * u + M[l][1] * v + M[l][2] * w;
      double* G = bufG + l * 5 * nQ + q;
      G[0] = Vl * U[0];
      G[nQ] = Vl * U[1] + p * M[l][0];
      G[2 * nQ] = Vl * U[2] + p * M[l][1];
      G[3 * nQ] = Vl * U[3] + p * M[l][2];
      G[4 * nQ] = Vl * Ep;
    }
  }
  __syncthreads();
  // H = sum_l D_l^T G_l (collocation derivative along each collapsed direction)
  {
    const double* Dt = dp + T.Dt;
    double* H = c.H + c.slot_hoff[s];
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      const double* G0 = bufG + jk;
      const double* G1 = bufG + 5 * nQ + i * n2 + k;
      const double* G2 = bufG + 10 * nQ + i * n2 + j * n;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[i * n + m], G0 + m * n2, nQ, acc);
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[j * n + m], G1 + m * n, nQ, acc);
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[k * n + m], G2 + m, nQ, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) H[v * nQ + o] = acc[v];
    }
  }
  __syncthreads();
}

template <bool ANY>
__device__ __forceinline__ void element_forward(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufG,
                                                int lane) {
  if (ANY && c.slot_coff[s] >= 0) element_forward_t<true>(c, T, s, bufA, bufG, lane);
  else if (c.split && T.type == HEX) element_forward_split(c, T, s, bufA, bufG, lane);
  else element_forward_t<false>(c, T, s, bufA, bufG, lane);
}

// Backward phase, first half: bufA = H + sign sum_faces E_f^T F_f with the
// face values F_f read from `faces` (the lifted fluxes with sign -1; the
// adjoint's trace cotangents with sign +1).  They are staged into bufG with
// coalesced loads first.
template <bool PSCALE>
__device__ __noinline__ void element_lift_t(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufG,
                                            int lane, const double* faces, double sign, const double* pscale) {
  const int n = T.n, nQ = T.nQ, n2 = n * n, nf = T.nfaces;
  const double* dp = c.dpool;
  const int64_t* ft = c.slot_ftoff + s * 6;
  {
    const int per = 5 * n2;
    for (int w = lane; w < nf * per; w += blockDim.x) {
      int lf = w / per, r = w - lf * per;
      bufG[w] = faces[ft[lf] + r];
    }
  }
  __syncthreads();
  const double* H = c.H + c.slot_hoff[s];
  for (int o = lane; o < nQ; o += blockDim.x) {
    int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
    double h[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) h[v] = H[v * nQ + o];
    for (int lf = 0; lf < nf; ++lf) {
      const FaceDesc d = T.faces[lf];
      int m = sel3(i, j, k, d.fixed);
      int p = sel3(i, j, k, d.alpha) + n * sel3(i, j, k, d.beta);
      DG_FMA5(sign * dp[T.ext + d.end * n + m], bufG + lf * 5 * n2 + p, n2, h);
    }
    if (PSCALE) {
      // curved hexahedron: M^{-1} V^T = V^T diag(1/J) (V square, V^T W V = I)
      const double sc = pscale[o];
#pragma unroll
      for (int v = 0; v < 5; ++v) h[v] *= sc;
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) bufA[v * nQ + o] = h[v];
  }
  __syncthreads();
}

template <bool ANY>
__device__ __forceinline__ void element_lift(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufG,
                                             int lane, const double* faces, double sign,
                                             const double* pscale = nullptr) {
  if (ANY && pscale) element_lift_t<true>(c, T, s, bufA, bufG, lane, faces, sign, pscale);
  else element_lift_t<false>(c, T, s, bufA, bufG, lane, faces, sign, nullptr);
}

// BR1 lifting face term: bufA += sum_f coef_f E_f^T L_f with coef_f =
// sign n_d(f), n(f) the element's outward unit normal of local face f and
// L_f the face values at its own points (staged through bufS).
template <bool CURVED>
__device__ __noinline__ void lift_scaled_t(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufS,
                                           int lane, const double* faces, int d, double sign) {
  const int n = T.n, nQ = T.nQ, n2 = n * n, nf = T.nfaces;
  const double* dp = c.dpool;
  const int64_t* ft = c.slot_ftoff + s * 6;
  {
    // curved: the normal varies over the face; it multiplies the staged
    // face values point by point (c.snrm holds each side's own normals)
    const int per = 5 * n2;
    for (int w = lane; w < nf * per; w += blockDim.x) {
      int lf = w / per, r = w - lf * per;
      double v = faces[ft[lf] + r];
      if (CURVED) v *= sign * c.snrm[3 * (ft[lf] / 5) + d * n2 + r % n2];
      bufS[w] = v;
    }
  }
  __syncthreads();
  double coef[6];
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) coef[lf] = lf < nf ? (CURVED ? 1.0 : sign * c.fnrm[(s * 6 + lf) * 3 + d]) : 0.0;
  for (int o = lane; o < nQ; o += blockDim.x) {
    int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
    double h[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) h[v] = bufA[v * nQ + o];
    for (int lf = 0; lf < nf; ++lf) {
      const FaceDesc fd = T.faces[lf];
      int m = sel3(i, j, k, fd.fixed);
      int p = sel3(i, j, k, fd.alpha) + n * sel3(i, j, k, fd.beta);
      DG_FMA5(coef[lf] * dp[T.ext + fd.end * n + m], bufS + lf * 5 * n2 + p, n2, h);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) bufA[v * nQ + o] = h[v];
  }
  __syncthreads();
}

// Navier-Stokes volume phase of the element at slot s (after the lifting face
// phase).  Per direction d the BR1 lifted gradient of W = (rho, u, v, w, p):
//   nodal  Hd = sum_l D_l^T (w J da_l/dx_d W)          (volume term, as H)
//   modal  G_d = -(1/J) M_ref^{-1} V^T (Hd - sum_f n_d(f) E_f^T L_f)
//   nodal  grad_d W = V G_d, and its traces on the own face points (Vt);
// then the total flux F_e(U) - F_v(U, grad W) at the volume points and
// H = sum_l D_l^T G_l(F) as in the Euler forward phase.
// smem: bufU [5 nQ] | bufDW [3][5][nQ] | bufG [15 nQ] | bufA [5 nQ].
template <bool CURVED>
__device__ __noinline__ void element_ns_volume_t(const Ctx& c, const TypeTab& T, int64_t s, double* smem, int lane) {
  const int n = T.n, nQ = T.nQ, n2 = n * n;
  // curved element: pointwise metric [9][nQ], J, 1/J, (prism, pyramid) dense M_e^{-1}
  const double* cblk = CURVED ? c.cpool + c.slot_coff[s] : nullptr;
  const int nQm = c.nQmax;
  double* bufU = smem;
  double* bufDW = smem + 5 * nQm;
  double* bufG = smem + 20 * nQm;
  double* bufA = smem + 35 * nQm;
  const double* dp = c.dpool;
  const double* Dt = dp + T.Dt;
  const double gm1 = c.gamma - 1.0;
  const ElemGeo& g = c.geo[s];
  double Jg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Jg[k] = g.Jg[k];
  // moving mesh (lift_phase != 0): prisms and pyramids split at the lifting's
  // M(t)^{-1}; hexahedra run whole in phase 2
  const bool dense_split = CURVED && c.lift_phase != 0 && T.type != HEX;
  if (CURVED && c.lift_phase == 1 && !dense_split) return;
  {
    const double* Un = c.Unod + c.slot_hoff[s];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufU[w] = Un[w];
  }
  __syncthreads();
  if (dense_split && c.lift_phase == 2) {
    // the solved modal gradient of every direction: nodal values, traces
    for (int d = 0; d < 3; ++d) {
      double* dW = bufDW + d * 5 * nQ;
      const double* Gm = c.lift + (int64_t)d * c.lift_stride + c.slot_qoff[s];
      double* sG = bufG + 5 * nQ;
      for (int w = lane; w < 5 * T.nM; w += blockDim.x) sG[w] = Gm[w];
      __syncthreads();
      modal_to_nodal(c, T, sG, dW, bufG, lane);
      write_traces(c, T, s, dW, c.Vt, 1.0, lane, 3, (int64_t)d * 5 * n2);
      __syncthreads();
    }
  } else {
  // Lifting volume terms through the reference directions: with
  // M[l][d] = sum_k wA[l][k] Jg[k][d] (wA = w da_l/dxi_k, structurally sparse
  // per type), Hd = sum_l D_l^T (M[l][d] W) = sum_k Jg[k][d] P_k with
  // P_k = sum_{l: wA[l][k] != 0} D_l^T (wA[l][k] W): 3 (hex) to 6 (tet)
  // directional passes instead of 9.  H_0..H_2 accumulate in bufDW.
  for (int q = lane; q < nQ; q += blockDim.x) {
    double U[5], W[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = bufU[v * nQ + q];
    primitive(U, gm1, W);
#pragma unroll
    for (int v = 0; v < 5; ++v) bufA[v * nQ + q] = W[v];
  }
  __syncthreads();
  if (CURVED) {
    // pointwise metric: Hd = sum_l D_l^T (M_q[l][d] W), one full set of
    // directional passes per direction d
    for (int d = 0; d < 3; ++d) {
      for (int q = lane; q < nQ; q += blockDim.x) {
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          const double f = cblk[(l * 3 + d) * nQ + q];
#pragma unroll
          for (int v = 0; v < 5; ++v) bufG[(l * 5 + v) * nQ + q] = f * bufA[v * nQ + q];
        }
      }
      __syncthreads();
      for (int o = lane; o < nQ; o += blockDim.x) {
        int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
        const double* G0 = bufG + jk;
        const double* G1 = bufG + 5 * nQ + i * n2 + k;
        const double* G2 = bufG + 10 * nQ + i * n2 + j * n;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[i * n + m], G0 + m * n2, nQ, acc);
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[j * n + m], G1 + m * n, nQ, acc);
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[k * n + m], G2 + m, nQ, acc);
        double* Hd = bufDW + d * 5 * nQ + o;
#pragma unroll
        for (int v = 0; v < 5; ++v) Hd[v * nQ] = acc[v];
      }
      __syncthreads();
    }
  }
  const unsigned nz = kMetricMask[T.type];
  for (int kr = 0; kr < (CURVED ? 0 : 3); ++kr) {
    const bool u0 = (nz >> (0 * 3 + kr)) & 1u, u1 = (nz >> (1 * 3 + kr)) & 1u, u2 = (nz >> (2 * 3 + kr)) & 1u;
    for (int q = lane; q < nQ; q += blockDim.x) {
      const double* wa = dp + T.wA + q * 9;
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if (!((nz >> (l * 3 + kr)) & 1u)) continue;
        const double f = wa[l * 3 + kr];
#pragma unroll
        for (int v = 0; v < 5; ++v) bufG[(l * 5 + v) * nQ + q] = f * bufA[v * nQ + q];
      }
    }
    __syncthreads();
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      double acc[5] = {0, 0, 0, 0, 0};
      if (u0) {
        const double* G0 = bufG + jk;
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[i * n + m], G0 + m * n2, nQ, acc);
      }
      if (u1) {
        const double* G1 = bufG + 5 * nQ + i * n2 + k;
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[j * n + m], G1 + m * n, nQ, acc);
      }
      if (u2) {
        const double* G2 = bufG + 10 * nQ + i * n2 + j * n;
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[k * n + m], G2 + m, nQ, acc);
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double* Hd = bufDW + d * 5 * nQ + o;
        const double jkd = Jg[kr * 3 + d];
#pragma unroll
        for (int v = 0; v < 5; ++v) Hd[v * nQ] = kr == 0 ? jkd * acc[v] : fma(jkd, acc[v], Hd[v * nQ]);
      }
    }
    __syncthreads();
  }
  for (int d = 0; d < 3; ++d) {
    {
      const double* Hd = bufDW + d * 5 * nQ;
      for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = Hd[w];
    }
    __syncthreads();
    lift_scaled_t<CURVED>(c, T, s, bufA, bufG, lane, c.L, d, -1.0);
    double* dW = bufDW + d * 5 * nQ;
    if (T.type == HEX) {
      // V is square for the hexahedron, so V M^{-1} V^T = (W J)^{-1}: the
      // projection onto the modal space is the identity at the nodes
      const double* wq = dp + T.W;
      if (CURVED) {
        const double* iJ = cblk + 10 * nQ;
        for (int w = lane; w < 5 * nQ; w += blockDim.x) dW[w] = -iJ[w % nQ] * bufA[w] / wq[w % nQ];
      } else {
        for (int w = lane; w < 5 * nQ; w += blockDim.x) dW[w] = -g.invJ * bufA[w] / wq[w % nQ];
      }
      __syncthreads();
    } else if (dense_split) {
      // phase 1: r_d = -V^T (lifting terms); M(t)^{-1} r_d is solved outside
      Epilogue ep{Epilogue::kStore, false, -1.0, c.lift + (int64_t)d * c.lift_stride + c.slot_qoff[s], nullptr,
                  nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
      nodal_to_modal<false>(c, T, bufA, bufG, lane, ep);
      continue;
    } else {
      double* sG = bufG + 5 * nQ;
      Epilogue ep{Epilogue::kStore, true, CURVED ? -1.0 : -g.invJ, sG, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
      if (CURVED) {
        ep.Md = cblk + 11 * nQ;
        ep.rbuf = bufG + 10 * nQ;
      }
      nodal_to_modal<CURVED>(c, T, bufA, bufG, lane, ep);
      modal_to_nodal(c, T, sG, dW, bufG, lane);
    }
    write_traces(c, T, s, dW, c.Vt, 1.0, lane, 3, (int64_t)d * 5 * n2);
    if (c.DW) {
      double* out = c.DW + 3 * c.slot_hoff[s] + d * 5 * nQ;
      for (int w = lane; w < 5 * nQ; w += blockDim.x) out[w] = dW[w];
    }
    __syncthreads();
  }
  if (dense_split) return;   // phase 1 ends with the lifting residuals
  }
  // total contravariant flux G_l = sum_d M[l][d] (F_e - F_v)_d
  for (int q = lane; q < nQ; q += blockDim.x) {
    double U[5], W[5], gr[15];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = bufU[v * nQ + q];
#pragma unroll
    for (int t = 0; t < 15; ++t) gr[t] = bufDW[t * nQ + q];
    primitive(U, gm1, W);
    double Fv[3][5];
    viscous_flux(W, gr, c.mu, c.kappa, Fv);
    double M[3][3];
    if (CURVED) {
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) M[l][dd] = cblk[(l * 3 + dd) * nQ + q];
    } else {
      point_metric(T.type, dp + T.wA + q * 9, Jg, M);
    }
    const double u = W[1], v = W[2], w = W[3], p = W[4], Ep = U[4] + p;
    if (CURVED && c.mpool) {
      // moving mesh: the convective flux in the moving frame, F(U) - U xdot
      const double* xd = c.mpool + c.slot_moff[s] + 31 * nQ;
      const double x0 = xd[q], x1 = xd[nQ + q], x2 = xd[2 * nQ + q];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double Vl = M[l][0] * u + M[l][1] * v + M[l][2] * w;
        const double Rl = Vl - (M[l][0] * x0 + M[l][1] * x1 + M[l][2] * x2);
        double* G = bufG + l * 5 * nQ + q;
        G[0] = Rl * U[0];
        G[nQ] = Rl * U[1] + p * M[l][0] - (M[l][0] * Fv[0][1] + M[l][1] * Fv[1][1] + M[l][2] * Fv[2][1]);
        G[2 * nQ] = Rl * U[2] + p * M[l][1] - (M[l][0] * Fv[0][2] + M[l][1] * Fv[1][2] + M[l][2] * Fv[2][2]);
        G[3 * nQ] = Rl * U[3] + p * M[l][2] - (M[l][0] * Fv[0][3] + M[l][1] * Fv[1][3] + M[l][2] * Fv[2][3]);
        G[4 * nQ] = Rl * U[4] + Vl * p - (M[l][0] * Fv[0][4] + M[l][1] * Fv[1][4] + M[l][2] * Fv[2][4]);
      }
      continue;
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double Vl = M[l][0] * u + M[l][1] * v + M[l][2] * w;
      double* G = bufG + l * 5 * nQ + q;
      G[0] = Vl * U[0];
      G[nQ] = Vl * U[1] + p * M[l][0] - (M[l][0] * Fv[0][1] + M[l][1] * Fv[1][1] + M[l][2] * Fv[2][1]);
      G[2 * nQ] = Vl * U[2] + p * M[l][1] - (M[l][0] * Fv[0][2] + M[l][1] * Fv[1][2] + M[l][2] * Fv[2][2]);
      G[3 * nQ] = Vl * U[3] + p * M[l][2] - (M[l][0] * Fv[0][3] + M[l][1] * Fv[1][3] + M[l][2] * Fv[2][3]);
      G[4 * nQ] = Vl * Ep - (M[l][0] * Fv[0][4] + M[l][1] * Fv[1][4] + M[l][2] * Fv[2][4]);
    }
  }
  __syncthreads();
  {
    double* H = c.H + c.slot_hoff[s];
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      const double* G0 = bufG + jk;
      const double* G1 = bufG + 5 * nQ + i * n2 + k;
      const double* G2 = bufG + 10 * nQ + i * n2 + j * n;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[i * n + m], G0 + m * n2, nQ, acc);
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[j * n + m], G1 + m * n, nQ, acc);
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[k * n + m], G2 + m, nQ, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) H[v * nQ + o] = acc[v];
    }
  }
  __syncthreads();
}

template <bool ANY>
__device__ __forceinline__ void element_ns_volume(const Ctx& c, const TypeTab& T, int64_t s, double* smem, int lane) {
  if (ANY && c.slot_coff[s] >= 0) element_ns_volume_t<true>(c, T, s, smem, lane);
  else element_ns_volume_t<false>(c, T, s, smem, lane);
}

// One element at slot s.  smem per block: bufA [5 nQmax], bufG [15 nQmax]
// (40 nQmax for the Navier-Stokes volume phase).
template <int MODE, bool ANY>
__device__ __forceinline__ void process_element(const Ctx& c, const StageArgs& io, int64_t s, double* bufA,
                                                double* bufG, int lane) {
  const TypeTab& T = c.tabs[c.slot_tab[s]];
  const int nM = T.nM, nQ = T.nQ;
  const int64_t qoff = c.slot_qoff[s];
  if (MODE == kNsVolume) {
    element_ns_volume<ANY>(c, T, s, bufA, lane);
    return;
  }
  if (MODE == kGather) {
    // hexahedra only: caller modal coefficients Q -> storage s = W^{1/2} V Q
    const double* Q = io.Qin + c.elem_qoff[c.elem_of_slot[s]];
    for (int w = lane; w < 5 * nM; w += blockDim.x) bufG[w] = Q[w];
    __syncthreads();
    modal_to_nodal_passes(c, T, bufG, bufA, bufG, lane);
    const double* sq = c.dpool + T.sqw;
    double* out = io.Qout + qoff;
    for (int w = lane; w < 5 * nQ; w += blockDim.x) out[w] = bufA[w] * sq[w % nQ];
    __syncthreads();
    return;
  }
  if (MODE == kScatter) {
    // hexahedra only: storage s -> caller modal coefficients V^T W^{1/2} s
    const double* S = io.Qin + qoff;
    const double* sq = c.dpool + T.sqw;
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = S[w] * sq[w % nQ];
    __syncthreads();
    Epilogue ep{Epilogue::kStore, false, 1.0, io.Qout + c.elem_qoff[c.elem_of_slot[s]], nullptr, nullptr, nullptr,
                nullptr, 0.0, 0.0, 0.0};
    ep.modal = true;
    nodal_to_modal_t<false>(c, T, bufA, bufG, lane, ep);
    return;
  }
  if (MODE == kFwd) {
    const double* Q = io.Qin + qoff;
    for (int w = lane; w < 5 * nM; w += blockDim.x) bufG[w] = Q[w];
    __syncthreads();
    element_forward<ANY>(c, T, s, bufA, bufG, lane);
    return;
  }
  if (MODE == kTraces) {
    // the stage's face traces rebuilt from its kept nodal state (and the
    // gradient traces from its kept nodal gradient) by the same trace
    // writes as the forward phases: bitwise the values they wrote
    const double* Un = c.Unod + c.slot_hoff[s];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = Un[w];
    __syncthreads();
    write_traces(c, T, s, bufA, c.T, 1.0, lane);
    if (c.ns) {
      for (int d = 0; d < 3; ++d) {
        const double* dW = c.DW + 3 * c.slot_hoff[s] + d * 5 * nQ;
        __syncthreads();
        for (int w = lane; w < 5 * nQ; w += blockDim.x) bufG[w] = dW[w];
        __syncthreads();
        write_traces(c, T, s, bufG, c.Vt, 1.0, lane, 3, (int64_t)d * 5 * T.n * T.n);
      }
    }
    __syncthreads();
    return;
  }
  if (MODE == kEval) {
    const double* Q = io.Qin + qoff;
    for (int w = lane; w < 5 * nM; w += blockDim.x) bufG[w] = Q[w];
    __syncthreads();
    modal_to_nodal(c, T, bufG, bufA, bufG, lane);
    double* out = io.Qout + c.elem_voff[c.elem_of_slot[s]];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) out[w] = bufA[w];
    __syncthreads();
    return;
  }
  // Curved element: pointwise J (cpool block [9][nQ] metric, [nQ] J, [nQ] 1/J,
  // then for prism / pyramid the dense M_e^{-1}); the affine scale 1/J_e and
  // the diagonal M_ref^{-1} are replaced by diag(1/J_q) before V^T (hex) or by
  // M_e^{-1} after it (prism, pyramid).  Tetrahedra are always affine.
  const int64_t coff = ANY ? c.slot_coff[s] : -1;
  const double* cblk = coff >= 0 ? c.cpool + coff : nullptr;
  // moving mesh: the backward phase returns vol - surf itself (the rate of
  // the mass-weighted state; the mass matrix is solved separately)
  const bool moving = ANY && c.mpool != nullptr;
  const bool dense = cblk && T.type != HEX && (!moving || MODE == kLoad || MODE == kProject);
  if (MODE == kLoad) {
    // b = V^T W J q: pointwise J_q (curved) or the element's constant J
    const int64_t e = c.elem_of_slot[s];
    const double* vals = io.Qin + c.elem_voff[e];
    const double* W = c.dpool + T.W;
    if (cblk) {
      const double* Jq = cblk + 9 * nQ;
      for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = W[w % nQ] * Jq[w % nQ] * vals[w];
    } else {
      for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = W[w % nQ] * vals[w];
    }
    __syncthreads();
    Epilogue ep{Epilogue::kStore, false, cblk ? 1.0 : 1.0 / c.geo[s].invJ, io.Qout + qoff, nullptr, nullptr, nullptr,
                nullptr, 0.0, 0.0, 0.0};
    nodal_to_modal<false>(c, T, bufA, bufG, lane, ep);
    return;
  }
  if (MODE == kProject) {
    const int64_t e = c.elem_of_slot[s];
    const double* vals = io.Qin + c.elem_voff[e];
    const double* W = c.dpool + T.W;
    if (dense) {
      const double* Jq = cblk + 9 * nQ;
      for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = W[w % nQ] * Jq[w % nQ] * vals[w];
    } else {
      for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = W[w % nQ] * vals[w];
    }
    __syncthreads();
    Epilogue ep{Epilogue::kStore, true, 1.0, io.Qout + qoff, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
    if (dense) {
      ep.Md = cblk + 11 * nQ;
      ep.rbuf = bufG + 5 * nQ;
    }
    nodal_to_modal<ANY>(c, T, bufA, bufG, lane, ep);
    return;
  }
  element_lift<ANY>(c, T, s, bufA, bufG, lane, c.T, -1.0,
                    (cblk && T.type == HEX && !moving) ? cblk + 10 * nQ : nullptr);
  const double invJ = cblk ? 1.0 : c.geo[s].invJ;
  if (MODE == kBwdRhs) {
    Epilogue ep{Epilogue::kStore, !moving, invJ, io.Qout + qoff, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
    if (dense) {
      ep.Md = cblk + 11 * nQ;
      ep.rbuf = bufG + 5 * nQ;
    }
    nodal_to_modal<ANY>(c, T, bufA, bufG, lane, ep);
    return;
  }
  Epilogue ep{Epilogue::kRk, !moving, invJ, nullptr, io.Qin + qoff, io.Qout + qoff, io.K + qoff,
              MODE == kBwdRkFwd ? bufG : nullptr, io.a, io.b, io.dt};
  if (dense) {
    ep.Md = cblk + 11 * nQ;
    ep.rbuf = bufG + 5 * nQ;
  }
  const bool bad = __syncthreads_or(nodal_to_modal<ANY>(c, T, bufA, bufG, lane, ep));
  if (bad && lane == 0) atomicOr(c.status, 1u);
  if (MODE == kBwdRkFwd) element_forward<ANY>(c, T, s, bufA, bufG, lane);
}

// ------------------------------------------------------------------ adjoint element phases
//
// With r = V^T (H - sum_f E_f^T Fhat_f), R = diag(M_ref^-1 / J) r and
// H = sum_l D_l^T G_l(U), U = V Q, the cotangent Rbar maps back as
//   Ybar = V diag(M_ref^-1 / J) Rbar          (nodal, a modal->nodal pass)
//   seed_f = -E_f Ybar                         (cotangent of Fhat_f, own side)
//   Gbar_l = D_l Ybar,  Ubar = sum_l (dG_l/dU)^T Gbar_l
// and, after the face phase turned the seeds into trace cotangents Tbar_f,
//   Qbar = V^T (Ubar + sum_f E_f^T Tbar_f).
// smem per block: bufA [5 nQmax], bufG [15 nQmax], bufC [5 nQmax].

// Phase A.  rk == 0: Rbar given.  rk == 1 (one reverse LSERK stage):
// Kbar <- Kbar + b Qbar is the Rbar of this stage and Kbar <- a (Kbar + b Qbar)
// is written back.
template <bool CURVED>
__device__ __noinline__ void element_vjp_a_t(const Ctx& c, const VjpArgs& va, int64_t s, double* bufA, double* bufG,
                                             double* bufC, int lane) {
  const TypeTab& T = c.tabs[c.slot_tab[s]];
  // curved element: pointwise metric, 1/J_q (hex) or the dense M_e^{-1}
  // (prism, pyramid) in place of the affine 1/J and diagonal M_ref^{-1}
  const double* cblk = CURVED ? c.cpool + c.slot_coff[s] : nullptr;
  const bool dense = CURVED && T.type != HEX;
  const int n = T.n, nM = T.nM, nQ = T.nQ, n2 = n * n;
  const double* dp = c.dpool;
  const int64_t qoff = c.slot_qoff[s];
  const int nQm = c.nQmax;
  // forward nodal state and its traces (read by the face phase): kept by the
  // forward pass, or recomputed from Q
  if (va.stored) {
    const double* Un = c.Unod + c.slot_hoff[s];
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufA[w] = Un[w];
    __syncthreads();
  } else {
    for (int w = lane; w < 5 * nM; w += blockDim.x) bufC[w] = va.Q[qoff + w];
    __syncthreads();
    modal_to_nodal(c, T, bufC, bufA, bufG, lane);
    write_traces(c, T, s, bufA, c.T, 1.0, lane);
  }
  // scaled cotangent of the modal residual, rbar = M_e^{-1} Rbar (M_e symmetric)
  const double invJ = CURVED ? 1.0 : c.geo[s].invJ;
  double* rdst = dense ? bufC : bufG;   // bufC is free here (Q consumed above)
  for (int w = lane; w < 5 * nM; w += blockDim.x) {
    const int m = w % nM;
    double rb;
    if (va.rk) {
      rb = va.Kbar[qoff + w] + va.b * va.Qbar[qoff + w];
      va.Kbar[qoff + w] = va.a * rb;
    } else {
      rb = va.Rbar[qoff + w];
    }
    rdst[w] = dense ? rb : rb * dp[T.minv + m] * invJ;
  }
  __syncthreads();
  if (dense) {
    const double* Md = cblk + 11 * nQ;
    for (int m = lane; m < nM; m += blockDim.x) {
      double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int j = 0; j < nM; ++j) DG_FMA5(Md[(size_t)j * nM + m], bufC + j, nM, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[v * nM + m] = acc[v];
    }
    __syncthreads();
  }
  modal_to_nodal(c, T, bufG, bufC, bufG + 5 * nQm, lane);  // Ybar in bufC
  if (CURVED && !dense) {
    // curved hexahedron: the forward's diag(1/J_q) before V^T, transposed
    const double* iJ = cblk + 10 * nQ;
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufC[w] *= iJ[w % nQ];
    __syncthreads();
  }
  write_traces(c, T, s, bufC, c.Tv, -1.0, lane);           // seeds
  // Gbar_l = D_l Ybar (collocation derivative), D[i][i'] = Dt[i'][i]
  {
    const double* Dt = dp + T.Dt;
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + i], bufC + m * n2 + jk, nQ, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[v * nQ + o] = acc[v];
      double acc1[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + j], bufC + i * n2 + m * n + k, nQ, acc1);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[(5 + v) * nQ + o] = acc1[v];
      double acc2[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + k], bufC + i * n2 + j * n + m, nQ, acc2);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[(10 + v) * nQ + o] = acc2[v];
    }
  }
  __syncthreads();
  // pointwise transpose of the contravariant flux
  {
    const ElemGeo& g = c.geo[s];
    double Jg[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Jg[k] = g.Jg[k];
    double* Hb = c.H + c.slot_hoff[s];
    for (int q = lane; q < nQ; q += blockDim.x) {
      double U[5], Gb[3][5], Ub[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = bufA[v * nQ + q];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int v = 0; v < 5; ++v) Gb[l][v] = bufG[(l * 5 + v) * nQ + q];
      double M[3][3];
      if (CURVED) {
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
          for (int d = 0; d < 3; ++d) M[l][d] = cblk[(l * 3 + d) * nQ + q];
      } else {
        point_metric(T.type, dp + T.wA + q * 9, Jg, M);
      }
      contravariant_vjp(U, M, c.gamma, Gb, Ub);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hb[v * nQ + q] = Ub[v];
    }
  }
  __syncthreads();
}

template <bool ANY>
__device__ __forceinline__ void element_vjp_a(const Ctx& c, const VjpArgs& va, int64_t s, double* bufA, double* bufG,
                                              double* bufC, int lane) {
  if (ANY && c.slot_coff[s] >= 0) element_vjp_a_t<true>(c, va, s, bufA, bufG, bufC, lane);
  else element_vjp_a_t<false>(c, va, s, bufA, bufG, bufC, lane);
}

// Phase C: Qbar = V^T (Ubar + sum_f E_f^T Tbar_f); stored (rk == 0) or added
// with weight dt (rk == 1).
__device__ __noinline__ void element_vjp_c(const Ctx& c, const VjpArgs& va, int64_t s, double* bufA, double* bufG,
                                           int lane) {
  const TypeTab& T = c.tabs[c.slot_tab[s]];
  element_lift<false>(c, T, s, bufA, bufG, lane, c.Tv, 1.0);
  Epilogue ep{va.rk ? Epilogue::kAxpy : Epilogue::kStore, false, va.rk ? va.dt : 1.0, va.Qbar + c.slot_qoff[s],
              nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
  nodal_to_modal<false>(c, T, bufA, bufG, lane, ep);
}

// ------------------------------------------------------------------ Navier-Stokes adjoint element phases
//
// The forward state at Q is recomputed first (traces T, nodal state Unod,
// lifting values, gradient traces Vt and the nodal gradient DW).  Then:
//   A: Ybar = V diag(M_ref^-1 / J) Rbar, seeds -E_f Ybar (Tv), Fbar_l = D_l Ybar;
//      per point the transposed total flux F_e(U) - F_v(U, DW): Ubar -> H,
//      gradient cotangent -> DW (in place);
//   face flux adjoint: trace cotangents (Tv) and gradient-trace cotangents (Vtb);
//   B: DWbar_d = DW + sum_f E_f^T Vtb_f,d; Bbar_d = V (-1/J) M_ref^-1 V^T DWbar_d;
//      Lbar_f = -sum_d n_d(f) E_f Bbar_d (own side of L);
//      Wbar = sum_d sum_l M[l][d] D_l Bbar_d, Ubar += (dW/dU)^T Wbar (H);
//   lifting-value adjoint: trace cotangents += (dW/dU)^T of the face means (Tv);
//   C (shared with Euler): Qbar = V^T (Ubar + sum_f E_f^T Tbar_f).

// bufA += sum_f coef_f E_f^T faces_f, face values at (ft_mult ft[lf] + ft_add)
// (staged through bufS).
__device__ __noinline__ void lift_add(const Ctx& c, const TypeTab& T, int64_t s, double* bufA, double* bufS, int lane,
                                      const double* faces, int ft_mult, int64_t ft_add, const double* coef) {
  const int n = T.n, nQ = T.nQ, n2 = n * n, nf = T.nfaces;
  const double* dp = c.dpool;
  const int64_t* ft = c.slot_ftoff + s * 6;
  {
    const int per = 5 * n2;
    for (int w = lane; w < nf * per; w += blockDim.x) {
      int lf = w / per, r = w - lf * per;
      bufS[w] = faces[ft_mult * ft[lf] + ft_add + r];
    }
  }
  __syncthreads();
  for (int o = lane; o < nQ; o += blockDim.x) {
    int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
    double h[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) h[v] = bufA[v * nQ + o];
    for (int lf = 0; lf < nf; ++lf) {
      const FaceDesc fd = T.faces[lf];
      int m = sel3(i, j, k, fd.fixed);
      int p = sel3(i, j, k, fd.alpha) + n * sel3(i, j, k, fd.beta);
      DG_FMA5(coef[lf] * dp[T.ext + fd.end * n + m], bufS + lf * 5 * n2 + p, n2, h);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) bufA[v * nQ + o] = h[v];
  }
  __syncthreads();
}

// Phase A (Navier-Stokes).  smem: bufY [5 nQ] | bufG [15 nQ] | bufS [5 nQ].
template <bool CURVED>
__device__ __noinline__ void element_vjp_a_ns_t(const Ctx& c, const VjpArgs& va, int64_t s, double* smem, int lane) {
  const TypeTab& T = c.tabs[c.slot_tab[s]];
  const int n = T.n, nM = T.nM, nQ = T.nQ, n2 = n * n;
  const int nQm = c.nQmax;
  double* bufY = smem;
  double* bufG = smem + 5 * nQm;
  double* bufS = smem + 20 * nQm;
  const double* dp = c.dpool;
  const int64_t qoff = c.slot_qoff[s];
  // curved element: dense M_e^{-1} (prism, pyramid) or 1/J_q (hex), pointwise metric
  const double* cblk = CURVED ? c.cpool + c.slot_coff[s] : nullptr;
  const bool dense = CURVED && T.type != HEX;
  const double invJ = CURVED ? 1.0 : c.geo[s].invJ;
  double* rdst = dense ? bufY : bufS;   // bufY is free until the modal -> nodal pass
  for (int w = lane; w < 5 * nM; w += blockDim.x) {
    const int m = w % nM;
    double rb;
    if (va.rk) {
      rb = va.Kbar[qoff + w] + va.b * va.Qbar[qoff + w];
      va.Kbar[qoff + w] = va.a * rb;
    } else {
      rb = va.Rbar[qoff + w];
    }
    rdst[w] = dense ? rb : rb * dp[T.minv + m] * invJ;
  }
  __syncthreads();
  if (dense) {
    const double* Md = cblk + 11 * nQ;
    for (int m = lane; m < nM; m += blockDim.x) {
      double acc[5] = {0, 0, 0, 0, 0};
#pragma unroll 4
      for (int j = 0; j < nM; ++j) DG_FMA5(Md[(size_t)j * nM + m], bufY + j, nM, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufS[v * nM + m] = acc[v];
    }
    __syncthreads();
  }
  modal_to_nodal(c, T, bufS, bufY, bufG, lane);
  if (CURVED && !dense) {
    const double* iJ = cblk + 10 * nQ;
    for (int w = lane; w < 5 * nQ; w += blockDim.x) bufY[w] *= iJ[w % nQ];
    __syncthreads();
  }
  write_traces(c, T, s, bufY, c.Tv, -1.0, lane);
  {
    const double* Dt = dp + T.Dt;
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + i], bufY + m * n2 + jk, nQ, acc);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[v * nQ + o] = acc[v];
      double acc1[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + j], bufY + i * n2 + m * n + k, nQ, acc1);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[(5 + v) * nQ + o] = acc1[v];
      double acc2[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + k], bufY + i * n2 + j * n + m, nQ, acc2);
#pragma unroll
      for (int v = 0; v < 5; ++v) bufG[(10 + v) * nQ + o] = acc2[v];
    }
  }
  __syncthreads();
  {
    const ElemGeo& g = c.geo[s];
    double Jg[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Jg[k] = g.Jg[k];
    const double gm1 = c.gamma - 1.0;
    const double* Un = c.Unod + c.slot_hoff[s];
    double* DWs = c.DW + 3 * c.slot_hoff[s];
    double* Hb = c.H + c.slot_hoff[s];
    for (int q = lane; q < nQ; q += blockDim.x) {
      double U[5], W[5], gr[15], Gb[3][5], Ub[5], Wb[5] = {0, 0, 0, 0, 0}, gb[15];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = Un[v * nQ + q];
#pragma unroll
      for (int t = 0; t < 15; ++t) {
        gr[t] = DWs[t * nQ + q];
        gb[t] = 0.0;
      }
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int v = 0; v < 5; ++v) Gb[l][v] = bufG[(l * 5 + v) * nQ + q];
      double M[3][3];
      if (CURVED) {
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
          for (int d = 0; d < 3; ++d) M[l][d] = cblk[(l * 3 + d) * nQ + q];
      } else {
        point_metric(T.type, dp + T.wA + q * 9, Jg, M);
      }
      contravariant_vjp(U, M, c.gamma, Gb, Ub);
      // G_l -= sum_d M[l][d] F_v[d]  =>  Fvbar[d] = -sum_l M[l][d] Gbar_l
      double Fvb[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) Fvb[d][v] = -(M[0][d] * Gb[0][v] + M[1][d] * Gb[1][v] + M[2][d] * Gb[2][v]);
      primitive(U, gm1, W);
      viscous_flux_vjp(W, gr, c.mu, c.kappa, Fvb, Wb, gb);
      primitive_vjp(U, gm1, Wb, Ub);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hb[v * nQ + q] = Ub[v];
#pragma unroll
      for (int t = 0; t < 15; ++t) DWs[t * nQ + q] = gb[t];
    }
  }
  __syncthreads();
}

// Phase B (Navier-Stokes lifting transpose).
// smem: bufD [15 nQ] | bufB [5 nQ] | bufX [5 nQ] | bufW [5 nQ] | bufL [15 nQ].
template <bool CURVED>
__device__ __noinline__ void element_vjp_b_ns_t(const Ctx& c, int64_t s, double* smem, int lane) {
  const TypeTab& T = c.tabs[c.slot_tab[s]];
  const double* cblk = CURVED ? c.cpool + c.slot_coff[s] : nullptr;
  const int n = T.n, nQ = T.nQ, n2 = n * n, nf = T.nfaces;
  const int nQm = c.nQmax;
  double* bufD = smem;                 // smem + 15 nQm .. 20 nQm is unused
  double* bufX = smem + 20 * nQm;
  double* bufW = smem + 25 * nQm;
  double* bufL = smem + 30 * nQm;
  const double* dp = c.dpool;
  const double* Dt = dp + T.Dt;
  const int64_t* ft = c.slot_ftoff + s * 6;
  const ElemGeo& g = c.geo[s];
  {
    const double* DWs = c.DW + 3 * c.slot_hoff[s];
    for (int w = lane; w < 15 * nQ; w += blockDim.x) bufD[w] = DWs[w];
  }
  __syncthreads();
  const double ones[6] = {1.0, 1.0, 1.0, 1.0, 1.0, 1.0};
  for (int d = 0; d < 3; ++d) lift_add(c, T, s, bufD + d * 5 * nQ, bufL, lane, c.Vtb, 3, (int64_t)d * 5 * n2, ones);
  for (int w = lane; w < 5 * nQ; w += blockDim.x) bufW[w] = 0.0;
  for (int w = lane; w < nf * 5 * n2; w += blockDim.x) bufL[w] = 0.0;
  __syncthreads();
  double Jg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Jg[k] = g.Jg[k];
  for (int d = 0; d < 3; ++d) {
    double* Bd = bufD + d * 5 * nQ;     // DWbar_d, replaced by Bbar_d
    if (T.type == HEX) {
      // V M^{-1} V^T = (W J)^{-1} (square V): pointwise
      const double* wq = dp + T.W;
      if (CURVED) {
        const double* iJ = cblk + 10 * nQ;
        for (int w = lane; w < 5 * nQ; w += blockDim.x) Bd[w] = -iJ[w % nQ] * Bd[w] / wq[w % nQ];
      } else {
        for (int w = lane; w < 5 * nQ; w += blockDim.x) Bd[w] = -g.invJ * Bd[w] / wq[w % nQ];
      }
      __syncthreads();
    } else {
      Epilogue ep{Epilogue::kStore, true, CURVED ? -1.0 : -g.invJ, bufX, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
      if (CURVED) {
        ep.Md = cblk + 11 * nQ;        // symmetric: its own transpose
        ep.rbuf = smem + 15 * nQm;
      }
      nodal_to_modal<CURVED>(c, T, Bd, bufX, lane, ep);
      modal_to_nodal(c, T, bufX, Bd, bufX, lane);
    }
    // Lbar_f -= n_d(f) E_f Bbar_d on the own face points
    for (int w = lane; w < nf * n2; w += blockDim.x) {
      int lf = w / n2, p = w - lf * n2;
      int ia = p % n, ib = p / n;
      const FaceDesc fd = T.faces[lf];
      int sa = fd.alpha == 0 ? n2 : (fd.alpha == 1 ? n : 1);
      int sb = fd.beta == 0 ? n2 : (fd.beta == 1 ? n : 1);
      int sf = fd.fixed == 0 ? n2 : (fd.fixed == 1 ? n : 1);
      const double* e = dp + T.ext + fd.end * n;
      const double* Bs = Bd + ia * sa + ib * sb;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int m = 0; m < n; ++m) DG_FMA5(e[m], Bs + m * sf, nQ, acc);
      const double nd = CURVED ? c.snrm[3 * (ft[lf] / 5) + d * n2 + p] : c.fnrm[(s * 6 + lf) * 3 + d];
#pragma unroll
      for (int v = 0; v < 5; ++v) bufL[(lf * 5 + v) * n2 + p] -= nd * acc[v];
    }
    __syncthreads();
  }
  // Wbar = sum_d sum_l M[l][d] D_l Bbar_d = sum_k sum_{l: wA[l][k] != 0} wA[l][k] D_l C_k
  // with C_k = sum_d Jg[k][d] Bbar_d (in place of the Bbar_d); a curved
  // element takes the first form with its pointwise metric
  if (CURVED) {
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      double wb[5] = {0, 0, 0, 0, 0};
      for (int d = 0; d < 3; ++d) {
        const double* B = bufD + d * 5 * nQ;
        double a0[5] = {0, 0, 0, 0, 0}, a1[5] = {0, 0, 0, 0, 0}, a2[5] = {0, 0, 0, 0, 0};
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + i], B + m * n2 + jk, nQ, a0);
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + j], B + i * n2 + m * n + k, nQ, a1);
        for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + k], B + i * n2 + j * n + m, nQ, a2);
        const double m0 = cblk[(0 * 3 + d) * nQ + o], m1 = cblk[(1 * 3 + d) * nQ + o], m2 = cblk[(2 * 3 + d) * nQ + o];
#pragma unroll
        for (int v = 0; v < 5; ++v) wb[v] += m0 * a0[v] + m1 * a1[v] + m2 * a2[v];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) bufW[v * nQ + o] = wb[v];
    }
    __syncthreads();
  }
  for (int w = lane; w < (CURVED ? 0 : 5 * nQ); w += blockDim.x) {
    const double b0 = bufD[w], b1 = bufD[5 * nQ + w], b2 = bufD[10 * nQ + w];
#pragma unroll
    for (int kr = 0; kr < 3; ++kr)
      bufD[kr * 5 * nQ + w] = Jg[kr * 3] * b0 + Jg[kr * 3 + 1] * b1 + Jg[kr * 3 + 2] * b2;
  }
  __syncthreads();
  if (!CURVED) {
    const unsigned nz = kMetricMask[T.type];
    for (int o = lane; o < nQ; o += blockDim.x) {
      int i = o / n2, jk = o - i * n2, j = jk / n, k = jk - j * n;
      const double* wa = dp + T.wA + o * 9;
      double wb[5] = {0, 0, 0, 0, 0};
      for (int kr = 0; kr < 3; ++kr) {
        const double* C = bufD + kr * 5 * nQ;
        if ((nz >> kr) & 1u) {
          double a[5] = {0, 0, 0, 0, 0};
          for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + i], C + m * n2 + jk, nQ, a);
#pragma unroll
          for (int v = 0; v < 5; ++v) wb[v] = fma(wa[kr], a[v], wb[v]);
        }
        if ((nz >> (3 + kr)) & 1u) {
          double a[5] = {0, 0, 0, 0, 0};
          for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + j], C + i * n2 + m * n + k, nQ, a);
#pragma unroll
          for (int v = 0; v < 5; ++v) wb[v] = fma(wa[3 + kr], a[v], wb[v]);
        }
        if ((nz >> (6 + kr)) & 1u) {
          double a[5] = {0, 0, 0, 0, 0};
          for (int m = 0; m < n; ++m) DG_FMA5(Dt[m * n + k], C + i * n2 + j * n + m, nQ, a);
#pragma unroll
          for (int v = 0; v < 5; ++v) wb[v] = fma(wa[6 + kr], a[v], wb[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) bufW[v * nQ + o] = wb[v];
    }
  }
  __syncthreads();
  {
    const double gm1 = c.gamma - 1.0;
    const double* Un = c.Unod + c.slot_hoff[s];
    double* Hb = c.H + c.slot_hoff[s];
    for (int q = lane; q < nQ; q += blockDim.x) {
      double U[5], Wb[5], Ub[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        U[v] = Un[v * nQ + q];
        Wb[v] = bufW[v * nQ + q];
      }
      primitive_vjp(U, gm1, Wb, Ub);
#pragma unroll
      for (int v = 0; v < 5; ++v) Hb[v * nQ + q] += Ub[v];
    }
    for (int w = lane; w < nf * 5 * n2; w += blockDim.x) {
      int lf = w / (5 * n2), r = w - lf * 5 * n2;
      c.L[ft[lf] + r] = bufL[w];
    }
  }
  __syncthreads();
}

template <bool ANY>
__device__ __forceinline__ void element_vjp_a_ns(const Ctx& c, const VjpArgs& va, int64_t s, double* smem, int lane) {
  if (ANY && c.slot_coff[s] >= 0) element_vjp_a_ns_t<true>(c, va, s, smem, lane);
  else element_vjp_a_ns_t<false>(c, va, s, smem, lane);
}

template <bool ANY>
__device__ __forceinline__ void element_vjp_b_ns(const Ctx& c, int64_t s, double* smem, int lane) {
  if (ANY && c.slot_coff[s] >= 0) element_vjp_b_ns_t<true>(c, s, smem, lane);
  else element_vjp_b_ns_t<false>(c, s, smem, lane);
}

// ------------------------------------------------------------------ kernels
//
// One block (1 to 4 warps) works on one element at a time; its threads share
// the element's shared-memory workspace bufA [5 nQmax] + bufG [15 nQmax].

// The launch's stage arguments with the state, register and time step taken
// from the device parameter block when the launch has one.
__device__ __forceinline__ StageArgs resolve_args(const StageArgs& a) {
  StageArgs r = a;
  if (a.dyn) {
    const RkDyn d = *a.dyn;
    r.Qin = d.Q;
    r.Qout = d.Q;
    r.K = d.K;
    r.dt = d.dt;
  }
  return r;
}

template <int MODE, bool ANY>
__global__ void __launch_bounds__(128) elem_naive_kernel(Ctx c, StageArgs io0, const int64_t* __restrict__ list,
                                                         int64_t count) {
  extern __shared__ double smem[];
  const int64_t idx = blockIdx.x;
  if (idx >= count) return;
  const StageArgs io = resolve_args(io0);
  double* bufA = smem;
  double* bufG = bufA + 5 * c.nQmax;
  process_element<MODE, ANY>(c, io, list ? list[idx] : idx, bufA, bufG, threadIdx.x);
}

template <int MODE, bool ANY>
__global__ void __launch_bounds__(128) elem_balanced_kernel(Ctx c, StageArgs io0, const int64_t* __restrict__ list,
                                                            const int64_t* __restrict__ chunk_start, int64_t nchunks,
                                                            unsigned int* counter, unsigned int* next_counter) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_chunk;
  const StageArgs io = resolve_args(io0);
  // The previous launch on this stream used next_counter and has finished.
  if (blockIdx.x == 0 && threadIdx.x == 0 && next_counter) *next_counter = 0u;
  const int lane = threadIdx.x;
  double* bufA = smem;
  double* bufG = bufA + 5 * c.nQmax;
  // Cost probe: time per element, summed per (type, N) table in shared bins
  // (thread 0 alone touches them) and flushed once at the end.
  __shared__ unsigned long long s_cost[2 * kMaxTabs];
  for (int t = lane; t < 2 * kMaxTabs; t += blockDim.x) s_cost[t] = 0ull;
  unsigned long long busy = 0;
  while (true) {
    if (lane == 0) s_chunk = atomicAdd(counter, 1u);
    __syncthreads();
    const unsigned int ch = s_chunk;
    __syncthreads();
    if (ch >= nchunks) break;
    for (int64_t i = chunk_start[ch]; i < chunk_start[ch + 1]; ++i) {
      const int64_t s = list ? list[i] : i;
      uint64_t t0 = global_ns();
      process_element<MODE, ANY>(c, io, s, bufA, bufG, lane);
      __syncthreads();
      uint64_t dtn = global_ns() - t0;
      if (lane == 0) {
        const int tab = c.slot_tab[s];
        s_cost[2 * tab] += dtn;
        s_cost[2 * tab + 1] += 1ull;
      }
      busy += dtn;
    }
  }
  if (lane == 0 && c.cost) {
    for (int t = 0; t < kMaxTabs; ++t)
      if (s_cost[2 * t + 1]) {
        atomicAdd(c.cost + 2 * t, s_cost[2 * t]);
        atomicAdd(c.cost + 2 * t + 1, s_cost[2 * t + 1]);
      }
    if (busy) atomicAdd(c.sm_ns + smid(), busy);
  }
}

template <bool CURVED>
__global__ void face_kernel(Ctx c) {
  extern __shared__ double sF[];
  const FaceBlock fb = c.fblocks[blockIdx.x];
  const int n = fb.n, n2 = n * n, items = fb.count * n2;
  const double gamma = c.gamma;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, p = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    const double* T0 = c.T + R.toff;
    const double* T1 = T0 + 5 * n2;
    double UL[5], UR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) UL[v] = T0[v * n2 + p];
    if (R.map >= 0) {
      int j = c.perms[(size_t)R.map + p];
#pragma unroll
      for (int v = 0; v < 5; ++v) UR[v] = T1[v * n2 + j];
    } else {
      const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int j = 0; j < n2; ++j) acc = fma(D[j], T1[v * n2 + j], acc);
        UR[v] = acc;
      }
    }
    double nrm[3] = {R.nrm[0], R.nrm[1], R.nrm[2]};
    const bool cg = CURVED && R.cgeo >= 0;
    if (cg) {
      // curved owner: the normal at this point
      const double* G = c.fgeo + R.cgeo;
      nrm[0] = G[p];
      nrm[1] = G[n2 + p];
      nrm[2] = G[2 * n2 + p];
    }
    const double wS = cg ? c.fgeo[R.cgeo + 3 * n2 + p] : c.dpool[c.tabs[R.owner_tab].fw + R.owner_lf * n2 + p] * R.S;
    double Fs[5];
    if (CURVED && c.fmot && cg) {
      // moving mesh (LF only): the normal mesh speed at the owner's point
      const double* xf = c.fmot + 3 * (int64_t)R.cgeo + 9 * n2 + p;
      const double sn = nrm[0] * xf[0] + nrm[1] * xf[n2] + nrm[2] * xf[2 * n2];
      flux_lf_moving_scaled(UL, UR, nrm, wS, sn, gamma, Fs);
    } else if (c.flux == 0) {
      flux_lf_scaled(UL, UR, nrm, wS, gamma, Fs);   // wS F*
    } else if (c.flux == 2) {
      // entropy-conservative: Chandrashekar's F# contracted with wS n
      double PL[kTP], PR[kTP];
      two_point_state(UL, gamma - 1.0, PL);
      two_point_state(UR, gamma - 1.0, PR);
      const double m[3] = {wS * nrm[0], wS * nrm[1], wS * nrm[2]};
      two_point_flux(PL, 1, PR, 1, m, 1.0 / (gamma - 1.0), Fs);
    } else {
      flux_roe(UL, UR, nrm, gamma, Fs);
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v] *= wS;
    }
    if (R.map >= 0) {
      // permutation map: this thread alone read T0[p] and T1[perm[p]], so it
      // writes both results in place at once
      const int j = c.perms[(size_t)R.map + p];
      double* W0 = c.T + R.toff;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        W0[v * n2 + p] = Fs[v];
        W0[(5 + v) * n2 + j] = -Fs[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[(fl * 5 + v) * n2 + p] = Fs[v];
    }
  }
  __syncthreads();
  // interpolating maps: the neighbour's share needs every owner point first
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, q = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    if (R.map >= 0) continue;
    double* T0 = c.T + R.toff;
    double* T1 = T0 + 5 * n2;
    const double* F = sF + fl * 5 * n2;
#pragma unroll
    for (int v = 0; v < 5; ++v) T0[v * n2 + q] = F[v * n2 + q];
    {
      const double* D = c.dense + (size_t)(-1 - R.map) + q;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int p = 0; p < n2; ++p) acc = fma(D[(size_t)p * n2], F[v * n2 + p], acc);
        T1[v * n2 + q] = -acc;
      }
    }
  }
}

// Navier-Stokes face phases.  KIND 0 (BR1 lifting): per owner point p,
// W* = (W(U-) + W(U+))/2 with U+ the neighbour trace mapped to the owner's
// points, and L = w S W* (owner side) / Map^T (w S W*) (neighbour side); the
// element multiplies by its own outward normal.  KIND 1 (flux): the inviscid
// Riemann flux minus the central viscous flux (F_v(U-, g-) + F_v(U+, g+)).n/2,
// g the lifted gradient traces, times w S, written over the traces as in the
// Euler face kernel.
template <int KIND, bool CURVED>
__global__ void face_ns_kernel(Ctx c) {
  extern __shared__ double sF[];
  const FaceBlock fb = c.fblocks[blockIdx.x];
  const int n = fb.n, n2 = n * n, items = fb.count * n2;
  const double gamma = c.gamma, gm1 = gamma - 1.0;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, p = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    const double* T0 = c.T + R.toff;
    const double* T1 = T0 + 5 * n2;
    double UL[5], UR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) UL[v] = T0[v * n2 + p];
    if (R.map >= 0) {
      int j = c.perms[(size_t)R.map + p];
#pragma unroll
      for (int v = 0; v < 5; ++v) UR[v] = T1[v * n2 + j];
    } else {
      const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int j = 0; j < n2; ++j) acc = fma(D[j], T1[v * n2 + j], acc);
        UR[v] = acc;
      }
    }
    const bool cg = CURVED && R.cgeo >= 0;   // curved owner: per-point normal and w S
    const double wS = cg ? c.fgeo[R.cgeo + 3 * n2 + p] : c.dpool[c.tabs[R.owner_tab].fw + R.owner_lf * n2 + p] * R.S;
    double Fs[5];
    if (KIND == 0) {
      double WL[5], WR[5];
      primitive(UL, gm1, WL);
      primitive(UR, gm1, WR);
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (WL[v] + WR[v]);
    } else {
      double nrm[3] = {R.nrm[0], R.nrm[1], R.nrm[2]};
      if (cg) {
        nrm[0] = c.fgeo[R.cgeo + p];
        nrm[1] = c.fgeo[R.cgeo + n2 + p];
        nrm[2] = c.fgeo[R.cgeo + 2 * n2 + p];
      }
      if (CURVED && c.fmot && cg) {
        // moving mesh: the LF flux in the frame of the normal mesh speed
        const double* xf = c.fmot + 3 * (int64_t)R.cgeo + 9 * n2 + p;
        const double sn = nrm[0] * xf[0] + nrm[1] * xf[n2] + nrm[2] * xf[2 * n2];
        flux_lf_moving_scaled(UL, UR, nrm, 1.0, sn, gamma, Fs);
      } else if (c.flux == 0) {
        flux_lf(UL, UR, nrm, gamma, Fs);
      } else {
        flux_roe(UL, UR, nrm, gamma, Fs);
      }
      const double* V0 = c.Vt + 3 * R.toff;
      const double* V1 = V0 + 15 * n2;
      double g[15], W[5], Fv[3][5];
#pragma unroll
      for (int t = 0; t < 15; ++t) g[t] = V0[t * n2 + p];
      primitive(UL, gm1, W);
      viscous_flux(W, g, c.mu, c.kappa, Fv);
      double Fvn[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) Fvn[v] = nrm[0] * Fv[0][v] + nrm[1] * Fv[1][v] + nrm[2] * Fv[2][v];
      if (R.map >= 0) {
        int j = c.perms[(size_t)R.map + p];
#pragma unroll
        for (int t = 0; t < 15; ++t) g[t] = V1[t * n2 + j];
      } else {
        const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
        for (int t = 0; t < 15; ++t) {
          double acc = 0.0;
          for (int j = 0; j < n2; ++j) acc = fma(D[j], V1[t * n2 + j], acc);
          g[t] = acc;
        }
      }
      primitive(UR, gm1, W);
      viscous_flux(W, g, c.mu, c.kappa, Fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Fvn[v] += nrm[0] * Fv[0][v] + nrm[1] * Fv[1][v] + nrm[2] * Fv[2][v];
        Fs[v] -= 0.5 * Fvn[v];
      }
    }
    if (R.map >= 0) {
      // permutation map: direct writes (this thread alone read the inputs at
      // p and perm[p]; the flux kind overwrites them in place)
      const int j = c.perms[(size_t)R.map + p];
      double* O0 = (KIND == 0 ? c.L : c.T) + R.toff;
      const double nb = KIND == 0 ? 1.0 : -1.0;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        O0[v * n2 + p] = wS * Fs[v];
        O0[(5 + v) * n2 + j] = nb * wS * Fs[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[(fl * 5 + v) * n2 + p] = wS * Fs[v];
    }
  }
  __syncthreads();
  double* out = KIND == 0 ? c.L : c.T;
  const double nb_sign = KIND == 0 ? 1.0 : -1.0;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, q = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    if (R.map >= 0) continue;
    double* O0 = out + R.toff;
    double* O1 = O0 + 5 * n2;
    const double* F = sF + fl * 5 * n2;
#pragma unroll
    for (int v = 0; v < 5; ++v) O0[v * n2 + q] = F[v * n2 + q];
    {
      const double* D = c.dense + (size_t)(-1 - R.map) + q;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int p = 0; p < n2; ++p) acc = fma(D[(size_t)p * n2], F[v * n2 + p], acc);
        O1[v * n2 + q] = nb_sign * acc;
      }
    }
  }
}

// ------------------------------------------------------------------ adjoint kernels

// One kernel per phase, so that each gets its own register allocation.
template <int PHASE, bool ANY>
__global__ void __launch_bounds__(128) elem_vjp_kernel(Ctx c, VjpArgs va) {
  extern __shared__ double smem[];
  const int64_t s = blockIdx.x;
  double* bufA = smem;
  double* bufG = bufA + 5 * c.nQmax;
  double* bufC = bufG + 15 * c.nQmax;
  if (PHASE == 0) element_vjp_a<ANY>(c, va, s, bufA, bufG, bufC, threadIdx.x);
  else if (PHASE == 10) element_vjp_a_ns<ANY>(c, va, s, smem, threadIdx.x);
  else if (PHASE == 11) element_vjp_b_ns<ANY>(c, s, smem, threadIdx.x);
  else element_vjp_c(c, va, s, bufA, bufG, threadIdx.x);
}

// Face phase of the adjoint.  Per owner face point p, with Map the
// neighbour -> owner point map of the forward face phase:
//   g(p) = wS_p (seed_own(p) - (Map seed_nb)(p))     (cotangent of F*)
//   (Tbar-, Tbar+) = (dF*/dU-, dF*/dU+)^T g
//   Tbar_own = Tbar-,  Tbar_nb = Map^T Tbar+        (written over the seeds)
template <bool CURVED>
__global__ void face_vjp_kernel(Ctx c) {
  extern __shared__ double sF[];
  const FaceBlock fb = c.fblocks[blockIdx.x];
  const int n = fb.n, n2 = n * n, items = fb.count * n2;
  double* sR = sF + 32 * 5 * n2;
  const double gamma = c.gamma;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, p = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    const double* T0 = c.T + R.toff;
    const double* T1 = T0 + 5 * n2;
    const double* S0 = c.Tv + R.toff;
    const double* S1 = S0 + 5 * n2;
    double UL[5], UR[5], g[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      UL[v] = T0[v * n2 + p];
      g[v] = S0[v * n2 + p];
    }
    if (R.map >= 0) {
      int j = c.perms[(size_t)R.map + p];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        UR[v] = T1[v * n2 + j];
        g[v] -= S1[v * n2 + j];
      }
    } else {
      const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < n2; ++j) {
          a = fma(D[j], T1[v * n2 + j], a);
          b = fma(D[j], S1[v * n2 + j], b);
        }
        UR[v] = a;
        g[v] -= b;
      }
    }
    const bool cg = CURVED && R.cgeo >= 0;
    const double wS = cg ? c.fgeo[R.cgeo + 3 * n2 + p]
                         : c.dpool[c.tabs[R.owner_tab].fw + R.owner_lf * n2 + p] * R.S;
#pragma unroll
    for (int v = 0; v < 5; ++v) g[v] *= wS;
    double nrm[3] = {R.nrm[0], R.nrm[1], R.nrm[2]};
    if (cg) {
      const double* G = c.fgeo + R.cgeo;
      nrm[0] = G[p];
      nrm[1] = G[n2 + p];
      nrm[2] = G[2 * n2 + p];
    }
    double UbL[5] = {0, 0, 0, 0, 0}, UbR[5] = {0, 0, 0, 0, 0};
    if (c.flux == 0) flux_lf_vjp(UL, UR, nrm, gamma, g, UbL, UbR);
    else flux_roe_vjp(UL, UR, nrm, gamma, g, UbL, UbR);
    if (R.map >= 0) {
      // permutation map: this thread alone read the seeds at p and perm[p]
      const int j = c.perms[(size_t)R.map + p];
      double* W0 = c.Tv + R.toff;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        W0[v * n2 + p] = UbL[v];
        W0[(5 + v) * n2 + j] = UbR[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sF[(fl * 5 + v) * n2 + p] = UbL[v];
        sR[(fl * 5 + v) * n2 + p] = UbR[v];
      }
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, q = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    if (R.map >= 0) continue;
    double* S0 = c.Tv + R.toff;
    double* S1 = S0 + 5 * n2;
    const double* Fl = sF + fl * 5 * n2;
    const double* Fr = sR + fl * 5 * n2;
#pragma unroll
    for (int v = 0; v < 5; ++v) S0[v * n2 + q] = Fl[v * n2 + q];
    {
      const double* D = c.dense + (size_t)(-1 - R.map) + q;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int p = 0; p < n2; ++p) acc = fma(D[(size_t)p * n2], Fr[v * n2 + p], acc);
        S1[v * n2 + q] = acc;
      }
    }
  }
}

// Navier-Stokes face adjoints.
// KIND 1 (flux): g = wS (seed_own - Map seed_nb) is the cotangent of the
//   unscaled flux F* = Riemann(U-, U+) - (F_v(U-, g-) + F_v(U+, g+)).n/2;
//   trace cotangents Tv (own side: Ubar-, neighbour: Map^T Ubar+) and
//   gradient-trace cotangents Vtb (likewise).  Faces with a permutation map
//   are finished by the thread that owns the point (it alone read the inputs
//   at p and perm[p]); on interpolating faces the neighbour's gradient
//   cotangent at the owner's points is parked in the owner half of Vt (read
//   only by the same thread) and the transposed map runs after a barrier.
// KIND 0 (lifting values): Wbar = wS (Lbar_own + Map Lbar_nb) / 2 for both
//   means' arguments; Tv += (dW/dU)^T Wbar (own), Map^T (neighbour).
// At most 7 warps (n <= 7) per block; two resident blocks at the largest n
// (three at n = 5) instead of the two that 168 registers allow.
template <int KIND, bool CURVED>
__global__ void __launch_bounds__(224, 2) face_ns_vjp_kernel(Ctx c) {
  extern __shared__ double sF[];
  const FaceBlock fb = c.fblocks[blockIdx.x];
  const int n = fb.n, n2 = n * n, items = fb.count * n2;
  double* sR = sF + 32 * 5 * n2;
  const double gamma = c.gamma, gm1 = gamma - 1.0;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, p = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    const double* T0 = c.T + R.toff;
    const double* T1 = T0 + 5 * n2;
    const double* S0 = (KIND == 1 ? c.Tv : c.L) + R.toff;
    const double* S1 = S0 + 5 * n2;
    double UL[5], UR[5], gs[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      UL[v] = T0[v * n2 + p];
      gs[v] = S0[v * n2 + p];
    }
    const double sgn = KIND == 1 ? -1.0 : 1.0;
    if (R.map >= 0) {
      int j = c.perms[(size_t)R.map + p];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        UR[v] = T1[v * n2 + j];
        gs[v] += sgn * S1[v * n2 + j];
      }
    } else {
      const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < n2; ++j) {
          a = fma(D[j], T1[v * n2 + j], a);
          b = fma(D[j], S1[v * n2 + j], b);
        }
        UR[v] = a;
        gs[v] += sgn * b;
      }
    }
    const bool cg = CURVED && R.cgeo >= 0;   // curved owner: per-point normal and w S
    const double wS = cg ? c.fgeo[R.cgeo + 3 * n2 + p] : c.dpool[c.tabs[R.owner_tab].fw + R.owner_lf * n2 + p] * R.S;
    double UbL[5] = {0, 0, 0, 0, 0}, UbR[5] = {0, 0, 0, 0, 0};
    if (KIND == 0) {
      double Wb[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) Wb[v] = 0.5 * wS * gs[v];
      primitive_vjp(UL, gm1, Wb, UbL);
      primitive_vjp(UR, gm1, Wb, UbR);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) gs[v] *= wS;
      double nrm[3] = {R.nrm[0], R.nrm[1], R.nrm[2]};
      if (cg) {
        nrm[0] = c.fgeo[R.cgeo + p];
        nrm[1] = c.fgeo[R.cgeo + n2 + p];
        nrm[2] = c.fgeo[R.cgeo + 2 * n2 + p];
      }
      if (c.flux == 0) flux_lf_vjp(UL, UR, nrm, gamma, gs, UbL, UbR);
      else flux_roe_vjp(UL, UR, nrm, gamma, gs, UbL, UbR);
      double Fvb[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) Fvb[d][v] = -0.5 * nrm[d] * gs[v];
      double* V0 = c.Vt + 3 * R.toff;
      const double* V1 = V0 + 15 * n2;
      double gr[15], gb[15], W[5], Wb[5];
      // owner side
#pragma unroll
      for (int t = 0; t < 15; ++t) {
        gr[t] = V0[t * n2 + p];
        gb[t] = 0.0;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) Wb[v] = 0.0;
      primitive(UL, gm1, W);
      viscous_flux_vjp(W, gr, c.mu, c.kappa, Fvb, Wb, gb);
      primitive_vjp(UL, gm1, Wb, UbL);
      double* B0 = c.Vtb + 3 * R.toff;
#pragma unroll
      for (int t = 0; t < 15; ++t) B0[t * n2 + p] = gb[t];
      // neighbour side at the owner's points
      if (R.map >= 0) {
        int j = c.perms[(size_t)R.map + p];
#pragma unroll
        for (int t = 0; t < 15; ++t) gr[t] = V1[t * n2 + j];
      } else {
        const double* D = c.dense + (size_t)(-1 - R.map) + (size_t)p * n2;
#pragma unroll
        for (int t = 0; t < 15; ++t) {
          double acc = 0.0;
          for (int j = 0; j < n2; ++j) acc = fma(D[j], V1[t * n2 + j], acc);
          gr[t] = acc;
        }
      }
#pragma unroll
      for (int t = 0; t < 15; ++t) gb[t] = 0.0;
#pragma unroll
      for (int v = 0; v < 5; ++v) Wb[v] = 0.0;
      primitive(UR, gm1, W);
      viscous_flux_vjp(W, gr, c.mu, c.kappa, Fvb, Wb, gb);
      primitive_vjp(UR, gm1, Wb, UbR);
      if (R.map >= 0) {
        const int j = c.perms[(size_t)R.map + p];
        double* B1 = B0 + 15 * n2;
#pragma unroll
        for (int t = 0; t < 15; ++t) B1[t * n2 + j] = gb[t];
      } else {
#pragma unroll
        for (int t = 0; t < 15; ++t) V0[t * n2 + p] = gb[t];
      }
    }
    if (R.map >= 0) {
      // permutation map: this thread alone read the inputs at p and perm[p]
      const int j = c.perms[(size_t)R.map + p];
      double* W0 = c.Tv + R.toff;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        if (KIND == 0) {
          W0[v * n2 + p] += UbL[v];
          W0[(5 + v) * n2 + j] += UbR[v];
        } else {
          W0[v * n2 + p] = UbL[v];
          W0[(5 + v) * n2 + j] = UbR[v];
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sF[(fl * 5 + v) * n2 + p] = UbL[v];
        sR[(fl * 5 + v) * n2 + p] = UbR[v];
      }
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int fl = w / n2, q = w - fl * n2;
    const FaceRec& R = c.faces[fb.first + fl];
    if (R.map >= 0) continue;
    double* S0 = c.Tv + R.toff;
    double* S1 = S0 + 5 * n2;
    const double* Fl = sF + fl * 5 * n2;
    const double* Fr = sR + fl * 5 * n2;
    const double keep = KIND == 0 ? 1.0 : 0.0;     // lifting values add to the flux cotangents
#pragma unroll
    for (int v = 0; v < 5; ++v) S0[v * n2 + q] = keep * S0[v * n2 + q] + Fl[v * n2 + q];
    const double* P0 = c.Vt + 3 * R.toff;          // parked neighbour gradient cotangents
    double* B1 = c.Vtb + 3 * R.toff + 15 * n2;
    {
      const double* D = c.dense + (size_t)(-1 - R.map) + q;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int p = 0; p < n2; ++p) acc = fma(D[(size_t)p * n2], Fr[v * n2 + p], acc);
        S1[v * n2 + q] = keep * S1[v * n2 + q] + acc;
      }
      if (KIND == 1) {
        for (int t = 0; t < 15; ++t) {
          double acc = 0.0;
          for (int p = 0; p < n2; ++p) acc = fma(D[(size_t)p * n2], P0[t * n2 + p], acc);
          B1[t * n2 + q] = acc;
        }
      }
    }
  }
}

// Storage <-> caller layout copies (warp per element).
// Halo exchange of a partition mesh: copies whole face-side trace blocks of
// `per` doubles between the face buffer at the listed offsets and a packed
// buffer (pack: buffer block k <- T[off[k]]; unpack: T[off[k]] <- block k).
__global__ void halo_copy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                 const int64_t* __restrict__ off, int64_t count, int per, int pack, int mult) {
  for (int64_t k = blockIdx.x; k < count; k += gridDim.x) {
    const int64_t o = mult * off[k];
    for (int w = threadIdx.x; w < per; w += blockDim.x) {
      if (pack) dst[k * per + w] = src[o + w];
      else dst[o + w] = src[k * per + w];
    }
  }
}

__global__ void rk_params_kernel(RkDyn* d, double* Q, double* K, double dt) {
  d->Q = Q;
  d->K = K;
  d->dt = dt;
}

__global__ void permute_kernel(Ctx c, const double* __restrict__ src, double* __restrict__ dst, int64_t E, int to_storage) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (s >= E) return;
  const int nM = c.tabs[c.slot_tab[s]].nM;
  int64_t so = c.slot_qoff[s], eo = c.elem_qoff[c.elem_of_slot[s]];
  const double* a = src + (to_storage ? eo : so);
  double* b = dst + (to_storage ? so : eo);
  for (int w = lane; w < 5 * nM; w += 32) b[w] = a[w];
}

// ------------------------------------------------------------------ moving meshes: stage mass matrices
//
// M^ = V^T diag(w J^) V with J^ = sum_k tau_k J_k per element (the stage
// value of J of a moving mesh).  Hexahedra hold s = W^{1/2} V q, so M^ q in
// their storage is J^ s pointwise and the solve a pointwise division.
// Prisms and pyramids: the product M^ x runs as the two sum-factorised
// transforms of the element kernel around the pointwise w J^ (FP64).  The
// solve is iterative refinement in FP64 around an FP32 Cholesky factor of the
// diagonally scaled S M^ S (S = diag(M^)^{-1/2}, condition number near
// max J / min J): x = 0, r = b; three times z = S (L L^T)^{-1} S r in FP32,
// x += z, r = b - M^ x in FP64.  Each FP32 solve gains about six digits,
// so the third correction leaves the FP64 rounding of M^ x.  Started from a
// nearby state x0 instead (the previous stage's, about 1e-3 away), two
// corrections reach the same.  FP64 work per solve is two products, against
// nM^3 / 3 FP64 flops for an FP64 Cholesky (FP64 issues at 1/64 of the FP32
// rate on this part).  A solve may keep its factor in global memory, and a
// later solve with a matrix equal to M^ within the FP32 rounding may use it
// instead of forming its own (the refinement runs with its own M^).
//
// smem: x, b, r [5][nM] and wJ [nQ] (FP64); bufA, bufB [5][nQ] (FP64,
// transforms; during the factor, bufA holds its two panel buffers); L
// (packed lower triangle), s, rdiag [nM] (FP32).  Block: 5 warps.
constexpr int kMassThreads = 160;
static_assert(kMassThreads % 32 == 0 && kMassThreads >= 64, "the factor needs warp 0 and at least one other warp");
constexpr int kMassRows = 4;   // rows per lane in the warp solves: nM <= 128

// the FP32 factor is kept packed: row i of the lower triangle at i (i + 1) / 2
__host__ __device__ __forceinline__ int lro(int i) { return i * (i + 1) / 2; }

__host__ __device__ __forceinline__ size_t mass_smem_doubles(int nM, int nQ) {
  return 15 * (size_t)nM + (size_t)nQ + 10 * (size_t)nQ;
}

// r = b - M^ x (or r = M^ x when b is null); tid = threadIdx.x
__device__ void mass_product(const Ctx& c, const TypeTab& T, const double* x, const double* wJ, const double* b,
                             double* r, double* bufA, double* bufB, int tid) {
  const int nQ = T.nQ, nM = T.nM;
  modal_to_nodal_passes(c, T, x, bufA, bufB, tid);
  for (int w = tid; w < 5 * nQ; w += blockDim.x) bufA[w] *= wJ[w % nQ];
  __syncthreads();
  Epilogue ep{Epilogue::kStore, false, 1.0, r, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
  nodal_to_modal_t<false>(c, T, bufA, bufB, tid, ep);
  if (b) {
    for (int w = tid; w < 5 * nM; w += blockDim.x) r[w] = b[w] - r[w];
    __syncthreads();
  }
}

// x += S (L L^T)^{-1} S r: warp v solves for variable v (ROWS rows per lane
// in registers, one shuffle per pivot, the rows already solved masked by a
// zero coefficient instead of a branch).  The five warps run side by side.
template <int ROWS>
__device__ void mass_correct_t(const float* L, const float* sc, const float* rdiag, const double* r, double* x,
                               int nM) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (v < 5) {
    const double* rv = r + v * nM;
    float y[ROWS], sl[ROWS];
#pragma unroll
    for (int m = 0; m < ROWS; ++m) {
      const int i = lane + 32 * m;
      sl[m] = i < nM ? sc[min(i, nM - 1)] : 0.0f;
      y[m] = i < nM ? sl[m] * (float)rv[min(i, nM - 1)] : 0.0f;
    }
    // L y = S r
#pragma unroll
    for (int m = 0; m < ROWS; ++m) {
      const int jend = min(32, nM - 32 * m);
      for (int jj = 0; jj < jend; ++jj) {
        const int j = 32 * m + jj;
        const float yj = __shfl_sync(0xffffffffu, y[m], jj) * rdiag[j];
        y[m] = lane == jj ? yj : y[m];
#pragma unroll
        for (int m2 = m; m2 < ROWS; ++m2) {
          const int i = lane + 32 * m2;
          const float lij = (i > j && i < nM) ? L[lro(min(i, nM - 1)) + j] : 0.0f;
          y[m2] = fmaf(-lij, yj, y[m2]);
        }
      }
    }
    // L^T z = y
#pragma unroll
    for (int m = ROWS - 1; m >= 0; --m) {
      const int jend = min(32, nM - 32 * m);
      for (int jj = jend - 1; jj >= 0; --jj) {
        const int j = 32 * m + jj;
        const float zj = __shfl_sync(0xffffffffu, y[m], jj) * rdiag[j];
        y[m] = lane == jj ? zj : y[m];
#pragma unroll
        for (int m2 = 0; m2 <= m; ++m2) {
          const int i = lane + 32 * m2;
          const float lji = i < j ? L[lro(j) + min(i, j)] : 0.0f;
          y[m2] = fmaf(-lji, zj, y[m2]);
        }
      }
    }
    double* xv = x + v * nM;
#pragma unroll
    for (int m = 0; m < ROWS; ++m) {
      const int i = lane + 32 * m;
      if (i < nM) xv[i] += (double)(sl[m] * y[m]);
    }
  }
  __syncthreads();
}

// The FP32 factor L L^T = S M^ S of one element (S = diag(M^)^{-1/2}), from
// the four packed FP32 coefficient triangles Mk and the powers f of the
// stage time; pan: two buffers of four floats per row on a 16-byte boundary
// (scratch).
// One warp: columns jh .. jh+3 of the FP32 factor (rows jh .. nM-1, by lane
// in registers).  With prev (the previous panel's rows, four values each),
// its rank-4 update of these columns comes first (the earlier panels' updates
// are in L already).  Leaves the factored columns in L, their reciprocal
// diagonal in rdiag and the rows below the panel in out.
template <int ROWS>
__device__ __forceinline__ void mass_panel(float* L, float* rdiag, float4* out, const float4* prev, int jh, int nM,
                                           int lane) {
  const int hw = min(4, nM - jh);
  float p[ROWS][4];
#pragma unroll
  for (int m = 0; m < ROWS; ++m) {
    const int i = jh + lane + 32 * m, ic = min(i, nM - 1);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      p[m][cc] = (i < nM && cc < hw && jh + cc <= i) ? L[lro(ic) + min(jh + cc, ic)] : 0.0f;
  }
  if (prev) {
#pragma unroll
    for (int m = 0; m < ROWS; ++m) {
      const float4 a = prev[min(jh + lane + 32 * m, nM - 1)];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const float4 bb = prev[min(jh + cc, nM - 1)];
        p[m][cc] = fmaf(-a.w, bb.w, fmaf(-a.z, bb.z, fmaf(-a.y, bb.y, fmaf(-a.x, bb.x, p[m][cc]))));
      }
    }
  }
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    if (cc < hw) {
      // row jh + cc is lane cc of the first register row
      const float rd = rsqrtf(__shfl_sync(0xffffffffu, p[0][cc], cc));
      if (lane == 0) rdiag[jh + cc] = rd;
#pragma unroll
      for (int m = 0; m < ROWS; ++m)
        if (lane + 32 * m > cc) p[m][cc] *= rd;
#pragma unroll
      for (int c2 = cc + 1; c2 < 4; ++c2) {
        const float l = __shfl_sync(0xffffffffu, p[0][cc], c2);
#pragma unroll
        for (int m = 0; m < ROWS; ++m) p[m][c2] = fmaf(-p[m][cc], l, p[m][c2]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < ROWS; ++m) {
    const int i = jh + lane + 32 * m;
    if (i < nM) {
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
        if (cc < hw && jh + cc < i) L[lro(i) + jh + cc] = p[m][cc];
      if (i >= jh + hw)
        out[i] = make_float4(p[m][0], hw > 1 ? p[m][1] : 0.0f, hw > 2 ? p[m][2] : 0.0f, hw > 3 ? p[m][3] : 0.0f);
    }
  }
}

template <int ROWS>
__device__ void mass_factor(const float* Mk, float f0, float f1, float f2, float f3, float* L, float* sc, float* rdiag,
                            float4* pan, int nM) {
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
  const int np = lro(nM);
  // FP32 S M^ S from the FP32 coefficients, all four kept packed (lower
  // triangle, the layout of L): contiguous loads, then the scaling in
  // shared memory
#pragma unroll 4
  for (int u = tid; u < np; u += bd)
    L[u] = fmaf(f3, Mk[3 * np + u], fmaf(f2, Mk[2 * np + u], fmaf(f1, Mk[np + u], f0 * Mk[u])));
  __syncthreads();
  for (int a = tid; a < nM; a += bd) sc[a] = rsqrtf(L[lro(a) + a]);
  __syncthreads();
  for (int a = warp; a < nM; a += nwarps) {
    const float sa = sc[a];
    for (int k = lane; k <= a; k += 32) L[lro(a) + k] *= sa * sc[k];
  }
  __syncthreads();
  // right-looking Cholesky in panels of four columns with one panel of
  // lookahead: while warps 1-4 apply the current panel's rank-4 update to the
  // trailing lower triangle beyond the next panel (four rows per warp at a
  // time, independent chains that share each column's load), warp 0 applies
  // it to the next panel's four columns in registers and factors them.  One
  // barrier per panel.  L's diagonal is kept as its reciprocal in rdiag.
  float4* cur = pan;
  float4* nxt = pan + nM;
  if (warp == 0) mass_panel<ROWS>(L, rdiag, cur, nullptr, 0, nM, lane);
  __syncthreads();
  for (int j0 = 0; j0 + 4 < nM; j0 += 4) {
    const int jt = j0 + 4;   // the next panel
    if (warp == 0) {
      mass_panel<ROWS>(L, rdiag, nxt, cur, jt, nM, lane);
    } else {
      const int j4 = jt + 4, wt = warp - 1, nwt = nwarps - 1;
      for (int i = j4 + wt; i < nM; i += 4 * nwt) {
        float4 lr[4];
        int last = i;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          lr[g] = cur[min(i + g * nwt, nM - 1)];
          if (i + g * nwt < nM) last = i + g * nwt;
        }
        for (int k = j4 + lane; k <= last; k += 32) {
          const float4 ck = cur[k];
          float v[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int ig = i + g * nwt;
            v[g] = (ig < nM && k <= ig) ? L[lro(min(ig, nM - 1)) + k] : 0.0f;
          }
#pragma unroll
          for (int g = 0; g < 4; ++g)
            v[g] = fmaf(-lr[g].w, ck.w, fmaf(-lr[g].z, ck.z, fmaf(-lr[g].y, ck.y, fmaf(-lr[g].x, ck.x, v[g]))));
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int ig = i + g * nwt;
            if (ig < nM && k <= ig) L[lro(ig) + k] = v[g];
          }
        }
      }
    }
    __syncthreads();
    float4* t = cur;
    cur = nxt;
    nxt = t;
  }
}

template <int ROWS, int MINB>
__global__ void __launch_bounds__(kMassThreads, MINB) moving_mass_kernel(Ctx c, const int64_t* list, int64_t E,
                                                                   const double* in, double* out, const double* x0,
                                                                   double t0, double t1, double t2, double t3,
                                                                   int weight, int max_nM, int max_nQ, int nblk,
                                                                   int64_t blk_stride, float* fac_out,
                                                                   const float* fac_in) {
  extern __shared__ double sm[];
  const int tid = threadIdx.x, bd = blockDim.x;
  double* x = sm;
  double* b = x + 5 * max_nM;
  double* r = b + 5 * max_nM;
  double* wJ = r + 5 * max_nM;
  double* bufA = wJ + max_nQ;
  double* bufB = bufA + 5 * max_nQ;
  float* L = reinterpret_cast<float*>(bufB + 5 * max_nQ);
  float* sc = L + lro(max_nM);
  float* rdiag = sc + max_nM;
  for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
    const int64_t s = list[e];
    const TypeTab& T = c.tabs[c.slot_tab[s]];
    const int nQ = T.nQ, nM = T.nM;
    const int64_t qoff = c.slot_qoff[s];
    const double* m = c.mpool + c.slot_moff[s];
    if (T.type == HEX) {
      for (int w = tid; w < 5 * nQ * nblk; w += bd) {
        const int kb = w / (5 * nQ), wl = w - kb * 5 * nQ, q = wl % nQ;
        const int64_t o = qoff + kb * blk_stride + wl;
        const double J = fma(t3, m[30 * nQ + q], fma(t2, m[29 * nQ + q], fma(t1, m[28 * nQ + q], t0 * m[27 * nQ + q])));
        const double v = in[o];
        out[o] = weight ? v * J : v / J;
      }
      continue;   // block-uniform branch, no shared memory used
    }
    const double* W = c.dpool + T.W;
    for (int q = tid; q < nQ; q += bd)
      wJ[q] = W[q] * fma(t3, m[30 * nQ + q], fma(t2, m[29 * nQ + q], fma(t1, m[28 * nQ + q], t0 * m[27 * nQ + q])));
    for (int w = tid; w < 5 * nM; w += bd) b[w] = in[qoff + w];
    __syncthreads();
    if (weight) {
      mass_product(c, T, b, wJ, nullptr, r, bufA, bufB, tid);
      for (int w = tid; w < 5 * nM; w += bd) out[qoff + w] = r[w];
      __syncthreads();
      continue;
    }
    const int np = lro(nM);
    if (fac_in) {
      // a factor kept from a solve with (nearly) the same matrix: the
      // refinement below corrects for the difference in FP64
      const float* F = fac_in + c.slot_mmoff[s];
      for (int u = tid; u < np; u += bd) L[u] = F[u];
      for (int a = tid; a < nM; a += bd) {
        sc[a] = F[np + a];
        rdiag[a] = F[np + nM + a];
      }
      __syncthreads();
    } else {
      // pan lives in the transform buffer, idle until the first product, on
      // a 16-byte boundary
      mass_factor<ROWS>(c.mk32 + c.slot_mmoff[s], (float)t0, (float)t1, (float)t2, (float)t3, L, sc, rdiag,
                  reinterpret_cast<float4*>(bufA + ((15 * max_nM + max_nQ) & 1)), nM);
      if (fac_out) {
        // kept for a later solve (the lifting of the stage): [L][s][rdiag]
        float* F = fac_out + c.slot_mmoff[s];
        for (int u = tid; u < np; u += bd) F[u] = L[u];
        for (int a = tid; a < nM; a += bd) {
          F[np + a] = sc[a];
          F[np + nM + a] = rdiag[a];
        }
      }
    }
    // every block of five variables with the one factor (nblk > 1: the
    // lifting's three directions), from x0 (a nearby solution: one
    // correction fewer) or from zero
    for (int kb = 0; kb < nblk; ++kb) {
      const int64_t o = qoff + kb * blk_stride;
      if (kb > 0) {
        for (int w = tid; w < 5 * nM; w += bd) b[w] = in[o + w];
        __syncthreads();
      }
      for (int w = tid; w < 5 * nM; w += bd) {
        x[w] = x0 ? x0[o + w] : 0.0;
        r[w] = b[w];
      }
      __syncthreads();
      if (x0) mass_product(c, T, x, wJ, b, r, bufA, bufB, tid);
      const int ncorr = x0 ? 2 : 3;
      for (int it = 0; it < ncorr; ++it) {
        mass_correct_t<ROWS>(L, sc, rdiag, r, x, nM);
        if (it + 1 < ncorr) mass_product(c, T, x, wJ, b, r, bufA, bufB, tid);
      }
      for (int w = tid; w < 5 * nM; w += bd) out[o + w] = x[w];
      __syncthreads();
    }
  }
}

}  // namespace

int element_smem_bytes(int nQmax, int) { return 20 * nQmax * (int)sizeof(double); }

int element_launch_smem_bytes(int nQmax, int wpb, bool split) {
  int b = element_smem_bytes(nQmax, wpb);
  if (!split) return b;
  int n = 1;
  while (n * n * n < nQmax) ++n;
  // bufA [5 nQ] + two-point quantities [kTP][nQ] + face states [kTP][6 n^2]
  // + one direction's pair fluxes [n^2][n(n-1)/2][5] and face-state fluxes [n^2][2 n][5]
  const int sb = (5 * nQmax + kTP * nQmax + kTP * 6 * n * n + n * n * (n * (n - 1) / 2) * 5 + n * n * 2 * n * 5) *
                 (int)sizeof(double);
  return b > sb ? b : sb;
}
int face_block_threads(int n) { return 32 * n; }

namespace {
template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <int MODE>
cudaError_t set_mode(int bytes) {
  cudaError_t e;
  if ((e = set_smem(elem_naive_kernel<MODE, false>, bytes)) != cudaSuccess) return e;
  if ((e = set_smem(elem_naive_kernel<MODE, true>, bytes)) != cudaSuccess) return e;
  if ((e = set_smem(elem_balanced_kernel<MODE, false>, bytes)) != cudaSuccess) return e;
  return set_smem(elem_balanced_kernel<MODE, true>, bytes);
}
template <int MODE, bool ANY>
void launch_mode_t(const Ctx& c, const StageArgs& a, const Sched& s, bool balanced, int grid, int wpb, int bytes,
                   cudaStream_t st) {
  if (balanced) {
    elem_balanced_kernel<MODE, ANY><<<grid, 32 * wpb, bytes, st>>>(c, a, s.list, s.chunk_start, s.count, s.counter,
                                                                   s.next_counter);
  } else {
    if (s.count <= 0) return;
    elem_naive_kernel<MODE, ANY><<<(unsigned)s.count, 32 * wpb, bytes, st>>>(c, a, s.list, s.count);
  }
}
template <int MODE>
void launch_mode(const Ctx& c, const StageArgs& a, const Sched& s, bool balanced, int grid, int wpb, int bytes,
                 cudaStream_t st) {
  if (c.slot_coff) launch_mode_t<MODE, true>(c, a, s, balanced, grid, wpb, bytes, st);
  else launch_mode_t<MODE, false>(c, a, s, balanced, grid, wpb, bytes, st);
}
}  // namespace

int element_smem_bytes_ns(int nQmax) { return 40 * nQmax * (int)sizeof(double); }

// The shared-memory limits are per kernel function and process-wide, so they
// are set for the largest element any mesh may hold (N = kMaxN); the
// occupancy query uses this mesh's own launch size.
constexpr int kMaxnQ = kMaxn * kMaxn * kMaxn;

cudaError_t element_kernel_attributes_ns(int nQmax, int wpb, int* blocks_per_sm, bool curved) {
  cudaError_t e;
  if ((e = set_mode<kNsVolume>(element_smem_bytes_ns(kMaxnQ))) != cudaSuccess) return e;
  const int fbytes = 32 * 5 * kMaxn * kMaxn * (int)sizeof(double);
  if ((e = set_smem(face_ns_kernel<0, false>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_kernel<1, false>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_kernel<0, true>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_kernel<1, true>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_vjp_kernel<0, false>, 2 * fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_vjp_kernel<1, false>, 2 * fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_vjp_kernel<0, true>, 2 * fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_ns_vjp_kernel<1, true>, 2 * fbytes)) != cudaSuccess) return e;
  if (curved)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, elem_balanced_kernel<kNsVolume, true>, 32 * wpb,
                                                         element_smem_bytes_ns(nQmax));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, elem_balanced_kernel<kNsVolume, false>, 32 * wpb,
                                                       element_smem_bytes_ns(nQmax));
}

cudaError_t element_kernel_attributes(int nQmax, int wpb, int* blocks_per_sm, bool curved, bool split) {
  const int bmax = element_launch_smem_bytes(kMaxnQ, wpb, true);
  cudaError_t e;
  if ((e = set_mode<kFwd>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kBwdRhs>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kBwdRk>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kBwdRkFwd>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kProject>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kEval>(bmax)) != cudaSuccess) return e;
  if ((e = set_mode<kLoad>(bmax)) != cudaSuccess) return e;
  if ((e = set_smem(elem_naive_kernel<kGather, false>, bmax)) != cudaSuccess) return e;
  if ((e = set_smem(elem_naive_kernel<kScatter, false>, bmax)) != cudaSuccess) return e;
  int fbytes = 32 * 5 * kMaxn * kMaxn * (int)sizeof(double);
  if ((e = set_smem(face_kernel<false>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_kernel<true>, fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_vjp_kernel<false>, 2 * fbytes)) != cudaSuccess) return e;
  if ((e = set_smem(face_vjp_kernel<true>, 2 * fbytes)) != cudaSuccess) return e;
  const int vb = (int)sizeof(double) * kMaxnQ;
  if ((e = set_smem(elem_vjp_kernel<0, false>, 25 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<2, false>, 20 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<10, false>, 25 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<11, false>, 45 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<0, true>, 25 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<2, true>, 20 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<10, true>, 25 * vb)) != cudaSuccess) return e;
  if ((e = set_smem(elem_vjp_kernel<11, true>, 45 * vb)) != cudaSuccess) return e;
  if (curved)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, elem_balanced_kernel<kBwdRkFwd, true>, 32 * wpb,
                                                         element_smem_bytes(nQmax, wpb));
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, elem_balanced_kernel<kBwdRkFwd, false>, 32 * wpb,
                                                       element_launch_smem_bytes(nQmax, wpb, split));
}

void launch_element(const Ctx& c, int mode, const StageArgs& a, const Sched& s, bool balanced, int grid, int wpb,
                    cudaStream_t st) {
  int bytes = mode == kNsVolume ? element_smem_bytes_ns(c.nQmax) : element_launch_smem_bytes(c.nQmax, wpb, c.split != 0);
  switch (mode) {
    case kNsVolume: launch_mode<kNsVolume>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kFwd: launch_mode<kFwd>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kBwdRhs: launch_mode<kBwdRhs>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kBwdRk: launch_mode<kBwdRk>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kBwdRkFwd: launch_mode<kBwdRkFwd>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kProject: launch_mode<kProject>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kEval: launch_mode<kEval>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kLoad: launch_mode<kLoad>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kTraces: launch_mode<kTraces>(c, a, s, balanced, grid, wpb, bytes, st); break;
    case kGather:   // one block per listed hexahedron
      if (s.count > 0) elem_naive_kernel<kGather, false><<<(unsigned)s.count, 32 * wpb, bytes, st>>>(c, a, s.list, s.count);
      break;
    case kScatter:
      if (s.count > 0) elem_naive_kernel<kScatter, false><<<(unsigned)s.count, 32 * wpb, bytes, st>>>(c, a, s.list, s.count);
      break;
  }
}

void launch_faces_ns_vjp(const Ctx& c, int64_t nblocks, int n, int kind, cudaStream_t st) {
  if (nblocks <= 0) return;
  int bytes = 2 * 32 * 5 * n * n * (int)sizeof(double);
  const unsigned nb = (unsigned)nblocks, nt = face_block_threads(n);
  if (c.fgeo) {
    if (kind == 0) face_ns_vjp_kernel<0, true><<<nb, nt, bytes, st>>>(c);
    else face_ns_vjp_kernel<1, true><<<nb, nt, bytes, st>>>(c);
  } else {
    if (kind == 0) face_ns_vjp_kernel<0, false><<<nb, nt, bytes, st>>>(c);
    else face_ns_vjp_kernel<1, false><<<nb, nt, bytes, st>>>(c);
  }
}

void launch_vjp(const Ctx& c, int phase, const VjpArgs& va, int64_t nelem, int wpb, cudaStream_t st) {
  if (nelem <= 0) return;
  const int per = phase == 0 || phase == 10 ? 25 : (phase == 11 ? 45 : 20);
  const int bytes = per * c.nQmax * (int)sizeof(double);
  const unsigned nb = (unsigned)nelem, nt = 32 * wpb;
  if (c.slot_coff) {
    switch (phase) {
      case 0: elem_vjp_kernel<0, true><<<nb, nt, bytes, st>>>(c, va); break;
      case 10: elem_vjp_kernel<10, true><<<nb, nt, bytes, st>>>(c, va); break;
      case 11: elem_vjp_kernel<11, true><<<nb, nt, bytes, st>>>(c, va); break;
      default: elem_vjp_kernel<2, false><<<nb, nt, bytes, st>>>(c, va); break;   // phase C has no geometry
    }
  } else {
    switch (phase) {
      case 0: elem_vjp_kernel<0, false><<<nb, nt, bytes, st>>>(c, va); break;
      case 10: elem_vjp_kernel<10, false><<<nb, nt, bytes, st>>>(c, va); break;
      case 11: elem_vjp_kernel<11, false><<<nb, nt, bytes, st>>>(c, va); break;
      default: elem_vjp_kernel<2, false><<<nb, nt, bytes, st>>>(c, va); break;
    }
  }
}

void launch_faces_vjp(const Ctx& c, int64_t nblocks, int n, cudaStream_t st) {
  if (nblocks <= 0) return;
  int bytes = 2 * 32 * 5 * n * n * (int)sizeof(double);
  if (c.fgeo) face_vjp_kernel<true><<<(unsigned)nblocks, face_block_threads(n), bytes, st>>>(c);
  else face_vjp_kernel<false><<<(unsigned)nblocks, face_block_threads(n), bytes, st>>>(c);
}

void launch_faces_ns(const Ctx& c, int64_t nblocks, int n, int kind, cudaStream_t st) {
  if (nblocks <= 0) return;
  int bytes = 32 * 5 * n * n * (int)sizeof(double);
  const unsigned nb = (unsigned)nblocks, nt = face_block_threads(n);
  if (c.fgeo) {
    if (kind == 0) face_ns_kernel<0, true><<<nb, nt, bytes, st>>>(c);
    else face_ns_kernel<1, true><<<nb, nt, bytes, st>>>(c);
  } else {
    if (kind == 0) face_ns_kernel<0, false><<<nb, nt, bytes, st>>>(c);
    else face_ns_kernel<1, false><<<nb, nt, bytes, st>>>(c);
  }
}

void launch_faces(const Ctx& c, int64_t nblocks, int n, cudaStream_t st) {
  if (nblocks <= 0) return;
  int bytes = 32 * 5 * n * n * (int)sizeof(double);
  if (c.fgeo) face_kernel<true><<<(unsigned)nblocks, face_block_threads(n), bytes, st>>>(c);
  else face_kernel<false><<<(unsigned)nblocks, face_block_threads(n), bytes, st>>>(c);
}

void launch_halo_copy(const double* src, double* dst, const int64_t* off, int64_t count, int per, bool pack,
                      cudaStream_t st, int mult) {
  if (count <= 0) return;
  const unsigned blocks = (unsigned)std::min<int64_t>(count, 65535);
  halo_copy_kernel<<<blocks, 128, 0, st>>>(src, dst, off, count, per, pack ? 1 : 0, mult);
}

void launch_rk_params(RkDyn* d, double* Q, double* K, double dt, cudaStream_t st) {
  rk_params_kernel<<<1, 1, 0, st>>>(d, Q, K, dt);
}

void rk_params_node(cudaKernelNodeParams* p, void** args) {
  p->func = (void*)rk_params_kernel;
  p->gridDim = dim3(1, 1, 1);
  p->blockDim = dim3(1, 1, 1);
  p->sharedMemBytes = 0;
  p->kernelParams = args;
  p->extra = nullptr;
}

bool is_rk_params_kernel(const void* func) { return func == (const void*)rk_params_kernel; }

void launch_permute(const Ctx& c, const double* src, double* dst, int64_t E, int to_storage, cudaStream_t st) {
  const int wpb = 4;
  int64_t blocks = (E + wpb - 1) / wpb;
  permute_kernel<<<(unsigned)blocks, 32 * wpb, 0, st>>>(c, src, dst, E, to_storage);
}


cudaError_t launch_moving_mass(const Ctx& c, const int64_t* list, int64_t n_slots, const double* in, double* out,
                               const double* x0, const double* tau, int weight, int max_nM, int max_nQ, int grid,
                               cudaStream_t st, int nblk, int64_t blk_stride, float* fac_out,
                               const float* fac_in) {
  if (weight && nblk != 1) return cudaErrorInvalidValue;
  if (weight && (fac_out || fac_in)) return cudaErrorInvalidValue;
  if (max_nM > 32 * kMassRows) return cudaErrorInvalidValue;
  size_t bytes = 0;
  if (max_nM > 0)
    bytes = sizeof(double) * mass_smem_doubles(max_nM, max_nQ) + sizeof(float) * ((size_t)lro(max_nM) + 2 * (size_t)max_nM);
  // rows per lane in the warp solves and the panel (nM <= 32 ROWS); with two
  // (pyramids and prisms up to N = 3) eight blocks fit an SM's registers
  auto launch = [&](auto kern) -> cudaError_t {
    if (bytes > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, kMassThreads, bytes, st>>>(c, list, n_slots, in, out, x0, tau[0], tau[1], tau[2], tau[3], weight,
                                             max_nM, max_nQ, nblk, blk_stride, fac_out, fac_in);
    return cudaSuccess;
  };
  cudaError_t e;
  if (max_nM <= 64) e = launch(moving_mass_kernel<2, 8>);
  else if (max_nM <= 96) e = launch(moving_mass_kernel<3, 7>);
  else e = launch(moving_mass_kernel<4, 7>);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dgk
