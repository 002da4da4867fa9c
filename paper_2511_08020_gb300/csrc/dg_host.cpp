// Host set-up: operator tables per (type, N), affine geometry, face
// connectivity with the owner rule, neighbour maps, Hilbert ordering.
//
// The discretisation is the modal weak form of Eq. 1 (Sec. 2 of Kopper et
// al.): orthonormal modal bases on the reference hex / prism / pyramid / tet,
// collapsed (Duffy) Gauss-Legendre quadrature with n = N+1 points per
// direction, faces integrated with the owner's face rule.
#include "dg_host.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <unordered_map>
#include <atomic>
#include <thread>

namespace dgh {

using dgk::FaceDesc;
using dgk::TypeTab;

// ============================================================ 1D building blocks

// Gauss-Legendre nodes (ascending) and weights by Newton iteration on the
// three-term Legendre recurrence, started from the Chebyshev-like guess
// cos(pi (i + 3/4) / (n + 1/2)); nodes are symmetrised exactly.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    x[n - 1 - i] = z;
    x[i] = -z;
    w[i] = w[n - 1 - i] = wt;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Jacobi P_n^(alpha,beta)(x) by the standard three-term recurrence.
double jacobi(int n, double al, double be, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * (al - be + (al + be + 2.0) * x);
  for (int k = 2; k <= n; ++k) {
    double a = al + be;
    double c1 = 2.0 * k * (k + a) * (2.0 * k + a - 2.0);
    double c2 = (2.0 * k + a - 1.0) * ((2.0 * k + a) * (2.0 * k + a - 2.0) * x + al * al - be * be);
    double c3 = 2.0 * (k + al - 1.0) * (k + be - 1.0) * (2.0 * k + a);
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double jhat(int n, int alpha, double x) {
  return jacobi(n, alpha, 0.0, x) * std::sqrt((2.0 * n + alpha + 1.0) / 2.0);
}

void lagrange_values(const double* nodes, int n, double x, double* out) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (x - nodes[k]) / (nodes[j] - nodes[k]);
    out[j] = v;
  }
}

// ============================================================ reference elements

const double kRefVerts[4][8][3] = {
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}, {1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}},
};
const int kNumVerts[4] = {8, 6, 5, 4};
const int kNumFaces[4] = {6, 5, 5, 4};
// Local faces as vertex lists; face parameters x(s,t) = c0 + (s+1)/2 (c1-c0) + (t+1)/2 (c2-c0).
const int kFaceVerts[4][6][4] = {
    {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 2, 4, 6}, {1, 3, 5, 7}},
    {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 3, 4}, {0, 2, 3, 5}, {1, 2, 4, 5}, {-1, -1, -1, -1}},
    {{0, 1, 2, 3}, {0, 1, 4, -1}, {0, 2, 4, -1}, {1, 3, 4, -1}, {2, 3, 4, -1}, {-1, -1, -1, -1}},
    {{0, 1, 2, -1}, {0, 1, 3, -1}, {0, 2, 3, -1}, {1, 2, 3, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}},
};
const int kFaceNV[4][6] = {{4, 4, 4, 4, 4, 4}, {3, 3, 4, 4, 4, 0}, {4, 3, 3, 3, 3, 0}, {3, 3, 3, 3, 0, 0}};

// Face points of every local face lie on the collapsed tensor grid: one
// collapsed coordinate is fixed at an end, the face parameters run along two
// others.  (Checked numerically in Tables::add.)
static const FaceDesc kFaceDesc[4][6] = {
    {{2, 0, 0, 1, 0}, {2, 1, 0, 1, 0}, {1, 0, 0, 2, 0}, {1, 1, 0, 2, 0}, {0, 0, 1, 2, 0}, {0, 1, 1, 2, 0}},
    {{2, 0, 0, 1, 1}, {2, 1, 0, 1, 1}, {1, 0, 0, 2, 0}, {0, 0, 1, 2, 0}, {0, 1, 1, 2, 0}, {0, 0, 0, 0, 0}},
    {{2, 0, 0, 1, 0}, {1, 0, 0, 2, 1}, {0, 0, 1, 2, 1}, {0, 1, 1, 2, 1}, {1, 1, 0, 2, 1}, {0, 0, 0, 0, 0}},
    {{2, 0, 0, 1, 1}, {1, 0, 0, 2, 1}, {0, 0, 1, 2, 1}, {0, 1, 1, 2, 1}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}},
};

int n_modes(int type, int N) {
  int n = N + 1;
  switch (type) {
    case dgk::HEX: return n * n * n;
    case dgk::PRISM: return n * n * (n + 1) / 2;
    case dgk::PYR: return n * (n + 1) * (2 * n + 1) / 6;
    case dgk::TET: return n * (n + 1) * (n + 2) / 6;
  }
  return 0;
}

static int q_count(int type, int N, int p) { return (type == dgk::PRISM || type == dgk::TET) ? N - p + 1 : N + 1; }
static int r_count(int type, int N, int p, int q) {
  switch (type) {
    case dgk::HEX:
    case dgk::PRISM: return N + 1;
    case dgk::TET: return N - p - q + 1;
    case dgk::PYR: return N - std::max(p, q) + 1;
  }
  return 0;
}

// The orthonormal basis phi_pqr = A_p(a) B_pq(b) C_pqr(c):
//   hex      L_p(a) L_q(b) L_r(c)
//   prism    L_p(a) ((1-b)/2)^p J_q^(2p+1)(b) L_r(c)
//   pyramid  L_p(a) L_q(b) ((1-c)/2)^m J_r^(2m+2)(c),        m = max(p, q)
//   tet      L_p(a) ((1-b)/2)^p J_q^(2p+1)(b) ((1-c)/2)^(p+q) J_r^(2p+2q+2)(c)
double factor_A(int, int p, double a) { return jhat(p, 0, a); }
double factor_B(int type, int p, int q, double b) {
  if (type == dgk::HEX || type == dgk::PYR) return jhat(q, 0, b);
  return std::pow(0.5 * (1.0 - b), p) * jhat(q, 2 * p + 1, b);
}
double factor_C(int type, int p, int q, int r, double c) {
  switch (type) {
    case dgk::HEX:
    case dgk::PRISM: return jhat(r, 0, c);
    case dgk::TET: return std::pow(0.5 * (1.0 - c), p + q) * jhat(r, 2 * p + 2 * q + 2, c);
    case dgk::PYR: {
      int m = std::max(p, q);
      return std::pow(0.5 * (1.0 - c), m) * jhat(r, 2 * m + 2, c);
    }
  }
  return 0.0;
}

void uncollapse(int type, double a, double b, double c, double* xi) {
  switch (type) {
    case dgk::HEX: xi[0] = a; xi[1] = b; xi[2] = c; break;
    case dgk::PRISM: xi[0] = 0.5 * (1 + a) * (1 - b) - 1; xi[1] = b; xi[2] = c; break;
    case dgk::TET:
      xi[0] = 0.25 * (1 + a) * (1 - b) * (1 - c) - 1;
      xi[1] = 0.5 * (1 + b) * (1 - c) - 1;
      xi[2] = c;
      break;
    case dgk::PYR:
      xi[0] = 0.5 * (1 + a) * (1 - c) - 1;
      xi[1] = 0.5 * (1 + b) * (1 - c) - 1;
      xi[2] = c;
      break;
  }
}

static void collapse(int type, const double* xi, double* abc) {
  switch (type) {
    case dgk::HEX: abc[0] = xi[0]; abc[1] = xi[1]; abc[2] = xi[2]; break;
    case dgk::PRISM: abc[0] = 2 * (1 + xi[0]) / (1 - xi[1]) - 1; abc[1] = xi[1]; abc[2] = xi[2]; break;
    case dgk::TET:
      abc[0] = 2 * (1 + xi[0]) / (-xi[1] - xi[2]) - 1;
      abc[1] = 2 * (1 + xi[1]) / (1 - xi[2]) - 1;
      abc[2] = xi[2];
      break;
    case dgk::PYR:
      abc[0] = 2 * (1 + xi[0]) / (1 - xi[2]) - 1;
      abc[1] = 2 * (1 + xi[1]) / (1 - xi[2]) - 1;
      abc[2] = xi[2];
      break;
  }
}

// Duffy Jacobian det d(xi)/d(abc) and the inverse map's derivatives
// d(a,b,c)_l / d(xi,eta,zeta)_k at a collapsed point.
static double duffy_det(int type, double, double b, double c) {
  switch (type) {
    case dgk::HEX: return 1.0;
    case dgk::PRISM: return 0.5 * (1 - b);
    case dgk::TET: return 0.5 * (1 - b) * 0.25 * (1 - c) * (1 - c);
    case dgk::PYR: return 0.25 * (1 - c) * (1 - c);
  }
  return 0.0;
}

static void collapse_metric(int type, double a, double b, double c, double M[3][3]) {
  std::memset(M, 0, sizeof(double) * 9);
  M[2][2] = 1.0;
  switch (type) {
    case dgk::HEX: M[0][0] = M[1][1] = 1.0; break;
    case dgk::PRISM:
      M[0][0] = 2.0 / (1 - b);
      M[0][1] = (1 + a) / (1 - b);
      M[1][1] = 1.0;
      break;
    case dgk::TET: {
      double s = 0.5 * (1 - b) * (1 - c);  // -eta - zeta
      M[0][0] = 2.0 / s;
      M[0][1] = M[0][2] = (1 + a) / s;
      M[1][1] = 2.0 / (1 - c);
      M[1][2] = (1 + b) / (1 - c);
      break;
    }
    case dgk::PYR:
      M[0][0] = 2.0 / (1 - c);
      M[0][2] = (1 + a) / (1 - c);
      M[1][1] = 2.0 / (1 - c);
      M[1][2] = (1 + b) / (1 - c);
      break;
  }
}

// ============================================================ operator tables

int Tables::find(int type, int N) const {
  for (size_t i = 0; i < tabs.size(); ++i)
    if (tabs[i].type == type && tabs[i].N == N) return (int)i;
  return -1;
}

int Tables::add(int type, int N, std::string* err) {
  int have = find(type, N);
  if (have >= 0) return have;
  TypeTab t;
  std::memset(&t, 0, sizeof(t));
  const int n = N + 1;
  t.type = type;
  t.N = N;
  t.n = n;
  t.nM = n_modes(type, N);
  t.nQ = n * n * n;
  t.nfaces = kNumFaces[type];
  std::vector<double> x(n), w(n);
  gauss_legendre(n, x.data(), w.data());
  auto dput = [&](double v) { dpool.push_back(v); };
  auto ialloc = [&](int cnt) { int o = (int)ipool.size(); ipool.resize(ipool.size() + cnt, 0); return o; };

  // A
  t.A = (int)dpool.size();
  for (int p = 0; p < n; ++p)
    for (int i = 0; i < n; ++i) dput(factor_A(type, p, x[i]));
  // columns (p, q) and B
  std::vector<int> cols_p, cols_q;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < q_count(type, N, p); ++q) { cols_p.push_back(p); cols_q.push_back(q); }
  t.ncols = (int)cols_p.size();
  t.p_cbase = ialloc(n);
  t.p_blen = ialloc(n);
  t.p_boff = ialloc(n);
  t.B = (int)dpool.size();
  {
    int col = 0;
    for (int p = 0; p < n; ++p) {
      ipool[t.p_cbase + p] = col;
      ipool[t.p_blen + p] = q_count(type, N, p);
      ipool[t.p_boff + p] = (int)dpool.size() - t.B;
      for (int q = 0; q < q_count(type, N, p); ++q)
        for (int j = 0; j < n; ++j) dput(factor_B(type, p, q, x[j]));
      col += q_count(type, N, p);
    }
  }
  // C and mode bookkeeping
  t.col_moff = ialloc(t.ncols);
  t.col_len = ialloc(t.ncols);
  t.col_coff = ialloc(t.ncols);
  t.col_p = ialloc(t.ncols);
  t.mode_col = ialloc(t.nM);
  t.C = (int)dpool.size();
  {
    int mode = 0;
    for (int col = 0; col < t.ncols; ++col) {
      int p = cols_p[col], q = cols_q[col];
      int len = r_count(type, N, p, q);
      ipool[t.col_moff + col] = mode;
      ipool[t.col_len + col] = len;
      ipool[t.col_coff + col] = (int)dpool.size() - t.C;
      ipool[t.col_p + col] = p;
      for (int r = 0; r < len; ++r) {
        ipool[t.mode_col + mode + r] = col;
        for (int k = 0; k < n; ++k) dput(factor_C(type, p, q, r, x[k]));
      }
      mode += len;
    }
    if (mode != t.nM) { *err = "internal: mode count mismatch"; return -1; }
    std::vector<int> order(t.ncols);
    for (int col = 0; col < t.ncols; ++col) order[col] = col;
    std::stable_sort(order.begin(), order.end(), [&](int ca, int cb) {
      return ipool[t.col_len + ca] > ipool[t.col_len + cb];
    });
    t.col_order = ialloc(t.ncols);
    for (int r = 0; r < t.ncols; ++r) ipool[t.col_order + r] = order[r];
  }
  // collocation derivative Dt[i'][i] = l'_{i'}(x_i) (barycentric formula)
  t.Dt = (int)dpool.size();
  std::vector<double> D(n * n, 0.0);  // D[i][j] = l'_j(x_i)
  {
    std::vector<double> lam(n, 1.0);
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k)
        if (k != j) lam[j] /= (x[j] - x[k]);
    for (int i = 0; i < n; ++i) {
      double diag = 0.0;
      for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
        diag -= D[i * n + j];
      }
      D[i * n + i] = diag;
    }
    for (int ip = 0; ip < n; ++ip)
      for (int i = 0; i < n; ++i) dput(D[i * n + ip]);
  }
  // hexahedra, entropy-stable split form: the antisymmetric part S = Q - Q^T
  // of the 1D Gauss collocation operator Q = W D, and the 1D weights
  t.sbp = -1;
  t.w1 = -1;
  if (type == dgk::HEX) {
    t.sbp = (int)dpool.size();
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) dput(w[i] * D[i * n + j] - w[j] * D[j * n + i]);
    t.w1 = (int)dpool.size();
    for (int i = 0; i < n; ++i) dput(w[i]);
  }
  // extrapolation to the ends
  t.ext = (int)dpool.size();
  {
    std::vector<double> l(n);
    lagrange_values(x.data(), n, -1.0, l.data());
    for (int m = 0; m < n; ++m) dput(l[m]);
    lagrange_values(x.data(), n, 1.0, l.data());
    for (int m = 0; m < n; ++m) dput(l[m]);
  }
  // volume weights times the collapse metric
  t.wA = (int)dpool.size();
  std::vector<double> wq(t.nQ);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        int q = (i * n + j) * n + k;
        wq[q] = w[i] * w[j] * w[k] * duffy_det(type, x[i], x[j], x[k]);
        double M[3][3];
        collapse_metric(type, x[i], x[j], x[k], M);
        for (int l = 0; l < 3; ++l)
          for (int kk = 0; kk < 3; ++kk) dput(wq[q] * M[l][kk]);
      }
  t.W = (int)dpool.size();
  for (int q = 0; q < t.nQ; ++q) dput(wq[q]);
  // mass matrix V^T W V: must be diagonal under the collapsed GL rule
  t.minv = (int)dpool.size();
  {
    std::vector<double> V((size_t)t.nQ * t.nM);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          int q = (i * n + j) * n + k;
          int mode = 0;
          for (int col = 0; col < t.ncols; ++col) {
            int p = cols_p[col], qq = cols_q[col];
            for (int r = 0; r < r_count(type, N, p, qq); ++r, ++mode)
              V[(size_t)q * t.nM + mode] = factor_A(type, p, x[i]) * factor_B(type, p, qq, x[j]) *
                                           factor_C(type, p, qq, r, x[k]);
          }
        }
    double maxd = 0.0, maxoff = 0.0;
    std::vector<double> diag(t.nM);
    for (int a = 0; a < t.nM; ++a)
      for (int b = 0; b < t.nM; ++b) {
        double s = 0.0;
        for (int q = 0; q < t.nQ; ++q) s += V[(size_t)q * t.nM + a] * wq[q] * V[(size_t)q * t.nM + b];
        if (a == b) { diag[a] = s; maxd = std::max(maxd, std::fabs(s)); }
        else maxoff = std::max(maxoff, std::fabs(s));
      }
    if (maxoff > 1e-12 * maxd) { *err = "mass matrix is not diagonal for this (type, N)"; return -7; }
    // hexahedron: the n-point rule integrates every product of two modes
    // exactly, so V^T W V is the identity (its computed diagonal differs
    // from 1 by rounding only)
    for (int a = 0; a < t.nM; ++a) dput(type == dgk::HEX ? 1.0 : 1.0 / diag[a]);
  }
  // Hexahedron: V is square and V^T W V = I, so W^{1/2} V is orthogonal and
  // the state is stored as the scaled nodal values s = W^{1/2} V Q.  Then
  // V Q = W^{-1/2} s and, for the projected residual, W^{1/2} V M^{-1} V^T h =
  // W^{-1/2} h: both transforms become pointwise scales (the hexahedron is
  // time-stepped in nodal values, as in the nodal DGSEM of Sec. 2, while the
  // other types stay modal -- the extra Vandermonde work of Sec. 2 falls on
  // them alone), and an orthogonal change of basis leaves inner products (so
  // every adjoint and cotangent) unchanged.  dg_set_state / dg_get_state
  // convert between the caller's modal coefficients and this storage.
  t.sqw = -1;
  if (type == dgk::HEX) {
    t.sqw = (int)dpool.size();
    for (int q = 0; q < t.nQ; ++q) dput(std::sqrt(wq[q]));
    for (int q = 0; q < t.nQ; ++q) dput(1.0 / std::sqrt(wq[q]));
  }
  // face descriptors + numerical check that the face rule points lie on the grid
  t.fw = (int)dpool.size();
  for (int lf = 0; lf < t.nfaces; ++lf) {
    FaceDesc d = kFaceDesc[type][lf];
    t.faces[lf] = d;
    const int* fv = kFaceVerts[type][lf];
    const double* c0 = kRefVerts[type][fv[0]];
    const double* c1 = kRefVerts[type][fv[1]];
    const double* c2 = kRefVerts[type][fv[2]];
    for (int ib = 0; ib < n; ++ib)
      for (int ia = 0; ia < n; ++ia) {
        double al = x[ia], be = x[ib];
        double s = d.tri ? 0.5 * (1 + al) * (1 - be) - 1 : al;
        double tt = be;
        double xi[3], abc[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k) xi[k] = c0[k] + 0.5 * (s + 1) * (c1[k] - c0[k]) + 0.5 * (tt + 1) * (c2[k] - c0[k]);
        collapse(type, xi, abc);
        double expect[3];
        expect[d.fixed] = d.end ? 1.0 : -1.0;
        expect[d.alpha] = al;
        expect[d.beta] = be;
        for (int k = 0; k < 3; ++k)
          if (std::fabs(abc[k] - expect[k]) > 1e-12) { *err = "internal: face table inconsistent"; return -1; }
        dput(d.tri ? w[ia] * w[ib] * 0.5 * (1 - be) : w[ia] * w[ib]);
      }
  }
  tabs.push_back(t);
  return (int)tabs.size() - 1;
}

double static_cost(const TypeTab& t) {
  // FP64 lane operations of one stage of one element (forward + backward
  // element work, pointwise flux, face share), used as the initial weight.
  double n = t.n, nQ = t.nQ;
  double vpass = 0;  // modal->nodal MACs per variable
  vpass += n * (double)t.nM;                        // c-pass (sum of r lengths times n)
  vpass += nQ * (t.type == dgk::PRISM || t.type == dgk::TET ? (n + 1) / 2.0 : n);  // b-pass
  vpass += nQ * n;                                  // a-pass
  double per_var = 2 * vpass + 3 * nQ * n + 2 * t.nfaces * n * n * n;
  return 5 * per_var + 60 * nQ + t.nfaces * n * n * 60;
}

// ============================================================ Hilbert keys

// Skilling (2004), "Programming the Hilbert curve": transpose form of the
// Hilbert index from axis coordinates, then bit interleaving into one key.
uint64_t hilbert_key3(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
  uint32_t X[3] = {x0, x1, x2};
  const uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    uint32_t P = Q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[2] & Q) t ^= Q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= t;
  uint64_t key = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
  return key;
}

// ============================================================ mesh

namespace {

struct Key3 {
  int64_t v[3];
  bool operator<(const Key3& o) const { return std::tie(v[0], v[1], v[2]) < std::tie(o.v[0], o.v[1], o.v[2]); }
  bool operator==(const Key3& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};
struct Key3Hash {
  size_t operator()(const Key3& k) const {
    uint64_t h = (uint64_t)k.v[0] * 0x9E3779B97F4A7C15ull ^ ((uint64_t)k.v[1] + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full ^
                 ((uint64_t)k.v[2] + 0x165667B19E3779F9ull);
    return (size_t)(h ^ (h >> 29));
  }
};

const int64_t kQuant = 1ll << 24;

Key3 reduce(const double* p, const double* period) {
  Key3 k;
  for (int d = 0; d < 3; ++d) {
    int64_t q = (int64_t)std::llround(p[d] / period[d] * (double)kQuant);
    q %= kQuant;
    if (q < 0) q += kQuant;
    k.v[d] = q;
  }
  return k;
}

struct FaceKey {
  Key3 c;
  Key3 v[4];
  int nv;
  bool operator<(const FaceKey& o) const {
    if (!(c == o.c)) return c < o.c;
    if (nv != o.nv) return nv < o.nv;
    for (int i = 0; i < nv; ++i)
      if (!(v[i] == o.v[i])) return v[i] < o.v[i];
    return false;
  }
};

void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

void inv3(const double A[3][3], double Ai[3][3]) {
  double d = det3(A);
  Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
  Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
  Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
}

// reference vertices spanning the affine map (images of the reference axes)
const int kAxisVert[4][3] = {{1, 2, 4}, {1, 2, 3}, {1, 2, 4}, {1, 2, 3}};

// ---- curved elements: vertex-interpolated maps x = sum_v N_v(xi) X_v
//   hex      N_v = prod_d (1 + r_vd xi_d)/2                     (trilinear)
//   prism    l_i(xi, eta) (1 -+ zeta)/2, l = (-(xi+eta)/2, (1+xi)/2, (1+eta)/2)
//   pyramid  (1 + r_v0 a)/2 (1 + r_v1 b)/2 (1 - c)/2 (base), (1 + c)/2 (apex),
//            in the pyramid's collapsed coordinates (a, b, c)
//   tet      barycentric
// Values N[v] and gradients dN[v][k] = d N_v / d xi_k at the collapsed point
// (a, b, c).
void shape_grad(int type, double a, double b, double c, double* N, double (*dN)[3]) {
  double xi[3];
  uncollapse(type, a, b, c, xi);
  switch (type) {
    case dgk::HEX:
      for (int v = 0; v < 8; ++v) {
        const double* r = kRefVerts[0][v];
        double f[3];
        for (int d = 0; d < 3; ++d) f[d] = 0.5 * (1.0 + r[d] * xi[d]);
        N[v] = f[0] * f[1] * f[2];
        dN[v][0] = 0.5 * r[0] * f[1] * f[2];
        dN[v][1] = 0.5 * r[1] * f[0] * f[2];
        dN[v][2] = 0.5 * r[2] * f[0] * f[1];
      }
      break;
    case dgk::PRISM: {
      const double lam[3] = {-0.5 * (xi[0] + xi[1]), 0.5 * (1.0 + xi[0]), 0.5 * (1.0 + xi[1])};
      const double dl[3][2] = {{-0.5, -0.5}, {0.5, 0.0}, {0.0, 0.5}};
      const double zl = 0.5 * (1.0 - xi[2]), zu = 0.5 * (1.0 + xi[2]);
      for (int i = 0; i < 3; ++i) {
        N[i] = lam[i] * zl;
        N[i + 3] = lam[i] * zu;
        dN[i][0] = dl[i][0] * zl;
        dN[i][1] = dl[i][1] * zl;
        dN[i][2] = -0.5 * lam[i];
        dN[i + 3][0] = dl[i][0] * zu;
        dN[i + 3][1] = dl[i][1] * zu;
        dN[i + 3][2] = 0.5 * lam[i];
      }
      break;
    }
    case dgk::TET: {
      N[0] = -0.5 * (1.0 + xi[0] + xi[1] + xi[2]);
      N[1] = 0.5 * (1.0 + xi[0]);
      N[2] = 0.5 * (1.0 + xi[1]);
      N[3] = 0.5 * (1.0 + xi[2]);
      const double g[4][3] = {{-0.5, -0.5, -0.5}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
      for (int v = 0; v < 4; ++v)
        for (int k = 0; k < 3; ++k) dN[v][k] = g[v][k];
      break;
    }
    case dgk::PYR: {
      double cm[3][3];  // d(a,b,c)_l / d xi_k
      collapse_metric(dgk::PYR, a, b, c, cm);
      for (int v = 0; v < 5; ++v) {
        double g[3];
        if (v < 4) {
          const double* r = kRefVerts[2][v];
          double fa = 0.5 * (1.0 + r[0] * a), fb = 0.5 * (1.0 + r[1] * b), fc = 0.5 * (1.0 - c);
          N[v] = fa * fb * fc;
          g[0] = 0.5 * r[0] * fb * fc;
          g[1] = 0.5 * r[1] * fa * fc;
          g[2] = -0.5 * fa * fb;
        } else {
          N[v] = 0.5 * (1.0 + c);
          g[0] = g[1] = 0.0;
          g[2] = 0.5;
        }
        for (int k = 0; k < 3; ++k) dN[v][k] = g[0] * cm[0][k] + g[1] * cm[1][k] + g[2] * cm[2][k];
      }
      break;
    }
  }
}

// dx/dxi (F[d][k]) and x - X_0 at the collapsed point from the element's
// vertex positions relative to its first vertex (Xrel [nv][3]).
void element_map(int type, const double* Xrel, double a, double b, double c, double F[3][3], double* xrel) {
  double N[8], dN[8][3];
  shape_grad(type, a, b, c, N, dN);
  for (int d = 0; d < 3; ++d) {
    xrel[d] = 0.0;
    for (int k = 0; k < 3; ++k) F[d][k] = 0.0;
  }
  for (int v = 0; v < kNumVerts[type]; ++v)
    for (int d = 0; d < 3; ++d) {
      xrel[d] += N[v] * Xrel[3 * v + d];
      for (int k = 0; k < 3; ++k) F[d][k] += Xrel[3 * v + d] * dN[v][k];
    }
}

// Generalized Vandermonde matrix V[q][mode] on the collapsed GL grid.
std::vector<double> vandermonde(int type, int N, const double* x) {
  const int n = N + 1, nQ = n * n * n, nM = n_modes(type, N);
  std::vector<double> V((size_t)nQ * nM);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        int q = (i * n + j) * n + k, mode = 0;
        for (int p = 0; p < n; ++p)
          for (int qq = 0; qq < q_count(type, N, p); ++qq)
            for (int r = 0; r < r_count(type, N, p, qq); ++r, ++mode)
              V[(size_t)q * nM + mode] = factor_A(type, p, x[i]) * factor_B(type, p, qq, x[j]) * factor_C(type, p, qq, r, x[k]);
      }
  return V;
}

// Inverse of a symmetric positive definite matrix (row-major, n x n) by a
// Cholesky factorisation A = L L^T and two triangular solves per column.
bool spd_inverse(int n, const double* A, double* Ainv) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = s / ljj;
    }
  }
  std::vector<double> y(n);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {  // L y = e_col
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
      y[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * Ainv[(size_t)k * n + col];
      Ainv[(size_t)i * n + col] = s / L[(size_t)i * n + i];
    }
  }
  return true;
}

// Pointwise geometry block of one curved element (layout of HostMesh::cpool).
// Returns false if det(dx/dxi) changes sign or vanishes at a volume point, or
// the mass matrix is not positive definite.
bool curved_block(const TypeTab& T, const std::vector<double>& dpool, const double* x, const double* Xrel,
                  const double* V, double* out) {
  const int n = T.n, nQ = T.nQ, nM = T.nM, type = T.type;
  const double* wq = dpool.data() + T.W;
  int sign = 0;
  std::vector<double> wJ(nQ);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const int q = (i * n + j) * n + k;
        double F[3][3], xr[3];
        element_map(type, Xrel, x[i], x[j], x[k], F, xr);
        const double det = det3(F);
        const int sg = det > 0 ? 1 : (det < 0 ? -1 : 0);
        if (sg == 0 || (sign != 0 && sg != sign)) return false;
        sign = sg;
        const double J = std::fabs(det);
        double Fi[3][3];
        inv3(F, Fi);
        double cm[3][3];
        collapse_metric(type, x[i], x[j], x[k], cm);
        for (int l = 0; l < 3; ++l)
          for (int d = 0; d < 3; ++d) {
            double m = 0.0;
            for (int kk = 0; kk < 3; ++kk) m += cm[l][kk] * J * Fi[kk][d];
            out[(size_t)(l * 3 + d) * nQ + q] = wq[q] * m;
          }
        out[(size_t)9 * nQ + q] = J;
        out[(size_t)10 * nQ + q] = 1.0 / J;
        wJ[q] = wq[q] * J;
      }
  if (type == dgk::PRISM || type == dgk::PYR) {
    std::vector<double> Me((size_t)nM * nM, 0.0);
    for (int q = 0; q < nQ; ++q) {
      const double* vq = V + (size_t)q * nM;
      for (int a = 0; a < nM; ++a) {
        const double s = wJ[q] * vq[a];
        for (int b2 = 0; b2 <= a; ++b2) Me[(size_t)a * nM + b2] += s * vq[b2];
      }
    }
    for (int a = 0; a < nM; ++a)
      for (int b2 = a + 1; b2 < nM; ++b2) Me[(size_t)a * nM + b2] = Me[(size_t)b2 * nM + a];
    if (!spd_inverse(nM, Me.data(), out + (size_t)11 * nQ)) return false;
  }
  return true;
}

// Adjugate of a 3x3 matrix (transpose of the cofactor matrix): adj(A) A = det(A) I.
void adj3(const double A[3][3], double R[3][3]) {
  R[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  R[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
  R[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  R[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  R[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  R[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
  R[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  R[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
  R[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
}

// Coefficients of det(A + t B) = d0 + d1 t + d2 t^2 + d3 t^3 and of
// adj(A + t B) = adj(A) + t D + t^2 adj(B) (adj is quadratic: D = adj(A + B)
// - adj(A) - adj(B)).
void det_adj_poly(const double A[3][3], const double B[3][3], double d[4], double adj[3][3][3]) {
  double AB[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) AB[i][j] = A[i][j] + B[i][j];
  double aA[3][3], aB[3][3], aAB[3][3];
  adj3(A, aA);
  adj3(B, aB);
  adj3(AB, aAB);
  d[0] = det3(A);
  d[3] = det3(B);
  d[1] = 0.0;
  d[2] = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      d[1] += aA[i][j] * B[j][i];     // tr(adj(A) B)
      d[2] += A[i][j] * aB[j][i];     // tr(A adj(B))
      adj[0][i][j] = aA[i][j];
      adj[1][i][j] = aAB[i][j] - aA[i][j] - aB[i][j];
      adj[2][i][j] = aB[i][j];
    }
}

int64_t curved_block_size(const TypeTab& T) {
  return 11 * (int64_t)T.nQ + ((T.type == dgk::PRISM || T.type == dgk::PYR) ? (int64_t)T.nM * T.nM : 0);
}

}  // namespace

int build_mesh(const MeshInput& in, HostMesh* out, std::string* err) {
  HostMesh& M = *out;
  if (in.N < 1 || in.N > dgk::kMaxN) { *err = "N out of range"; return -1; }
  if (!in.xyz || !in.type || !in.off || !in.verts || !in.period) { *err = "null pointer in mesh description"; return -1; }
  if (in.n_elems <= 0 || in.n_vertices <= 0) { *err = "empty mesh"; return -1; }
  for (int d = 0; d < 3; ++d)
    if (!(in.period[d] > 0)) { *err = "period must be positive"; return -1; }
  const int N = in.N, n = N + 1, n2 = n * n;
  M.N = N;
  M.n = n;
  M.n_elems = in.n_elems;
  M.x1d.resize(n);
  M.w1d.resize(n);
  gauss_legendre(n, M.x1d.data(), M.w1d.data());
  const int64_t E = in.n_elems;
  int tab_of_type[4] = {-1, -1, -1, -1};
  for (int64_t e = 0; e < E; ++e) {
    int t = in.type[e];
    if (t < 0 || t > 3) { *err = "bad element type"; return -1; }
    if (in.off[e + 1] - in.off[e] != kNumVerts[t]) { *err = "wrong vertex count for element type"; return -2; }
    for (int64_t k = in.off[e]; k < in.off[e + 1]; ++k)
      if (in.verts[k] < 0 || in.verts[k] >= in.n_vertices) { *err = "vertex index out of range"; return -1; }
    if (tab_of_type[t] < 0) {
      int r = M.tables.add(t, N, err);
      if (r < 0) return r;
      tab_of_type[t] = r;
    }
    M.type_count[t]++;
  }

  // ---- affine geometry (caller order first)
  std::vector<dgk::ElemGeo> geo(E);
  std::vector<std::array<double, 12>> affine(E);  // X0, A columns
  std::vector<std::array<double, 3>> centroid(E);
  std::vector<char> curved(E, 0);
  if (in.geometry != 0 && in.geometry != 1) { *err = "unknown geometry kind"; return -1; }
  for (int64_t e = 0; e < E; ++e) {
    int t = in.type[e];
    const int64_t* V = in.verts + in.off[e];
    const double* X0 = in.xyz + 3 * V[0];
    double A[3][3];  // A[d][k]: column k = image of reference axis k
    for (int k = 0; k < 3; ++k) {
      const double* Xk = in.xyz + 3 * V[kAxisVert[t][k]];
      for (int d = 0; d < 3; ++d) A[d][k] = Xk[d] - X0[d];
    }
    double scale = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) scale = std::max(scale, std::fabs(A[d][k]));
    bool is_affine = true;
    for (int m = 0; m < kNumVerts[t]; ++m) {
      const double* Xm = in.xyz + 3 * V[m];
      for (int d = 0; d < 3; ++d) {
        double pred = X0[d];
        for (int k = 0; k < 3; ++k) pred += A[d][k] * 0.5 * (kRefVerts[t][m][k] + 1.0);
        if (std::fabs(pred - Xm[d]) > 1e-10 * scale) is_affine = false;
      }
    }
    {
      double c[3] = {0, 0, 0};
      for (int m = 0; m < kNumVerts[t]; ++m)
        for (int d = 0; d < 3; ++d) c[d] += in.xyz[3 * V[m] + d] / kNumVerts[t];
      for (int d = 0; d < 3; ++d) centroid[e][d] = c[d];
    }
    if (!is_affine || (in.force_curved && t != dgk::TET)) {
      if (in.geometry != 1 && !in.force_curved) { *err = "element is not an affine image of its reference element"; return -2; }
      curved[e] = 1;   // pointwise geometry below; the affine record stays zero
      std::memset(&geo[e], 0, sizeof(geo[e]));
      for (int d = 0; d < 12; ++d) affine[e][d] = 0.0;
      continue;
    }
    double det = det3(A);
    if (!(std::fabs(det) > 1e-300)) { *err = "degenerate element"; return -2; }
    double J = std::fabs(det) / 8.0;
    double Ai[3][3];
    inv3(A, Ai);  // d(xi+1)/2 / dx
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) geo[e].Jg[k * 3 + d] = J * 2.0 * Ai[k][d];
    geo[e].invJ = 1.0 / J;
    for (int d = 0; d < 3; ++d) {
      affine[e][d] = X0[d];
      for (int k = 0; k < 3; ++k) affine[e][3 + 3 * k + d] = A[d][k];
    }
  }

  // ---- Hilbert order of the centroids (ties: caller index)
  {
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) { lo[d] = 1e300; hi[d] = -1e300; }
    for (int64_t e = 0; e < E; ++e)
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], centroid[e][d]); hi[d] = std::max(hi[d], centroid[e][d]); }
    const int bits = 21;
    const double cells = (double)((1u << bits) - 1);
    std::vector<std::pair<uint64_t, int64_t>> keys(E);
    for (int64_t e = 0; e < E; ++e) {
      uint32_t q[3];
      for (int d = 0; d < 3; ++d) {
        double span = hi[d] - lo[d];
        double u = span > 0 ? (centroid[e][d] - lo[d]) / span : 0.0;
        q[d] = (uint32_t)std::llround(u * cells);
      }
      keys[e] = {hilbert_key3(q[0], q[1], q[2], bits), e};
    }
    std::sort(keys.begin(), keys.end());
    M.elem_of_slot.resize(E);
    M.slot_of_elem.resize(E);
    for (int64_t s = 0; s < E; ++s) {
      M.elem_of_slot[s] = keys[s].second;
      M.slot_of_elem[keys[s].second] = s;
    }
  }

  // ---- per-slot records and state offsets
  M.slot_tab.resize(E);
  M.slot_type.resize(E);
  M.slot_qoff.resize(E);
  M.slot_hoff.resize(E);
  M.slot_geo.resize(E);
  M.elem_qoff.resize(E);
  {
    int64_t q = 0;
    for (int64_t e = 0; e < E; ++e) { M.elem_qoff[e] = q; q += 5 * (int64_t)n_modes(in.type[e], N); }
    M.elem_voff.resize(E);
    for (int64_t e = 0; e < E; ++e) M.elem_voff[e] = e * 5 * (int64_t)n * n * n;
    M.inst_elem_off = {0, E};
    M.inst_dof_off = {0, q};
    M.n_dof = q;
    int64_t qs = 0, hs = 0;
    for (int64_t s = 0; s < E; ++s) {
      int64_t e = M.elem_of_slot[s];
      int t = in.type[e];
      M.slot_tab[s] = tab_of_type[t];
      M.slot_type[s] = (int8_t)t;
      M.slot_qoff[s] = qs;
      M.slot_hoff[s] = hs;
      M.slot_geo[s] = geo[e];
      qs += 5 * (int64_t)n_modes(t, N);
      hs += 5 * (int64_t)n * n * n;
    }
    M.h_total = hs;
  }
  for (int t = 0; t < 4; ++t) M.type_slots[t].clear();
  M.slot_ghost.assign(E, 0);
  M.n_ghost = 0;
  for (int64_t e = 0; e < E; ++e) {
    if (in.ghost && in.ghost[e]) {
      M.slot_ghost[M.slot_of_elem[e]] = 1;
      M.n_ghost++;
      continue;
    }
    M.type_slots[(int)in.type[e]].push_back(M.slot_of_elem[e]);
  }
  if (M.n_ghost == E) { *err = "a partition mesh needs at least one owned element"; return -1; }

  // ---- curved elements: pointwise metric, J, 1/J and (prism, pyramid) the
  // dense inverse mass matrix of Algorithm 1, per slot
  M.slot_coff.assign(E, -1);
  M.cpool.clear();
  M.n_curved = 0;
  {
    int64_t csize = 0;
    for (int64_t s = 0; s < E; ++s)
      if (curved[M.elem_of_slot[s]]) {
        M.slot_coff[s] = csize;
        csize += curved_block_size(M.tables.tabs[M.slot_tab[s]]);
        M.n_curved++;
      }
    if (M.n_curved) {
      M.cpool.assign((size_t)csize, 0.0);
      std::vector<double> Vt[4];
      for (int t = 0; t < 4; ++t)
        if (tab_of_type[t] >= 0 && (t == dgk::PRISM || t == dgk::PYR)) Vt[t] = vandermonde(t, N, M.x1d.data());
      std::vector<int64_t> todo;
      for (int64_t s = 0; s < E; ++s)
        if (M.slot_coff[s] >= 0) todo.push_back(s);
      std::atomic<int64_t> next(0);
      std::atomic<int> bad(0);
      auto work = [&]() {
        std::vector<double> Xrel(24);
        for (;;) {
          const int64_t i = next.fetch_add(1);
          if (i >= (int64_t)todo.size() || bad.load()) break;
          const int64_t s = todo[i], e = M.elem_of_slot[s];
          const int t = in.type[e];
          const int64_t* V = in.verts + in.off[e];
          for (int v = 0; v < kNumVerts[t]; ++v)
            for (int d = 0; d < 3; ++d) Xrel[3 * v + d] = in.xyz[3 * V[v] + d] - in.xyz[3 * V[0] + d];
          const TypeTab& T = M.tables.tabs[M.slot_tab[s]];
          if (!curved_block(T, M.tables.dpool, M.x1d.data(), Xrel.data(), Vt[t].data(), M.cpool.data() + M.slot_coff[s]))
            bad.store(1);
        }
      };
      unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
      nth = (unsigned)std::min<int64_t>(nth, (int64_t)todo.size());
      std::vector<std::thread> pool;
      for (unsigned i = 1; i < nth; ++i) pool.emplace_back(work);
      work();
      for (auto& th : pool) th.join();
      if (bad.load()) { *err = "curved element is inverted or degenerate at a quadrature point"; return -2; }
    }
  }

  // ---- canonical (periodically reduced) vertex ids
  std::vector<int64_t> canon(in.n_vertices);
  {
    std::unordered_map<Key3, int64_t, Key3Hash> ids;
    ids.reserve((size_t)in.n_vertices * 2);
    for (int64_t v = 0; v < in.n_vertices; ++v) {
      Key3 k = reduce(in.xyz + 3 * v, in.period);
      auto it = ids.find(k);
      if (it == ids.end()) it = ids.emplace(k, (int64_t)ids.size()).first;
      canon[v] = it->second;
    }
  }

  // ---- face matching
  struct Side { int64_t e; int lf; };
  std::map<FaceKey, std::vector<Side>> table;
  for (int64_t e = 0; e < E; ++e) {
    int t = in.type[e];
    const int64_t* V = in.verts + in.off[e];
    for (int lf = 0; lf < kNumFaces[t]; ++lf) {
      FaceKey fk;
      fk.nv = kFaceNV[t][lf];
      double c[3] = {0, 0, 0};
      for (int i = 0; i < fk.nv; ++i) {
        const double* P = in.xyz + 3 * V[kFaceVerts[t][lf][i]];
        fk.v[i] = reduce(P, in.period);
        for (int d = 0; d < 3; ++d) c[d] += P[d] / fk.nv;
      }
      fk.c = reduce(c, in.period);
      for (int i = 1; i < fk.nv; ++i)      // insertion sort of the (at most 4) vertex keys
        for (int j = i; j > 0 && fk.v[j] < fk.v[j - 1]; --j) std::swap(fk.v[j], fk.v[j - 1]);
      table[fk].push_back({e, lf});
    }
  }
  struct FaceTmp { int64_t e0, e1; int l0, l1; };
  std::vector<FaceTmp> ftmp;
  ftmp.reserve(table.size());
  auto is_ghost = [&](int64_t e) { return in.ghost != nullptr && in.ghost[e] != 0; };
  for (auto& kv : table) {
    if (kv.second.size() == 1 && is_ghost(kv.second[0].e)) continue;     // a ghost's face towards other parts
    if (kv.second.size() != 2) { *err = "a face does not have exactly one partner (mesh must be conforming and periodic)"; return -2; }
    Side a = kv.second[0], b = kv.second[1];
    if (is_ghost(a.e) && is_ghost(b.e)) continue;                         // between two ghosts: not needed
    if (std::tie(b.e, b.lf) < std::tie(a.e, a.lf)) std::swap(a, b);  // owner: smaller caller index
    ftmp.push_back({a.e, b.e, a.lf, b.lf});
  }
  // face-kernel order: by owner slot (Hilbert locality)
  std::sort(ftmp.begin(), ftmp.end(), [&](const FaceTmp& x, const FaceTmp& y) {
    int64_t sx = M.slot_of_elem[x.e0], sy = M.slot_of_elem[y.e0];
    if (sx != sy) return sx < sy;
    return x.l0 < y.l0;
  });
  const int64_t F = (int64_t)ftmp.size();
  if (F >= ((int64_t)1 << 31)) { *err = "too many faces for 32-bit face-block indices"; return -7; }
  M.n_faces = F;
  M.faces.resize(F);
  M.face_e0.resize(F);
  M.face_e1.resize(F);
  M.face_l0.resize(F);
  M.face_l1.resize(F);
  for (int64_t f = 0; f < F; ++f) {
    M.face_e0[f] = ftmp[f].e0;
    M.face_e1[f] = ftmp[f].e1;
    M.face_l0[f] = (int8_t)ftmp[f].l0;
    M.face_l1[f] = (int8_t)ftmp[f].l1;
  }
  M.slot_ftoff.assign((size_t)E * 6, -1);
  M.slot_fnrm.assign((size_t)E * 18, 0.0);
  M.perms.clear();
  M.dense.clear();
  M.fgeo.clear();
  M.n_curved_faces = 0;
  std::map<std::vector<int16_t>, int> perm_ids;
  std::map<std::vector<int>, int> dense_ids;  // key: (nb type, nb lf, sigma, owner tri)
  const double* x = M.x1d.data();
  for (int64_t f = 0; f < F; ++f) {
    const FaceTmp& ft = ftmp[f];
    int t0 = in.type[ft.e0], t1 = in.type[ft.e1];
    int nv = kFaceNV[t0][ft.l0];
    if (kFaceNV[t1][ft.l1] != nv) { *err = "matched faces of different shapes"; return -2; }
    const int64_t* V0 = in.verts + in.off[ft.e0];
    const int64_t* V1 = in.verts + in.off[ft.e1];
    int64_t c0[4], c1[4];
    for (int i = 0; i < nv; ++i) {
      c0[i] = canon[V0[kFaceVerts[t0][ft.l0][i]]];
      c1[i] = canon[V1[kFaceVerts[t1][ft.l1][i]]];
    }
    for (int i = 0; i < nv; ++i)
      for (int j = i + 1; j < nv; ++j)
        if (c0[i] == c0[j]) { *err = "face vertices coincide modulo the period (box too small)"; return -2; }
    int sigma[4];  // neighbour slot m <-> owner slot sigma[m]
    for (int m = 0; m < nv; ++m) {
      sigma[m] = -1;
      for (int i = 0; i < nv; ++i)
        if (c1[m] == c0[i]) sigma[m] = i;
      if (sigma[m] < 0) { *err = "face vertex correspondence failed"; return -2; }
    }
    dgk::FaceRec& R = M.faces[f];
    R.toff = f * 2 * 5 * (int64_t)n2;
    R.owner_tab = tab_of_type[t0];
    R.owner_lf = ft.l0;
    R.cgeo = -1;
    if (curved[ft.e0]) {
      // curved owner: per face point p = ia + n ib (the owner's face grid)
      // the area vector (dx/dxi t_s) x (dx/dxi t_t), t_s, t_t the reference
      // tangents of the face parameters, oriented outward: sign(det dx/dxi)
      // times the orientation of t_s x t_t against the reference outward side
      const int* fv = kFaceVerts[t0][ft.l0];
      const double* c0r = kRefVerts[t0][fv[0]];
      const double* c1r = kRefVerts[t0][fv[1]];
      const double* c2r = kRefVerts[t0][fv[2]];
      double tsr[3], ttr[3], nref[3], out_ref[3] = {0, 0, 0}, cen[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) {
        tsr[k] = 0.5 * (c1r[k] - c0r[k]);
        ttr[k] = 0.5 * (c2r[k] - c0r[k]);
      }
      cross(tsr, ttr, nref);
      for (int v = 0; v < kNumVerts[t0]; ++v)
        for (int k = 0; k < 3; ++k) cen[k] += kRefVerts[t0][v][k] / kNumVerts[t0];
      for (int i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) out_ref[k] += kRefVerts[t0][fv[i]][k] / nv - cen[k] / nv;
      const double orient = (nref[0] * out_ref[0] + nref[1] * out_ref[1] + nref[2] * out_ref[2]) > 0 ? 1.0 : -1.0;
      double Xrel[24];
      for (int v = 0; v < kNumVerts[t0]; ++v)
        for (int d = 0; d < 3; ++d) Xrel[3 * v + d] = in.xyz[3 * V0[v] + d] - in.xyz[3 * V0[0] + d];
      const TypeTab& T0 = M.tables.tabs[tab_of_type[t0]];
      const FaceDesc fd = T0.faces[ft.l0];
      const double* fw = M.tables.dpool.data() + T0.fw + (size_t)ft.l0 * n2;
      const size_t base = M.fgeo.size();
      M.fgeo.resize(base + (size_t)4 * n2);
      for (int ib = 0; ib < n; ++ib)
        for (int ia = 0; ia < n; ++ia) {
          const int p = ia + n * ib;
          double abc[3];
          abc[fd.fixed] = fd.end ? 1.0 : -1.0;
          abc[fd.alpha] = x[ia];
          abc[fd.beta] = x[ib];
          double Fp[3][3], xr[3], ts[3], tt[3], cr[3];
          element_map(t0, Xrel, abc[0], abc[1], abc[2], Fp, xr);
          for (int d = 0; d < 3; ++d) {
            ts[d] = Fp[d][0] * tsr[0] + Fp[d][1] * tsr[1] + Fp[d][2] * tsr[2];
            tt[d] = Fp[d][0] * ttr[0] + Fp[d][1] * ttr[1] + Fp[d][2] * ttr[2];
          }
          cross(ts, tt, cr);
          const double S = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
          const double sg = (det3(Fp) > 0 ? 1.0 : -1.0) * orient;
          for (int d = 0; d < 3; ++d) M.fgeo[base + (size_t)d * n2 + p] = sg * cr[d] / S;
          M.fgeo[base + (size_t)3 * n2 + p] = fw[p] * S;
          if (p == 0) {
            for (int d = 0; d < 3; ++d) R.nrm[d] = sg * cr[d] / S;
          }
        }
      R.S = 0.0;
      if (base >= ((size_t)1 << 31)) { *err = "too many curved faces for 32-bit face-geometry offsets"; return -7; }
      R.cgeo = (int)base;
      M.n_curved_faces++;
    } else {
      // owner geometry: normal and area scale
      const auto& af = affine[ft.e0];
      const int* fv = kFaceVerts[t0][ft.l0];
      double ts[3], tt[3];
      for (int d = 0; d < 3; ++d) {
        ts[d] = tt[d] = 0.0;
        for (int k = 0; k < 3; ++k) {
          double A = af[3 + 3 * k + d];
          ts[d] += 0.25 * A * (kRefVerts[t0][fv[1]][k] - kRefVerts[t0][fv[0]][k]);
          tt[d] += 0.25 * A * (kRefVerts[t0][fv[2]][k] - kRefVerts[t0][fv[0]][k]);
        }
      }
      double cr[3];
      cross(ts, tt, cr);
      double S = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      double fc[3] = {0, 0, 0};
      for (int i = 0; i < nv; ++i)
        for (int d = 0; d < 3; ++d) fc[d] += in.xyz[3 * V0[fv[i]] + d] / nv;
      double dot = 0.0;
      for (int d = 0; d < 3; ++d) dot += cr[d] * (fc[d] - centroid[ft.e0][d]);
      double sgn = dot >= 0 ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) R.nrm[d] = sgn * cr[d] / S;
      R.S = S;
    }
    // neighbour map
    if (nv == 4) {
      // dihedral map of the Gauss-Legendre tensor grid
      static const int kap[4][2] = {{-1, -1}, {1, -1}, {-1, 1}, {1, 1}};
      int s0 = kap[sigma[0]][0], t0c = kap[sigma[0]][1];
      int ax[2][2];  // for nb axis a: (owner axis, flip)
      for (int a = 0; a < 2; ++a) {
        int m = a == 0 ? 1 : 2;
        int ds = kap[sigma[m]][0] - s0, dt = kap[sigma[m]][1] - t0c;
        if (ds != 0 && dt == 0) { ax[a][0] = 0; ax[a][1] = ds < 0; }
        else if (dt != 0 && ds == 0) { ax[a][0] = 1; ax[a][1] = dt < 0; }
        else { *err = "quadrilateral face correspondence is not a symmetry"; return -2; }
      }
      if (ax[0][0] == ax[1][0]) { *err = "quadrilateral face correspondence is degenerate"; return -2; }
      std::vector<int16_t> perm(2 * n2);
      for (int ib = 0; ib < n; ++ib)
        for (int ia = 0; ia < n; ++ia) {
          int own[2] = {ia, ib};
          int j[2];
          for (int a = 0; a < 2; ++a) {
            int v = own[ax[a][0]];
            j[a] = ax[a][1] ? n - 1 - v : v;
          }
          int p = ia + n * ib, q = j[0] + n * j[1];
          perm[p] = (int16_t)q;
          perm[n2 + q] = (int16_t)p;
        }
      auto it = perm_ids.find(perm);
      if (it == perm_ids.end()) {
        it = perm_ids.emplace(perm, (int)M.perms.size()).first;
        M.perms.insert(M.perms.end(), perm.begin(), perm.end());
      }
      R.map = it->second;
    } else if (sigma[2] == 2) {
      // collapse vertex shared: the collapsed grid maps onto itself (alpha -> +-alpha)
      bool flip = sigma[0] != 0;
      std::vector<int16_t> perm(2 * n2);
      for (int ib = 0; ib < n; ++ib)
        for (int ia = 0; ia < n; ++ia) {
          int p = ia + n * ib, q = (flip ? n - 1 - ia : ia) + n * ib;
          perm[p] = (int16_t)q;
          perm[n2 + q] = (int16_t)p;
        }
      auto it = perm_ids.find(perm);
      if (it == perm_ids.end()) {
        it = perm_ids.emplace(perm, (int)M.perms.size()).first;
        M.perms.insert(M.perms.end(), perm.begin(), perm.end());
      }
      R.map = it->second;
    } else {
      // general triangle correspondence: interpolate the neighbour's face
      // values (tensor Lagrange in its collapsed face coordinates) at the
      // owner's points, located by barycentric coordinates.
      std::vector<int> key = {sigma[0], sigma[1], sigma[2]};
      auto it = dense_ids.find(key);
      if (it == dense_ids.end()) {
        it = dense_ids.emplace(key, (int)M.dense.size()).first;
        std::vector<double> la(n), lb(n);
        size_t base = M.dense.size();
        M.dense.resize(base + (size_t)n2 * n2);
        for (int ib = 0; ib < n; ++ib)
          for (int ia = 0; ia < n; ++ia) {
            double al = x[ia], be = x[ib];
            double lam[3];
            lam[1] = 0.25 * (1 + al) * (1 - be);
            lam[2] = 0.5 * (1 + be);
            lam[0] = 1.0 - lam[1] - lam[2];
            double lp[3];
            for (int m = 0; m < 3; ++m) lp[m] = lam[sigma[m]];
            double alp = 2.0 * lp[1] / (1.0 - lp[2]) - 1.0;
            double bep = 2.0 * lp[2] - 1.0;
            lagrange_values(x, n, alp, la.data());
            lagrange_values(x, n, bep, lb.data());
            int p = ia + n * ib;
            for (int jb = 0; jb < n; ++jb)
              for (int ja = 0; ja < n; ++ja) M.dense[base + (size_t)p * n2 + ja + n * jb] = la[ja] * lb[jb];
          }
      }
      R.map = -1 - it->second;
    }
    int64_t s0 = M.slot_of_elem[ft.e0], s1 = M.slot_of_elem[ft.e1];
    M.slot_ftoff[(size_t)s0 * 6 + ft.l0] = R.toff;
    M.slot_ftoff[(size_t)s1 * 6 + ft.l1] = R.toff + 5 * (int64_t)n2;
    for (int d = 0; d < 3; ++d) {
      M.slot_fnrm[((size_t)s0 * 6 + ft.l0) * 3 + d] = R.nrm[d];
      M.slot_fnrm[((size_t)s1 * 6 + ft.l1) * 3 + d] = -R.nrm[d];
    }
  }
  M.n_perm = (int)perm_ids.size();
  M.n_dense = (int)dense_ids.size();
  M.t_total = F * 2 * 5 * (int64_t)n2;
  // per-side normals at the side's own points (curved geometry requested):
  // the owner's normal at its points; the neighbour's is the negated owner
  // normal at the matching owner point (a permutation), or the constant
  // negated normal of a planar triangle (interpolating maps)
  M.snrm.clear();
  if (in.geometry == 1) {
    M.snrm.assign((size_t)(3 * (M.t_total / 5)), 0.0);
    for (int64_t f = 0; f < F; ++f) {
      const dgk::FaceRec& R = M.faces[f];
      double* N0 = M.snrm.data() + 3 * (R.toff / 5);
      double* N1 = M.snrm.data() + 3 * ((R.toff + 5 * (int64_t)n2) / 5);
      for (int p = 0; p < n2; ++p)
        for (int d = 0; d < 3; ++d)
          N0[d * n2 + p] = R.cgeo >= 0 ? M.fgeo[(size_t)R.cgeo + (size_t)d * n2 + p] : R.nrm[d];
      for (int p = 0; p < n2; ++p) {
        const int q = R.map >= 0 ? M.perms[(size_t)R.map + p] : p;
        for (int d = 0; d < 3; ++d) N1[d * n2 + q] = R.map >= 0 ? -N0[d * n2 + p] : -N0[d * n2];
      }
    }
  }
  for (int64_t s = 0; s < E; ++s) {
    if (M.slot_ghost[s]) continue;     // a ghost's faces towards other parts are not in this mesh
    for (int lf = 0; lf < kNumFaces[M.slot_type[s]]; ++lf)
      if (M.slot_ftoff[(size_t)s * 6 + lf] < 0) { *err = "internal: unassigned face"; return -1; }
  }
  // face blocks of up to 32 faces (uniform n)
  M.face_blocks.clear();
  for (int64_t f = 0; f < F; f += 32) {
    dgk::FaceBlock b;
    b.first = (int)f;
    b.count = (int)std::min<int64_t>(32, F - f);
    b.n = n;
    b.pad = 0;
    M.face_blocks.push_back(b);
  }

  // ---- physical quadrature points (caller order)
  M.quad_xyz.resize((size_t)E * n * n * n * 3);
  for (int64_t e = 0; e < E; ++e) {
    int t = in.type[e];
    const auto& af = affine[e];
    if (curved[e]) {
      const int64_t* V = in.verts + in.off[e];
      const double* X0 = in.xyz + 3 * V[0];
      double Xrel[24];
      for (int v = 0; v < kNumVerts[t]; ++v)
        for (int d = 0; d < 3; ++d) Xrel[3 * v + d] = in.xyz[3 * V[v] + d] - X0[d];
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) {
            double Fq[3][3], xr[3];
            element_map(t, Xrel, x[i], x[j], x[k], Fq, xr);
            size_t q = (size_t)e * n * n * n + (size_t)(i * n + j) * n + k;
            for (int d = 0; d < 3; ++d) M.quad_xyz[3 * q + d] = X0[d] + xr[d];
          }
      continue;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          double xi[3];
          uncollapse(t, x[i], x[j], x[k], xi);
          size_t q = (size_t)e * n * n * n + (size_t)(i * n + j) * n + k;
          for (int d = 0; d < 3; ++d) {
            double v = af[d];
            for (int kk = 0; kk < 3; ++kk) v += af[3 + 3 * kk + d] * 0.5 * (xi[kk] + 1.0);
            M.quad_xyz[3 * q + d] = v;
          }
        }
  }
  return 0;
}

int partition_plan(const HostMesh& M, int nparts, const double* type_weight, std::vector<int64_t>* part_of_elem,
                   std::vector<int64_t>* halo_off, std::vector<int64_t>* halo_elems, std::string* err) {
  const int64_t E = M.n_elems;
  if (nparts < 1 || nparts > E) { *err = "nparts must be between 1 and the number of elements"; return -1; }
  if (M.inst_elem_off.size() != 2) { *err = "partition plans are for single meshes"; return -7; }
  // equal-weight cuts of the prefix sum along the Hilbert order
  std::vector<double> w(E);
  double total = 0.0;
  for (int64_t s = 0; s < E; ++s) {
    const double ws = type_weight ? type_weight[(int)M.slot_type[s]] : 1.0;
    if (!(ws > 0.0) || !std::isfinite(ws)) { *err = "element weights must be finite and positive"; return -1; }
    w[s] = ws;
    total += ws;
  }
  part_of_elem->assign(E, -1);
  {
    double acc = 0.0;
    int p = 0;
    for (int64_t s = 0; s < E; ++s) {
      // part p takes the slots whose weight midpoint lies in [p W / P, (p+1) W / P)
      const double mid = acc + 0.5 * w[s];
      while (p + 1 < nparts && mid >= total * (double)(p + 1) / (double)nparts) ++p;
      (*part_of_elem)[M.elem_of_slot[s]] = p;
      acc += w[s];
    }
  }
  // faces -> the two slots: trace offsets are f (2 sides) (5 n^2), side 1 at + 5 n^2
  const int64_t side = 5 * (int64_t)M.n * M.n;
  std::vector<int64_t> face_slot(2 * (size_t)M.n_faces, -1);
  for (int64_t s = 0; s < E; ++s)
    for (int lf = 0; lf < 6; ++lf) {
      const int64_t t = M.slot_ftoff[(size_t)s * 6 + lf];
      if (t < 0) continue;
      face_slot[(size_t)(t / side)] = s;   // index 2 f + side
    }
  std::vector<std::vector<int64_t>> halo(nparts);
  for (int64_t f = 0; f < M.n_faces; ++f) {
    const int64_t a = face_slot[2 * f], b = face_slot[2 * f + 1];
    if (a < 0 || b < 0) { *err = "internal: face without two sides"; return -1; }
    const int64_t ea = M.elem_of_slot[a], eb = M.elem_of_slot[b];
    const int64_t pa = (*part_of_elem)[ea], pb = (*part_of_elem)[eb];
    if (pa != pb) {
      halo[pa].push_back(eb);
      halo[pb].push_back(ea);
    }
  }
  halo_off->assign(nparts + 1, 0);
  halo_elems->clear();
  for (int p = 0; p < nparts; ++p) {
    std::sort(halo[p].begin(), halo[p].end());
    halo[p].erase(std::unique(halo[p].begin(), halo[p].end()), halo[p].end());
    halo_elems->insert(halo_elems->end(), halo[p].begin(), halo[p].end());
    (*halo_off)[p + 1] = (int64_t)halo_elems->size();
  }
  return 0;
}

int build_batch(const std::vector<MeshInput>& ins, HostMesh* out, std::string* err) {
  if (ins.empty()) { *err = "empty batch"; return -1; }
  HostMesh& M = *out;
  M = HostMesh();
  int64_t e_off = 0, q_off = 0, h_off = 0, t_off = 0, v_off = 0, f_off = 0;
  M.inst_elem_off = {0};
  M.inst_dof_off = {0};
  for (size_t i = 0; i < ins.size(); ++i) {
    HostMesh Mi;
    Mi.tables = M.tables;  // (type, N) tables are shared by all instances
    int r = build_mesh(ins[i], &Mi, err);
    if (r != 0) {
      *err = "instance " + std::to_string(i) + ": " + *err;
      return r;
    }
    M.tables = std::move(Mi.tables);
    const int64_t E = Mi.n_elems;
    const int64_t p_off = (int64_t)M.perms.size(), d_off = (int64_t)M.dense.size();
    const int64_t c_off = (int64_t)M.cpool.size(), g_off = (int64_t)M.fgeo.size();
    for (int64_t s = 0; s < E; ++s) {
      M.elem_of_slot.push_back(Mi.elem_of_slot[s] + e_off);
      M.slot_tab.push_back(Mi.slot_tab[s]);
      M.slot_type.push_back(Mi.slot_type[s]);
      M.slot_qoff.push_back(Mi.slot_qoff[s] + q_off);
      M.slot_hoff.push_back(Mi.slot_hoff[s] + h_off);
      M.slot_geo.push_back(Mi.slot_geo[s]);
      M.slot_coff.push_back(Mi.slot_coff[s] >= 0 ? Mi.slot_coff[s] + c_off : -1);
      for (int lf = 0; lf < 6; ++lf) {
        int64_t t = Mi.slot_ftoff[(size_t)s * 6 + lf];
        M.slot_ftoff.push_back(t >= 0 ? t + t_off : -1);
        for (int d = 0; d < 3; ++d) M.slot_fnrm.push_back(Mi.slot_fnrm[((size_t)s * 6 + lf) * 3 + d]);
      }
    }
    for (int64_t e = 0; e < E; ++e) {
      M.slot_of_elem.push_back(Mi.slot_of_elem[e] + e_off);
      M.elem_qoff.push_back(Mi.elem_qoff[e] + q_off);
      M.elem_voff.push_back(Mi.elem_voff[e] + v_off);
    }
    M.perms.insert(M.perms.end(), Mi.perms.begin(), Mi.perms.end());
    M.dense.insert(M.dense.end(), Mi.dense.begin(), Mi.dense.end());
    M.cpool.insert(M.cpool.end(), Mi.cpool.begin(), Mi.cpool.end());
    M.fgeo.insert(M.fgeo.end(), Mi.fgeo.begin(), Mi.fgeo.end());
    if (Mi.snrm.empty() != (i == 0 ? Mi.snrm.empty() : M.snrm.empty())) {
      *err = "all instances of a batch must request the same geometry kind";
      return -1;
    }
    M.snrm.insert(M.snrm.end(), Mi.snrm.begin(), Mi.snrm.end());
    M.n_curved += Mi.n_curved;
    M.n_curved_faces += Mi.n_curved_faces;
    for (dgk::FaceRec R : Mi.faces) {
      R.toff += t_off;
      if (R.cgeo >= 0) R.cgeo += (int)g_off;
      R.map = R.map >= 0 ? (int)(R.map + p_off) : (int)(-1 - ((-1 - R.map) + d_off));
      M.faces.push_back(R);
    }
    for (dgk::FaceBlock b : Mi.face_blocks) {
      b.first += (int)f_off;
      M.face_blocks.push_back(b);
    }
    for (int t = 0; t < 4; ++t) {
      for (int64_t s : Mi.type_slots[t]) M.type_slots[t].push_back(s + e_off);
      M.type_count[t] += Mi.type_count[t];
    }
    M.quad_xyz.insert(M.quad_xyz.end(), Mi.quad_xyz.begin(), Mi.quad_xyz.end());
    M.n_perm += Mi.n_perm;
    M.n_dense += Mi.n_dense;
    M.N = std::max(M.N, Mi.N);
    M.n = std::max(M.n, Mi.n);
    e_off += E;
    q_off += Mi.n_dof;
    h_off += Mi.h_total;
    t_off += Mi.t_total;
    v_off += E * 5 * (int64_t)Mi.n * Mi.n * Mi.n;
    f_off += Mi.n_faces;
    M.inst_elem_off.push_back(e_off);
    M.inst_dof_off.push_back(q_off);
  }
  M.n_elems = e_off;
  M.n_dof = q_off;
  M.h_total = h_off;
  M.t_total = t_off;
  M.n_faces = f_off;
  if (f_off >= (int64_t)1 << 31 || (int64_t)M.perms.size() >= (int64_t)1 << 31 || (int64_t)M.dense.size() >= (int64_t)1 << 31 ||
      (int64_t)M.fgeo.size() >= (int64_t)1 << 31) {
    *err = "batch too large for 32-bit face indices";
    return -7;
  }
  return 0;
}

int motion_geometry_at(const HostMesh& M, const Motion& mo, double t, std::vector<double>* cpool,
                       std::vector<double>* fgeo, std::string* err) {
  const int n2 = M.n * M.n;
  const double tk[4] = {1.0, t, t * t, t * t * t};
  cpool->assign(M.cpool.size(), 0.0);
  fgeo->assign(M.fgeo.size(), 0.0);
  for (int64_t s = 0; s < M.n_elems; ++s) {
    const TypeTab& T = M.tables.tabs[M.slot_tab[s]];
    const int nQ = T.nQ, nM = T.nM;
    const double* m = mo.mpool.data() + mo.slot_moff[s];
    double* cb = cpool->data() + M.slot_coff[s];
    for (int q = 0; q < nQ; ++q) {
      for (int i = 0; i < 9; ++i) {
        double v = 0.0;
        for (int k = 0; k < 3; ++k) v += tk[k] * m[(size_t)(9 * k + i) * nQ + q];
        cb[(size_t)i * nQ + q] = v;
      }
      double J = 0.0;
      for (int k = 0; k < 4; ++k) J += tk[k] * m[(size_t)(27 + k) * nQ + q];
      if (!(J > 0.0)) { *err = "an element is inside out at this time"; return -2; }
      cb[(size_t)9 * nQ + q] = J;
      cb[(size_t)10 * nQ + q] = 1.0 / J;
    }
    if (T.type == dgk::PRISM || T.type == dgk::PYR) {
      std::vector<double> Me((size_t)nM * nM, 0.0);
      for (int k = 0; k < 4; ++k)
        for (size_t w = 0; w < Me.size(); ++w) Me[w] += tk[k] * mo.mmat[(size_t)mo.slot_mmoff[s] + (size_t)k * nM * nM + w];
      if (!spd_inverse(nM, Me.data(), cb + (size_t)11 * nQ)) { *err = "mass matrix not positive definite"; return -2; }
    }
  }
  for (int64_t f = 0; f < M.n_faces; ++f) {
    const dgk::FaceRec& R = M.faces[f];
    if (R.cgeo < 0) continue;
    const double* a = mo.fpool.data() + (size_t)3 * R.cgeo;
    double* g = fgeo->data() + R.cgeo;
    for (int p = 0; p < n2; ++p) {
      double A[3];
      for (int d = 0; d < 3; ++d) A[d] = a[(size_t)d * n2 + p] + t * a[(size_t)(3 + d) * n2 + p] + t * t * a[(size_t)(6 + d) * n2 + p];
      const double S = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
      if (!(S > 0.0)) { *err = "a face has zero area at this time"; return -2; }
      for (int d = 0; d < 3; ++d) g[(size_t)d * n2 + p] = A[d] / S;
      g[(size_t)3 * n2 + p] = S;
    }
  }
  return 0;
}

int64_t curved_block_doubles(const dgk::TypeTab& T) { return curved_block_size(T); }

int64_t motion_block_size(const dgk::TypeTab& T) { return 34 * (int64_t)T.nQ; }

int build_motion(const HostMesh& M, const MeshInput& in, const double* vel, Motion* out, std::string* err) {
  const int64_t E = M.n_elems;
  const int n = M.n, n2 = n * n;
  const double* x = M.x1d.data();
  for (int64_t s = 0; s < E; ++s)
    if (M.slot_type[s] == dgk::TET) { *err = "moving meshes cover hexahedra, prisms and pyramids"; return -7; }
  if (M.n_curved != E) { *err = "a moving mesh needs every element on the curved path"; return -7; }
  out->slot_moff.assign(E, -1);
  out->slot_mmoff.assign(E, -1);
  int64_t total = 0, mtotal = 0;
  for (int64_t s = 0; s < E; ++s) {
    const TypeTab& T = M.tables.tabs[M.slot_tab[s]];
    out->slot_moff[s] = total;
    total += motion_block_size(T);
    if (T.type == dgk::PRISM || T.type == dgk::PYR) {
      out->slot_mmoff[s] = mtotal;
      mtotal += 4 * (int64_t)T.nM * T.nM;
    }
  }
  out->mpool.assign((size_t)total, 0.0);
  out->mmat.assign((size_t)mtotal, 0.0);
  std::vector<double> Vt[4];
  for (int t = 1; t <= 2; ++t)
    if (M.type_count[t]) Vt[t] = vandermonde(t, M.N, x);
  for (int64_t s = 0; s < E; ++s) {
    const int64_t e = M.elem_of_slot[s];
    const int type = M.slot_type[s];
    const TypeTab& T = M.tables.tabs[M.slot_tab[s]];
    const int nQ = T.nQ, nM = T.nM;
    const int64_t* V = in.verts + in.off[e];
    double Xrel[24], Urel[24], u0[3];
    for (int d = 0; d < 3; ++d) u0[d] = vel[3 * V[0] + d];
    for (int v = 0; v < kNumVerts[type]; ++v)
      for (int d = 0; d < 3; ++d) {
        Xrel[3 * v + d] = in.xyz[3 * V[v] + d] - in.xyz[3 * V[0] + d];
        Urel[3 * v + d] = vel[3 * V[v] + d] - u0[d];
      }
    const double* wq = M.tables.dpool.data() + T.W;
    double* blk = out->mpool.data() + out->slot_moff[s];
    std::vector<double> Jk((size_t)4 * nQ);
    int sign = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
          const int q = (i * n + j) * n + k;
          double F0[3][3], F1[3][3], xr[3], ur[3];
          element_map(type, Xrel, x[i], x[j], x[k], F0, xr);
          element_map(type, Urel, x[i], x[j], x[k], F1, ur);
          double dk[4], ad[3][3][3];
          det_adj_poly(F0, F1, dk, ad);
          const int sg = dk[0] > 0 ? 1 : -1;
          if (dk[0] == 0.0 || (sign != 0 && sg != sign)) { *err = "degenerate element"; return -2; }
          sign = sg;
          double cm[3][3];
          collapse_metric(type, x[i], x[j], x[k], cm);
          for (int c = 0; c < 3; ++c)
            for (int l = 0; l < 3; ++l)
              for (int d = 0; d < 3; ++d) {
                double m = 0.0;
                for (int kk = 0; kk < 3; ++kk) m += cm[l][kk] * sg * ad[c][kk][d];
                blk[((size_t)c * 9 + l * 3 + d) * nQ + q] = wq[q] * m;
              }
          for (int c = 0; c < 4; ++c) {
            Jk[(size_t)c * nQ + q] = sg * dk[c];
            blk[(size_t)(27 + c) * nQ + q] = sg * dk[c];
          }
          for (int d = 0; d < 3; ++d) blk[(size_t)(31 + d) * nQ + q] = u0[d] + ur[d];
        }
    if (type == dgk::PRISM || type == dgk::PYR) {
      const double* Vq = Vt[type].data();
      for (int c = 0; c < 4; ++c) {
        double* Mc = out->mmat.data() + out->slot_mmoff[s] + (size_t)c * nM * nM;
        for (int q = 0; q < nQ; ++q) {
          const double* vq = Vq + (size_t)q * nM;
          const double w = wq[q] * Jk[(size_t)c * nQ + q];
          for (int a = 0; a < nM; ++a)
            for (int b = 0; b <= a; ++b) Mc[(size_t)a * nM + b] += w * vq[a] * vq[b];
        }
        for (int a = 0; a < nM; ++a)
          for (int b = a + 1; b < nM; ++b) Mc[(size_t)a * nM + b] = Mc[(size_t)b * nM + a];
      }
    }
  }
  // faces: the area vector w S n of the owner's face points (sign of det
  // dx/dxi times the reference orientation, as the static curved faces) and
  // the mesh velocity there
  out->fpool.assign((size_t)M.n_curved_faces * 12 * n2, 0.0);
  for (int64_t f = 0; f < M.n_faces; ++f) {
    const dgk::FaceRec& R = M.faces[f];
    if (R.cgeo < 0) { *err = "a moving mesh needs every face owner curved"; return -7; }
    const int64_t e0 = M.face_e0[f];
    const int l0 = M.face_l0[f];
    const int t0 = in.type[e0];
    const int64_t* V0 = in.verts + in.off[e0];
    const int* fv = kFaceVerts[t0][l0];
    const double* c0r = kRefVerts[t0][fv[0]];
    const double* c1r = kRefVerts[t0][fv[1]];
    const double* c2r = kRefVerts[t0][fv[2]];
    const int nv = kFaceNV[t0][l0];
    double tsr[3], ttr[3], nref[3], out_ref[3] = {0, 0, 0}, cen[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      tsr[k] = 0.5 * (c1r[k] - c0r[k]);
      ttr[k] = 0.5 * (c2r[k] - c0r[k]);
    }
    cross(tsr, ttr, nref);
    for (int v = 0; v < kNumVerts[t0]; ++v)
      for (int k = 0; k < 3; ++k) cen[k] += kRefVerts[t0][v][k] / kNumVerts[t0];
    for (int i = 0; i < nv; ++i)
      for (int k = 0; k < 3; ++k) out_ref[k] += kRefVerts[t0][fv[i]][k] / nv - cen[k] / nv;
    const double orient = (nref[0] * out_ref[0] + nref[1] * out_ref[1] + nref[2] * out_ref[2]) > 0 ? 1.0 : -1.0;
    double Xrel[24], Urel[24], u0[3];
    for (int d = 0; d < 3; ++d) u0[d] = vel[3 * V0[0] + d];
    for (int v = 0; v < kNumVerts[t0]; ++v)
      for (int d = 0; d < 3; ++d) {
        Xrel[3 * v + d] = in.xyz[3 * V0[v] + d] - in.xyz[3 * V0[0] + d];
        Urel[3 * v + d] = vel[3 * V0[v] + d] - u0[d];
      }
    const TypeTab& T0 = M.tables.tabs[M.slot_tab[M.slot_of_elem[e0]]];
    const FaceDesc fd = T0.faces[l0];
    const double* fw = M.tables.dpool.data() + T0.fw + (size_t)l0 * n2;
    double* blk = out->fpool.data() + (size_t)3 * R.cgeo;
    for (int ib = 0; ib < n; ++ib)
      for (int ia = 0; ia < n; ++ia) {
        const int p = ia + n * ib;
        double abc[3];
        abc[fd.fixed] = fd.end ? 1.0 : -1.0;
        abc[fd.alpha] = x[ia];
        abc[fd.beta] = x[ib];
        double F0[3][3], F1[3][3], xr[3], ur[3];
        element_map(t0, Xrel, abc[0], abc[1], abc[2], F0, xr);
        element_map(t0, Urel, abc[0], abc[1], abc[2], F1, ur);
        double a0[3], a1[3], b0[3], b1[3];
        for (int d = 0; d < 3; ++d) {
          a0[d] = F0[d][0] * tsr[0] + F0[d][1] * tsr[1] + F0[d][2] * tsr[2];
          a1[d] = F1[d][0] * tsr[0] + F1[d][1] * tsr[1] + F1[d][2] * tsr[2];
          b0[d] = F0[d][0] * ttr[0] + F0[d][1] * ttr[1] + F0[d][2] * ttr[2];
          b1[d] = F1[d][0] * ttr[0] + F1[d][1] * ttr[1] + F1[d][2] * ttr[2];
        }
        double c0[3], c1a[3], c1b[3], c2[3];
        cross(a0, b0, c0);
        cross(a0, b1, c1a);
        cross(a1, b0, c1b);
        cross(a1, b1, c2);
        const double sg = (det3(F0) > 0 ? 1.0 : -1.0) * orient * fw[p];
        for (int d = 0; d < 3; ++d) {
          blk[(size_t)(0 * 3 + d) * n2 + p] = sg * c0[d];
          blk[(size_t)(1 * 3 + d) * n2 + p] = sg * (c1a[d] + c1b[d]);
          blk[(size_t)(2 * 3 + d) * n2 + p] = sg * c2[d];
          blk[(size_t)(9 + d) * n2 + p] = u0[d] + ur[d];
        }
      }
  }
  return 0;
}

}  // namespace dgh
