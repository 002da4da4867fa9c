// Records shared by the host set-up (dg_host.cpp) and the device kernels.
//
// Every element of type T and degree N works on the collapsed tensor grid of
// n^3 Gauss-Legendre points (a_i, b_j, c_k), n = N+1 (the Duffy transform of
// Sec. 2).  Nodal arrays are indexed q = (i*n + j)*n + k (c fastest).  The
// orthonormal modal basis factorises as phi_pqr = A_p(a) B_pq(b) C_pqr(c), so
// the modal->nodal map V (the generalized Vandermonde matrix of Algorithm 1)
// is applied as three ragged 1D contractions (sum factorisation):
//   c-pass  X[col][k]   = sum_t C[col][t][k] Q[moff[col] + t]   col = (p, q)
//   b-pass  Y[p][j][k]  = sum_t B[p][t][j]   X[cbase[p] + t][k]
//   a-pass  U[i][j][k]  = sum_p A[p][i]      Y[p][j][k]
// and V^T by the same passes transposed, in reverse order.
#pragma once
#include <stdint.h>

namespace dgk {

constexpr int kMaxN = 6;
constexpr int kMaxn = kMaxN + 1;
constexpr int kNumTypes = 4;
constexpr int kMaxTabs = kNumTypes * kMaxN;   // (type, N) tables, N = 1..kMaxN
enum { HEX = 0, PRISM = 1, PYR = 2, TET = 3 };

// Face descriptor of a local face: the face points are the tensor grid of
// two collapsed coordinates (alpha, beta) with the third fixed at an end.
struct FaceDesc {
  int fixed;    // collapsed coordinate held fixed: 0 = a, 1 = b, 2 = c
  int end;      // 0: -1, 1: +1
  int alpha;    // collapsed coordinate running along the face's first index
  int beta;     // collapsed coordinate running along the face's second index
  int tri;      // 1 for a triangular face (collapsed face rule)
};

// Per (type, N) operator tables.  Offsets index the shared double / int pools.
struct TypeTab {
  int type, N, n, nM, nQ, ncols, nfaces;
  // double pool
  int A;        // [n(p)][n(i)]           A_p(a_i)
  int B;        // per p: [blen[p](t)][n(j)] at boff[p]
  int C;        // per col: [len[col](t)][n(k)] at coff[col]
  int Dt;       // [n(i')][n(i)]          l'_{i'}(x_i): H(i') = sum_i Dt[i'][i] G(i)
  int ext;      // [2][n]                 l_m(-1), l_m(+1)
  int W;        // [nQ]                   w_q (Gauss-Legendre weights times the Duffy Jacobian)
  int wA;       // [nQ][3][3]             w_q d(a,b,c)_l / d(xi,eta,zeta)_k
  int minv;     // [nM]                   1 / (V^T W V)_ii   (the mass matrix is diagonal)
  int sqw;      // hexahedron: [nQ] sqrt(w_q), then [nQ] 1 / sqrt(w_q) (scaled nodal storage); -1 otherwise
  int fw;       // [nfaces][n*n]          reference face weights at the face points
  int sbp;      // hexahedron: [n][n] S_ij = w_i D_ij - w_j D_ji (D_ij = l'_j(x_i)), the antisymmetric
                //   part of the 1D collocation operator W D (split form); -1 otherwise
  int w1;       // hexahedron: [n] 1D Gauss-Legendre weights; -1 otherwise
  // int pool
  int col_moff, col_len, col_coff, col_p;   // [ncols]
  int col_order;                            // [ncols] columns by decreasing length (uniform trip counts per warp)
  int p_cbase, p_blen, p_boff;              // [n]
  int mode_col;                             // [nM]
  FaceDesc faces[6];
};

// Per-element geometry (affine): Jg = J * dxi/dx (row k = xi_k, column d = x_d)
// and 1/J, J = |det dx/dxi|.  Curved elements keep their pointwise geometry
// in a separate pool (HostMesh::cpool) and leave this record zero.
struct ElemGeo {
  double Jg[9];
  double invJ;
};

// Face record for the face kernel.  Side 0 = owner (smaller caller index);
// its face points and outward normal are used.  The neighbour's face values
// at its own points are mapped to the owner's points by `map`:
//   map >= 0 : index permutation at perms + map: perm[p] (n^2 entries),
//              then its inverse (n^2 entries)
//   map <  0 : dense interpolation matrix I[p][j] at dense + (-1 - map)
struct FaceRec {
  int64_t toff;     // double offset of side 0 trace block; side 1 at toff + 5 n^2
  int map;
  int owner_tab;    // type table of the owner (reference face weights)
  int owner_lf;     // owner's local face
  int cgeo;         // curved owner: double offset of the face's per-point normals and w S ([4][n^2]); -1 otherwise
  double nrm[3];
  double S;         // area scale |dx/ds x dx/dt| (affine owner)
};

struct FaceBlock {
  int first, count, n, pad;
};

}  // namespace dgk
