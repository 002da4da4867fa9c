// Host-side set-up of the modal DG library: operator tables per (type, N),
// mesh geometry and connectivity, Hilbert ordering.  Pure C++ (no CUDA).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "dg_common.h"

namespace dgh {

// ----------------------------------------------------------------- 1D tools
void gauss_legendre(int n, double* x, double* w);
double jacobi(int n, double alpha, double beta, double x);
double jhat(int n, int alpha, double x);  // int ((1-x)/2)^alpha jhat^2 = 1
void lagrange_values(const double* nodes, int n, double x, double* out);

// ----------------------------------------------------------------- tables
struct Tables {
  std::vector<double> dpool;
  std::vector<int> ipool;
  std::vector<dgk::TypeTab> tabs;
  int find(int type, int N) const;
  // returns table index or -1 with *err set
  int add(int type, int N, std::string* err);
};

int n_modes(int type, int N);
double factor_A(int type, int p, double a);
double factor_B(int type, int p, int q, double b);
double factor_C(int type, int p, int q, int r, double c);
void uncollapse(int type, double a, double b, double c, double* xi);
extern const double kRefVerts[4][8][3];
extern const int kNumVerts[4];
extern const int kNumFaces[4];
extern const int kFaceVerts[4][6][4];
extern const int kFaceNV[4][6];

// ----------------------------------------------------------------- mesh
struct MeshInput {
  int64_t n_vertices;
  const double* xyz;
  int64_t n_elems;
  const int8_t* type;
  const int64_t* off;
  const int64_t* verts;
  const double* period;
  int N;
  int geometry = 0;   // 0: affine elements only; 1: vertex-interpolated (curved) maps allowed
  // partition meshes: per element 1 for a ghost (a neighbour owned by another
  // part: its face traces arrive by the halo exchange, no element work runs
  // on it); a face with one ghost side and no partner, or with two ghost
  // sides, is dropped.  Null: no ghosts.
  const uint8_t* ghost = nullptr;
  // moving meshes: every hexahedron, prism and pyramid takes the pointwise
  // (curved) geometry path, affine or not, since the motion bends it
  int force_curved = 0;
};

struct HostMesh {
  int N = 0, n = 0;
  int64_t n_elems = 0, n_faces = 0, n_dof = 0, h_total = 0, t_total = 0;
  int64_t type_count[4] = {0, 0, 0, 0};
  Tables tables;
  // per slot (Hilbert order)
  std::vector<int64_t> elem_of_slot, slot_of_elem;
  std::vector<int> slot_tab;                 // table index
  std::vector<int8_t> slot_type;
  std::vector<int64_t> slot_qoff, slot_hoff; // double offsets
  std::vector<dgk::ElemGeo> slot_geo;
  // curved (non-affine) elements: per slot the offset of its block in cpool,
  // -1 for an affine element.  Block: [9][nQ] weighted contravariant metric
  // w_q (d(a,b,c)/dxi)(J dxi/dx), [nQ] J_q, [nQ] 1/J_q, and for prism and
  // pyramid the dense inverse mass matrix (V^T diag(w J) V)^{-1} [nM][nM].
  std::vector<int64_t> slot_coff;
  std::vector<double> cpool;
  int64_t n_curved = 0;
  // face-point geometry of faces whose owner is curved (per face [4][n^2]:
  // outward unit normal x, y, z and w S per owner point); FaceRec::cgeo is
  // the double offset of a face's block
  std::vector<double> fgeo;
  int64_t n_curved_faces = 0;
  // meshes built with the curved geometry: every face side's outward unit
  // normal at its own face points, [3][n^2] at 3 * (side trace offset / 5)
  // (the Navier-Stokes lifting multiplies W* by it point by point)
  std::vector<double> snrm;
  std::vector<int64_t> slot_ftoff;           // [slot][6] trace offset of (face, own side)
  std::vector<double> slot_fnrm;             // [slot][6][3] outward unit normal of each local face
                                             // (the owner's normal, negated on the neighbour side)
  // per caller element
  std::vector<int64_t> elem_qoff;            // caller-layout offsets
  std::vector<int64_t> elem_voff;            // offsets of [5][n^3] point values (projection input)
  // instances of a batch (one instance for a plain mesh): element and dof offsets
  std::vector<int64_t> inst_elem_off, inst_dof_off;
  // faces (face-kernel order)
  std::vector<dgk::FaceRec> faces;
  std::vector<dgk::FaceBlock> face_blocks;
  std::vector<int16_t> perms;                // [nperm][2][n^2]: perm then inverse
  std::vector<double> dense;                 // [ndense][n^2][n^2]
  int n_perm = 0, n_dense = 0;
  // per-type slot lists in caller order (naive scheduler; ghosts excluded)
  std::vector<int64_t> type_slots[4];
  // partition meshes: 1 for a ghost slot (no element work), and the count
  std::vector<uint8_t> slot_ghost;
  int64_t n_ghost = 0;
  // per face, the two sides' caller elements and local faces (owner first)
  std::vector<int64_t> face_e0, face_e1;
  std::vector<int8_t> face_l0, face_l1;
  // physical quadrature points, caller order [n_elems][n^3][3]
  std::vector<double> quad_xyz;
  std::vector<double> x1d, w1d;
};

// returns 0 on success, -2 (mesh) / -1 (argument) / -7 (unsupported) with *err
int build_mesh(const MeshInput& in, HostMesh* out, std::string* err);

// Several independent meshes (any mix of N) as one: instances are
// concatenated (slots, caller elements, states, faces); operator tables are
// shared per (type, N).
int build_batch(const std::vector<MeshInput>& ins, HostMesh* out, std::string* err);

uint64_t hilbert_key3(uint32_t x, uint32_t y, uint32_t z, int bits);

// Space-filling-curve partition of Sec. 3 for nparts ranks: contiguous runs
// of the Hilbert order of (nearly) equal weight, the weight of an element
// type_weight[its type] (1 each when null); part_of_elem [n_elems] in caller
// order.  Halo of every part: the elements of other parts that share a face
// with one of its elements, ascending caller indices, part p's list at
// halo_elems[halo_off[p] .. halo_off[p+1]).  Plain meshes only.
int partition_plan(const HostMesh& M, int nparts, const double* type_weight, std::vector<int64_t>* part_of_elem,
                   std::vector<int64_t>* halo_off, std::vector<int64_t>* halo_elems, std::string* err);

// Moving meshes (constant vertex velocities, x_v(t) = x_v + t u_v with t
// measured from the positions the mesh was built from): per element and face
// the polynomial coefficients in t of the geometry.  dx/dxi = F0 + t F1 at
// every point, so J (sign times det) is a cubic and the weighted contravariant
// metric w (da/dxi) (J dxi/dx) a quadratic in t.  Per slot (mpool at
// slot_moff[s]): [3][9][nQ] metric coefficients of t^0, t^1, t^2,
// [4][nQ] J coefficients, [3][nQ] mesh velocity; for prisms and pyramids
// (mmat at slot_mmoff[s], -1 for a hexahedron) [4][nM][nM] the coefficients
// of M = V^T diag(w J) V.  Per curved-owner face (fpool at
// 3 FaceRec::cgeo): [3][3][n^2] coefficients of the area vector w S n and
// [3][n^2] the mesh velocity at the owner's face points.
struct Motion {
  std::vector<int64_t> slot_moff, slot_mmoff;
  std::vector<double> mpool, mmat, fpool;
};
int build_motion(const HostMesh& M, const MeshInput& in, const double* vel, Motion* out, std::string* err);
// The geometry of a moving mesh at time t evaluated on the host from the
// coefficients, in the layouts of HostMesh::cpool (prisms and pyramids:
// the inverse of sum_k t^k M_k) and HostMesh::fgeo.
int motion_geometry_at(const HostMesh& M, const Motion& mo, double t, std::vector<double>* cpool,
                       std::vector<double>* fgeo, std::string* err);
int64_t motion_block_size(const dgk::TypeTab& T);
int64_t curved_block_doubles(const dgk::TypeTab& T);   // per-slot doubles of HostMesh::cpool

// Static per-element FP64 work estimate of one stage (initial chunk weights).
double static_cost(const dgk::TypeTab& t);

}  // namespace dgh
