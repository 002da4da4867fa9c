// Device side of the modal DG hot path (sm_103a, FP64).
//
// Per RK stage the residual of Eq. 1 is evaluated in three phases:
//   forward  (element kernel)  Q -> nodal U = V Q on the collapsed grid (three
//            sum-factorised passes), traces of U on the element's own face
//            points, contravariant fluxes G_l = w J (da_l/dxi) (dxi/dx) F(U)
//            and the nodal volume residual H = sum_l D_l^T G_l (collocation
//            derivative, exact because every 1D factor has degree <= N);
//   faces    (face kernel)     Riemann flux (LF or Roe) at the owner's points,
//            scaled by w S; the neighbour's share is mapped back to its own
//            points (permutation or interpolation);
//   backward (element kernel)  H -= sum_faces E_f^T Fhat_f, then V^T H by the
//            transposed passes, times the diagonal M_ref^{-1} and 1/J, and the
//            fused LSERK update K <- a K + dt R, Q <- Q + b K.
// The backward phase of stage s is fused with the forward phase of stage s+1.
// One thread block (1 to 4 warps, the tile shape chosen per (type, N)) owns
// one element at a time; all work inside an element is spread over
// (variable, output) pairs so the lanes stay busy for every N.  The
// Navier-Stokes path adds a lifting face phase and a volume phase per stage
// (BR1), and every phase has a hand-written adjoint.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_common.h"

namespace dgk {

enum ElemMode : int {
  kFwd = 0,        // forward only (prime a stage)
  kBwdRhs = 1,     // backward, write R
  kBwdRk = 2,      // backward + LSERK update
  kBwdRkFwd = 3,   // backward + LSERK update + forward of the new state
  kProject = 4,    // Algorithm 1 projection of point values
  kGather = 5,     // hexahedra: caller modal coefficients -> scaled nodal storage
  kScatter = 6,    // hexahedra: scaled nodal storage -> caller modal coefficients
  kNsVolume = 7,   // Navier-Stokes: BR1 lifting, gradient traces, volume residual H
  kEval = 8,       // modal -> nodal values at the volume points (caller element order)
  kLoad = 9,       // load vector V^T W J q of point values (Algorithm 1's projection without M^{-1})
  kTraces = 10     // adjoint: face traces of a kept nodal state (Unod) and, Navier-Stokes, of a kept nodal gradient (DW)
};

struct Ctx {
  const double* dpool;
  const int* ipool;
  const TypeTab* tabs;
  const int* slot_tab;
  const int8_t* slot_type;
  const int64_t* slot_qoff;
  const int64_t* slot_hoff;
  const int64_t* slot_ftoff;   // [slot][6]
  const int64_t* elem_of_slot;
  const int64_t* elem_qoff;    // caller layout offsets
  const int64_t* elem_voff;    // caller element -> offset of its [5][n^3] point values (projection input)
  const ElemGeo* geo;
  double* H;
  double* T;
  double* Tv;                  // adjoint face buffer (seeds, then trace cotangents)
  const FaceRec* faces;
  const FaceBlock* fblocks;
  const int16_t* perms;
  const double* dense;
  unsigned int* status;        // bit 0: non-finite state seen
  unsigned long long* cost;    // [kMaxTabs tables][2]: ns, count
  unsigned long long* sm_ns;   // [num SMs]
  double gamma;
  int flux;                    // 0 LF, 1 Roe, 2 entropy-conservative (Chandrashekar F#.n, no dissipation)
  int split;                   // 1: hexahedra evaluate the entropy-stable split form of the volume term
  int nQmax;
  // Navier-Stokes (BR1) state; ns == 0 for the Euler equations
  int ns;
  double mu, kappa;            // viscosity, heat conductivity mu gamma / ((gamma - 1) Pr)
  const double* fnrm;          // [slot][6][3] outward unit normal per local face
  double* Unod;                // [slot][5][nQ] nodal state (slot_hoff offsets)
  double* L;                   // lifting face values, layout of T
  double* Vt;                  // gradient traces [face][2][3][5][n^2] (3x the offsets of T)
  double* DW;                  // adjoint: nodal lifted gradient [slot][3][5][nQ] (3x slot_hoff), or null
  double* Usave;               // Euler forward: also keep the nodal state here (slot_hoff), or null
  double* Vtb;                 // adjoint: gradient-trace cotangents, layout of Vt
  // curved (non-affine) elements; null / -1 entries for an affine mesh or element
  const int64_t* slot_coff;    // [slot] offset into cpool, -1 for an affine element
  const double* cpool;         // per curved slot: [9][nQ] metric, [nQ] J, [nQ] 1/J, (prism, pyramid) [nM][nM] M_e^{-1}
  const double* fgeo;          // per curved-owner face: [4][n^2] normal x, y, z and w S (FaceRec::cgeo)
  const double* snrm;          // curved meshes: per face side [3][n^2] outward normal at 3 * (side offset / 5)
  // moving meshes (null otherwise): the polynomial-in-t geometry per slot
  // (mpool at slot_moff: [3][9][nQ] metric, [4][nQ] J, [3][nQ] mesh
  // velocity), per prism and pyramid the mass matrix coefficients, four
  // packed lower triangles rounded to FP32 (mk32 at slot_mmoff, row i of a
  // triangle at i (i + 1) / 2: the preconditioner of the stage solves) and
  // per curved-owner face (fmot at 3 FaceRec::cgeo:
  // [3][3][n^2] area vector, [3][n^2] mesh velocity).  With mpool set, the
  // volume flux is F(q) - q xdot, the face flux the moving-frame LF flux, and
  // the backward phase returns the rate of the mass-weighted state (no M^{-1}).
  const double* mpool = nullptr;
  const int64_t* slot_moff = nullptr;
  const double* fmot = nullptr;
  const float* mk32 = nullptr;
  const int64_t* slot_mmoff = nullptr;
  // moving meshes, Navier-Stokes: the lifting of prisms and pyramids projects
  // with M(t)^{-1}, solved between two volume phases.  lift_phase 1: those
  // elements write r_d = -V^T (lifting terms) for d = 0..2 to lift (at
  // d n_dof + the slot's storage offset) and stop; 2: they read the solved
  // modal gradient there and finish; hexahedra (pointwise 1/J) run whole in
  // phase 2.  0: the fused phase of static meshes.
  double* lift = nullptr;
  int64_t lift_stride = 0;
  int lift_phase = 0;
};

// Adjoint arguments (storage layout, device).  rk == 0: Qbar = (dR/dQ)^T Rbar.
// rk == 1: one reverse LSERK stage, Kbar <- a (Kbar + b Qbar) and
// Qbar += dt (dR/dQ)^T (Kbar + b Qbar) at the stage input state Q.
struct VjpArgs {
  const double* Q;
  const double* Rbar;
  double* Kbar;
  double* Qbar;
  double a, b, dt;
  int rk;
  int stored;   // 1: the forward nodal state (Unod) and traces (T) of Q were kept by the forward pass
};

// State, register and time step of dg_rk_step, read by the element kernels
// from device memory so that one captured stage graph serves every call (the
// graph's first node, rk_params_kernel, writes them).
struct RkDyn {
  double* Q;
  double* K;
  double dt;
  double pad;
};

struct StageArgs {
  const double* Qin;   // state (storage layout) or point values / ext state
  double* Qout;        // updated state (may alias Qin) or R / storage output
  double* K;           // LSERK register
  double a, b, dt;     // K <- a K + dt R (a == 0: K <- dt R), Q <- Q + b K
  const RkDyn* dyn = nullptr;   // non-null: Qin = Qout = dyn->Q, K = dyn->K, dt = dyn->dt
};

struct Sched {
  const int64_t* list;         // naive: slots of one type in caller order
  int64_t count;               // naive: number of list entries / balanced: n chunks
  const int64_t* chunk_start;  // balanced: [count + 1] slot ranges
  unsigned int* counter;       // balanced: atomic queue head (zero at launch)
  unsigned int* next_counter;  // balanced: zeroed by this launch for the next one
};

void launch_element(const Ctx& c, int mode, const StageArgs& a, const Sched& s, bool balanced, int grid,
                    int warps_per_block, cudaStream_t st);
void launch_faces(const Ctx& c, int64_t nblocks, int n, cudaStream_t st);
// Navier-Stokes face phases: kind 0 = BR1 lifting values (T -> L), kind 1 =
// inviscid + central viscous flux (T, Vt -> T).
void launch_faces_ns(const Ctx& c, int64_t nblocks, int n, int kind, cudaStream_t st);
int element_smem_bytes_ns(int nQmax);
// phase 0: adjoint phase A (Euler), 2: phase C; Navier-Stokes adds 10: phase A
// (inviscid + viscous flux transposes), 11: phase B (lifting transpose).
void launch_vjp(const Ctx& c, int phase, const VjpArgs& va, int64_t nelem, int warps_per_block, cudaStream_t st);
// Navier-Stokes face adjoints: kind 1 = flux (before phase B), kind 0 =
// lifting values (after phase B).
void launch_faces_ns_vjp(const Ctx& c, int64_t nblocks, int n, int kind, cudaStream_t st);
void launch_faces_vjp(const Ctx& c, int64_t nblocks, int n, cudaStream_t st);
void launch_permute(const Ctx& c, const double* src, double* dst, int64_t E, int to_storage, cudaStream_t st);
// One-thread kernel that writes (Q, K, dt) into *d; the head node of the
// captured stage graphs.  rk_params_node fills the kernel-node parameters of
// that node for cudaGraphExecKernelNodeSetParams (args: &d, &Q, &K, &dt), and
// is_rk_params_kernel recognises the node's function in a captured graph.
void launch_rk_params(RkDyn* d, double* Q, double* K, double dt, cudaStream_t st);
// partition meshes: pack (T -> buffer) or unpack (buffer -> T) count face-side
// trace blocks of `per` doubles at the face-buffer offsets mult * off[]
// (mult = 3: the gradient traces, laid out at three times the trace offsets)
void launch_halo_copy(const double* src, double* dst, const int64_t* off, int64_t count, int per, bool pack,
                      cudaStream_t st, int mult = 1);
void rk_params_node(cudaKernelNodeParams* p, void** args);
bool is_rk_params_kernel(const void* func);
int element_smem_bytes(int nQmax, int warps_per_block);
// shared memory of an element launch: element_smem_bytes, or the split form's
// larger workspace when c.split is set
int element_launch_smem_bytes(int nQmax, int warps_per_block, bool split);
int face_block_threads(int n);
// curved: the mesh holds curved elements (occupancy of the kernel variants that handle them)
cudaError_t element_kernel_attributes(int nQmax, int warps_per_block, int* blocks_per_sm, bool curved = false,
                                      bool split = false);
cudaError_t element_kernel_attributes_ns(int nQmax, int warps_per_block, int* blocks_per_sm, bool curved = false);

// Moving meshes.  Geometry at time t: the curved metric, J and 1/J of every
// slot, the normals and w S of every curved-owner face and, when snrm is not
// null, both sides' own normals (the Navier-Stokes lifting), from the
// coefficients; bit 2 of *status is set where J or S is no longer positive
// (an element turned inside out).
void launch_moving_geometry(const Ctx& c, double* cpool, double* fgeo, double* snrm, int64_t n_slots,
                            int64_t n_faces, int n, double t, int grid, cudaStream_t st);
// Per slot of list[0 .. n_slots): out = M^ in (weight = 1) or out = M^{-1} in
// (weight = 0), with M^ = V^T diag(w J^) V and J^ = sum_k tau_k J_k
// (hexahedra, in their scaled nodal storage: pointwise J^).  x0 (or null):
// a nearby solution the solve starts from.  out may alias in or x0.
// max_nM / max_nQ: the largest prism / pyramid mode and point counts among
// the listed slots (0 if none: shared memory).  nblk (solves only): blocks of
// five variables at the slot's storage offset + k blk_stride, all solved
// with one factor of M^.  fac_out (solves only, or null): keep each prism's
// and pyramid's FP32 factor there, at its c.mk32 offset; fac_in (or null):
// use the factor kept there instead of forming one (the FP64 refinement
// corrects for a matrix that differs from M^ within the FP32 rounding).
cudaError_t launch_moving_mass(const Ctx& c, const int64_t* list, int64_t n_slots, const double* in, double* out,
                               const double* x0, const double* tau, int weight, int max_nM, int max_nQ, int grid,
                               cudaStream_t st, int nblk = 1, int64_t blk_stride = 0, float* fac_out = nullptr,
                               const float* fac_in = nullptr);

}  // namespace dgk
