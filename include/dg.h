/*
 * dg.h - C ABI of the GB300 modal DG hot-path library (libdg.so).
 *
 * The library evaluates the right-hand side of the modal discontinuous
 * Galerkin discretisation of the compressible Euler equations on periodic
 * meshes (affine, or curved with vertex-interpolated element maps) that mix
 * hexahedra, prisms, pyramids and tetrahedra, and
 * advances it with a low-storage Runge-Kutta scheme, as described in
 * "In-Memory Load Balancing for Discontinuous Galerkin Methods on Polytopal
 * Meshes" (Kopper, Schwarz, Keim, Beck):
 *   - weak form: Sec. 2, Eq. 1 (volume integral, numerical surface flux);
 *   - collapsed-coordinate (Duffy) quadrature on non-hex types: Sec. 2;
 *   - modal time stepping and the projection M^{-1} V^T W J: Sec. 2,
 *     Algorithm 1;
 *   - LSERK time integration (method of lines): Sec. 2;
 *   - space-filling-curve ordering and runtime-timer load balancing: Sec. 3,
 *     Listing 1 (per-element cost attribution) and the imbalance trigger.
 * The adjoint entry points (dg_rhs_vjp, dg_rk_vjp) have no counterpart in the
 * paper; they are the exact transposes of dg_rhs and dg_rk_step.
 *
 * Everything is FP64.  All compute runs in CUDA kernels for sm_103a; there is
 * no CPU fallback: without a usable CUDA device every call that computes
 * returns DG_ERR_CUDA.
 *
 * Conventions shared by all calls
 *   - Pointers named *_store are DEVICE pointers to FP64 arrays of n_dof
 *     doubles in the library's storage layout (per element in Hilbert order,
 *     5 blocks of nM values: [slot][var][mode]).  Prisms, pyramids and
 *     tetrahedra hold their modal coefficients there; a hexahedron holds
 *     the scaled nodal values s = W^{1/2} V Q at its n^3 volume points
 *     (point order, nM = n^3), an orthogonal change of basis (V^T W V = I for
 *     the hexahedron), so the hexahedra are time-stepped in nodal values as
 *     in the nodal DGSEM, and inner products, adjoints and cotangents are
 *     the same in both bases.  They are owned by the caller, must be 8-byte
 *     aligned, and must stay valid until the work queued on the stream has
 *     finished.
 *   - The external (caller) layout is [element][var][mode] blocks of modal
 *     coefficients for every type, in the caller's element order.
 *     dg_set_state / dg_get_state are the only conversions between the two
 *     (a permutation, and for hexahedra the change of basis); they apply to
 *     states and cotangents alike.
 *   - Modes are ordered lexicographically in (p, q, r), r fastest, over the
 *     type's index set (hex p,q,r<=N; prism p+q<=N, r<=N; pyramid p,q<=N,
 *     r<=N-max(p,q); tet p+q+r<=N).  Variables are (rho, rho u, rho v, rho w, E).
 *   - Every computing call is asynchronous on the given stream (0 = legacy
 *     default stream) and never synchronises the device, except
 *     dg_mesh_create, dg_mesh_destroy, dg_sync and the host-pointer variants
 *     of dg_set_state / dg_get_state.
 *   - A call returns DG_OK or a negative dg_status; dg_last_error() gives a
 *     thread-local message for the last failure.  Device-side conditions
 *     (non-finite residual) are sticky in the mesh and reported by dg_sync.
 *     No call aborts the process or throws across the ABI.
 *   - A mesh object may be used from one host thread at a time.  All calls
 *     on one mesh share its workspace on the device -- nodal residual, face
 *     buffer, the balanced scheduler's queue counters (each launch zeroes
 *     the counter of the next), the cost bins and dg_rk_step's parameter
 *     block -- so they must be ordered on the GPU: one stream, or streams
 *     ordered by events.  Calls on the same mesh that overlap on the GPU
 *     race on that workspace and give wrong results.  Distinct meshes share
 *     nothing (except dg_rhs_vjp_noalloc's scratch array) and may run
 *     concurrently.
 */
#ifndef DG_H_
#define DG_H_

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh; /* opaque, library-owned */

typedef enum { DG_HEX = 0, DG_PRISM = 1, DG_PYR = 2, DG_TET = 3 } dg_elem_type;

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,         /* invalid argument (null pointer, size, enum)       */
  DG_ERR_MESH = -2,        /* non-affine (or inverted) element, unmatched face  */
  DG_ERR_CUDA = -3,        /* a CUDA runtime call failed (no device, launch...) */
  DG_ERR_OOM = -4,         /* device or host allocation failed                  */
  DG_ERR_TIMEOUT = -5,     /* reserved: a bounded device wait gave up           */
  DG_ERR_NONFINITE = -6,   /* a residual or state entry was not finite          */
  DG_ERR_UNSUPPORTED = -7  /* option outside what the build supports            */
} dg_status;

/* Numerical surface flux (F.n)* of Eq. 1.  DG_FLUX_EC is Chandrashekar's
 * entropy-conservative two-point flux F#(U-, U+).n with no dissipation (the
 * interface flux under which the split form of dg_set_volume_form conserves
 * entropy); the adjoint entry points and Navier-Stokes take LF or Roe. */
typedef enum { DG_FLUX_LF = 0, DG_FLUX_ROE = 1, DG_FLUX_EC = 2 } dg_flux;

/* Volume term of the hexahedra (dg_set_volume_form). */
typedef enum { DG_VOLUME_WEAK = 0, DG_VOLUME_SPLIT = 1 } dg_volume_form;
/* Element scheduling (Sec. 3's load balancing on one GPU; results are
 * bitwise identical for all four):
 *   BALANCED  persistent launches whose blocks pop cost-weighted chunks of the
 *             Hilbert order from an atomic queue (guided self-scheduling);
 *   NAIVE     one launch per element type and phase in caller order;
 *   STATIC    one contiguous Hilbert segment of equal element count per
 *             resident block (the paper's partition without balancing);
 *   WEIGHTED  one contiguous Hilbert segment of equal weight per resident
 *             block, with the per-(type, N) weights of the timers once
 *             dg_rebalance has read them (the paper's balanced partition). */
typedef enum { DG_SCHED_BALANCED = 0, DG_SCHED_NAIVE = 1, DG_SCHED_STATIC = 2, DG_SCHED_WEIGHTED = 3 } dg_scheduler;
typedef enum { DG_EULER = 0, DG_NAVIER_STOKES = 1 } dg_physics;

/* Element geometry (Sec. 2: x = chi(xi) with a pointwise Jacobian J; with
 * Algorithm 1 the projection M^{-1} V^T W J then differs per element).
 *   DG_GEOM_AFFINE  every element must be an affine image of its reference
 *                   element (DG_ERR_MESH otherwise).
 *   DG_GEOM_VERTEX  elements that are not affine are curved: their map is the
 *                   vertex interpolant of the reference element (trilinear
 *                   hex; prism linear on the triangle times linear in zeta;
 *                   pyramid (1 +- a)(1 +- b)(1 - c)/8 on the base vertices
 *                   and (1 + c)/2 on the apex in its collapsed coordinates
 *                   a, b, c; tetrahedra are always affine), so quadrilateral
 *                   faces are bilinear.  A curved element keeps J, the
 *                   contravariant metric and, for prisms and pyramids, the
 *                   dense inverse mass matrix (V^T diag(w J) V)^{-1} of
 *                   Algorithm 1 per quadrature point in device memory; a
 *                   curved hexahedron applies M^{-1} V^T as V^T diag(1/J)
 *                   (exact: its V is square with V^T W V = I).  Affine
 *                   elements of such a mesh take the affine path.  Every
 *                   call supports curved meshes, for the Euler and the
 *                   Navier-Stokes equations (the BR1 lifting then uses the
 *                   pointwise metric and the normals at each face point).
 *                   All instances of a batch must request the same
 *                   geometry kind (DG_ERR_ARG otherwise). */
typedef enum { DG_GEOM_AFFINE = 0, DG_GEOM_VERTEX = 1 } dg_geometry;

/* Mesh description, caller-owned, read only during dg_mesh_create.
 * Elements are affine images of the reference elements (or curved, see
 * dg_geometry); the local vertex
 * order of element e (elem_verts[elem_vert_off[e] .. elem_vert_off[e+1]-1])
 * follows the reference vertex order:
 *   hex     (-1,-1,-1) (1,-1,-1) (-1,1,-1) (1,1,-1) then the same at zeta=+1
 *   prism   (-1,-1,-1) (1,-1,-1) (-1,1,-1) then the same at zeta=+1
 *   pyramid (-1,-1,-1) (1,-1,-1) (-1,1,-1) (1,1,-1) apex (-1,-1,1)
 *   tet     (-1,-1,-1) (1,-1,-1) (-1,1,-1) (-1,-1,1)
 * Faces are matched by their vertex positions reduced modulo `period`
 * (periodic in all three directions); every face must have exactly one
 * partner, and the vertices of one face must be distinct modulo the period. */
typedef struct {
  int64_t n_vertices;
  const double* xyz;            /* host [n_vertices][3]                          */
  int64_t n_elems;
  const int8_t* type;           /* host [n_elems], dg_elem_type                   */
  const int64_t* elem_vert_off; /* host [n_elems + 1], CSR offsets                */
  const int64_t* elem_verts;    /* host [elem_vert_off[n_elems]] vertex ids       */
  const double* period;         /* host [3] box lengths; required (non-NULL)      */
  int N;                        /* polynomial degree, 1 <= N <= DG_MAX_N          */
  int flux;                     /* dg_flux                                        */
  double gamma;                 /* ratio of specific heats (1.4)                  */
  int scheduler;                /* dg_scheduler                                   */
  double imbalance_threshold;   /* rebalance when max/mean SM load - 1 exceeds it */
  int geometry;                 /* dg_geometry (0 = affine elements only)         */
} dg_mesh_desc;

#define DG_MAX_N 6

/* Build the mesh: reference tables per (type, N), affine metrics, face
 * connectivity with the owner rule (owner = smaller caller index; flux and
 * face points on the owner's side), Hilbert ordering of element centroids,
 * and the device workspace.  Synchronises `stream`.  *out receives a handle
 * to free with dg_mesh_destroy. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, cudaStream_t stream, dg_mesh** out);
dg_status dg_mesh_destroy(dg_mesh* mesh);

/* Moving mesh (Sec. 2: the mesh may move in time; Algorithm 1: the
 * projection is then solved afresh because J depends on time).
 * vertex_velocity: host [n_vertices][3], caller-owned, read during the call:
 * vertex v sits at xyz[v] + t vertex_velocity[v] at mesh time t, which starts
 * at 0 (the positions of desc).  Periodic images of one point must share
 * its velocity.  Every hexahedron, prism and pyramid takes the pointwise
 * (curved) geometry path, its map the vertex interpolant at every time, so
 * J is a cubic and the contravariant metric a quadratic in t; their
 * coefficients and the mesh velocity at every point stay in device memory
 * (dg_mesh_geometry does not count them).  The residual is the moving-frame
 * weak form: fluxes F(q) - q xdot in the volume and the LF flux in the frame
 * of the face's normal mesh speed on the faces.  dg_rk_step evolves the
 * mass-weighted state M Q: each stage solves M^ Q_s = (M Q)_s with M^ built
 * from the LSERK stage values of t^k, so that a constant state stays
 * constant (a discrete geometric conservation law), and advances the mesh
 * time by nsteps dt; Q_store holds Q at the mesh time before and after.  The
 * solves reach the exact Cholesky solve to FP64 rounding (FP64 iterative
 * refinement around an FP32 Cholesky factor).
 * dg_rhs returns M(t)^{-1} (vol - surf) at the mesh time; dg_project and
 * dg_load_vector use the geometry of the mesh time (dg_quad_points returns
 * the points at t = 0).  Navier-Stokes (dg_set_physics) runs the BR1 lifting
 * on the geometry of each stage time -- the lifting of prisms and pyramids
 * projects with M(t_s)^{-1}, three more stage solves between the two halves
 * of the volume phase -- with the viscous fluxes unchanged and the convective
 * flux in the moving frame.  Requirements: flux DG_FLUX_LF, no tetrahedra,
 * the weak volume form; the adjoint, the checkpointed steps, dg_autotune and
 * the stage-by-stage calls of partitioned solves (dg_rk_prime, dg_rk_stage,
 * dg_rk_stage_lift) return DG_ERR_UNSUPPORTED.  An element that the motion turns
 * inside out makes the next dg_sync return DG_ERR_MESH. */
dg_status dg_mesh_create_moving(const dg_mesh_desc* desc, const double* vertex_velocity, cudaStream_t stream,
                                dg_mesh** out);
/* Host only (no device needed): the pointwise geometry of desc with every
 * hexahedron, prism and pyramid on the curved path, per element
 * ([9][nQ] weighted contravariant metric w (da/dxi)(J dxi/dx), [nQ] J, [nQ]
 * 1/J, prisms and pyramids [nM][nM] M^{-1} = (V^T diag(w J) V)^{-1}), in
 * caller element order, and per face with a curved owner ([3][n^2] unit
 * normal, [n^2] w S at the owner's face points) in the order of (owner, the
 * owner's local face), the owner being the smaller caller index.  With
 * vertex_velocity (host [n_vertices][3]) it is the moving mesh's geometry at
 * time t evaluated from the coefficients that dg_mesh_create_moving keeps; with
 * NULL the static geometry of desc itself (t ignored).  Two-call pattern: the
 * sizes are always written; elem_geo / face_geo (host, caller-owned) are
 * filled when non-NULL.  DG_ERR_MESH if an element is inside out at t. */
dg_status dg_geometry_at(const dg_mesh_desc* desc, const double* vertex_velocity, double t, int64_t* n_elem_doubles,
                         int64_t* n_face_doubles, double* elem_geo, double* face_geo);
/* The mesh time of a moving mesh (0 for a static one); dg_set_mesh_time sets
 * it (DG_ERR_UNSUPPORTED for a static mesh). */
dg_status dg_mesh_time(const dg_mesh* mesh, double* t);
dg_status dg_set_mesh_time(dg_mesh* mesh, double t);

/* Batch of independent meshes as one handle.  The paper advances one mesh at
 * one N; a batch evaluates Eq. 1 on each instance separately (no face couples
 * two instances), so every call below acts on all instances at once: one
 * persistent element launch and one face launch per phase cover the whole
 * batch, whatever the mix of types and N.  descs (host, [n_instances],
 * caller-owned, read during the call): each instance's mesh and N; flux and
 * gamma must be equal across instances (DG_ERR_ARG otherwise), scheduler and
 * imbalance_threshold are taken from descs[0].  Operator tables are shared per
 * (type, N).  Layouts (caller, storage, point values, quadrature points) are
 * the instances' own layouts concatenated in instance order; element e of
 * instance i is caller element instance_elem_off[i] + e.  Errors in one
 * instance report its index in dg_last_error().  Synchronises `stream`;
 * free with dg_mesh_destroy. */
dg_status dg_batch_create(const dg_mesh_desc* descs, int n_instances, cudaStream_t stream, dg_mesh** out);

/* Curved-geometry summary (host-only): number of curved elements, of faces
 * whose owner is curved (per-point normals and w S), and the doubles of
 * pointwise geometry the mesh holds in device memory.  Pointers may be NULL. */
dg_status dg_mesh_geometry(const dg_mesh* mesh, int64_t* n_curved_elems, int64_t* n_curved_faces, int64_t* geometry_doubles);

/* Instance offsets of a handle from dg_batch_create (a plain mesh is a batch
 * of one).  instance_elem_off, instance_dof_off (host, [n_instances + 1],
 * may be NULL): first caller element and first state entry of each instance,
 * the last entry being the totals. */
dg_status dg_batch_layout(const dg_mesh* mesh, int64_t* instance_elem_off, int64_t* instance_dof_off);

/* Host-only validation of a mesh description: runs the same set-up as
 * dg_mesh_create without touching a GPU.  counts (host, [8], may be NULL):
 * n_elems, n_faces, hex, prism, pyramid, tet counts, number of distinct
 * index-permutation face maps, number of interpolating face maps.
 * quad_xyz (host, [n_elems * (N+1)^3][3], may be NULL) receives the physical
 * volume quadrature points in caller order (as dg_quad_points).
 * slot_of_elem (host, [n_elems], may be NULL) receives the Hilbert slots. */
dg_status dg_mesh_check(const dg_mesh_desc* desc, int64_t* counts, double* quad_xyz, int64_t* slot_of_elem);

/* Host-only (no GPU): the space-filling-curve partition of Sec. 3 for nparts
 * ranks and the halo each rank needs -- the bookkeeping of a multi-GPU
 * decomposition of one mesh (this library runs one GPU per mesh; the plan is
 * what a partitioned run, or a redistribution after the imbalance trigger,
 * would exchange).  Parts are contiguous runs of the Hilbert order of
 * (nearly) equal weight, an element weighing type_weight[its dg_elem_type]
 * (host [4], e.g. the per-type costs of dg_cost_table; NULL: 1 each).
 * part_of_elem (host, [n_elems]) receives each caller element's part;
 * halo_off (host, [nparts + 1]) the offsets of every part's halo list in
 * halo_elems (host, [halo_off[nparts]], may be NULL to query the sizes): the
 * caller indices, ascending, of the elements of other parts that share a face
 * with the part's elements (the states a rank must receive to evaluate Eq. 1
 * on its own elements).  1 <= nparts <= n_elems. */
dg_status dg_partition_plan(const dg_mesh_desc* desc, int nparts, const double* type_weight, int64_t* part_of_elem,
                            int64_t* halo_off, int64_t* halo_elems);

/* One part of a partitioned mesh (Sec. 3: each rank owns a contiguous
 * space-filling-curve segment of the elements and exchanges the traces on
 * the faces it shares with other ranks every stage).  desc describes the
 * whole mesh; part_of_elem (host, [n_elems], e.g. from dg_partition_plan)
 * assigns every caller element to one of nparts parts.  The part mesh holds
 * the elements of `part` and, as ghosts, every element of another part that
 * shares a face with one of them; its caller element order is ascending
 * global caller index (dg_part_elements), so the owner rule and every face
 * computation match the whole mesh's, and a partitioned run reproduces the
 * whole mesh's residual and steps bit for bit on the owned elements.  No
 * element work runs on ghosts: their face traces arrive by the halo exchange
 * (dg_halo_pack / dg_halo_unpack; for Navier-Stokes also the gradient traces,
 * dg_halo_pack_gradients / dg_halo_unpack_gradients).  A partition mesh runs
 * the Euler or the Navier-Stokes equations with the balanced or naive
 * scheduler and steps stage by stage (dg_rk_prime / dg_rk_stage_lift /
 * dg_rk_stage); whole-residual calls (dg_rhs, dg_rk_step, dg_autotune, the
 * adjoint) return DG_ERR_UNSUPPORTED.  Synchronous. */
dg_status dg_mesh_create_part(const dg_mesh_desc* desc, const int64_t* part_of_elem, int nparts, int part,
                              cudaStream_t stream, dg_mesh** out);

/* Host-only (no GPU): the halo plan of part `part` that dg_mesh_create_part
 * builds -- send_faces / recv_faces (host [nparts]) as dg_halo_counts, and
 * (host, may be NULL) the faces' global keys, 8 * (global owner element) +
 * (owner's local face), in send and in receive order (peers ascending, keys
 * ascending within a peer).  Part q's send keys for part p equal part p's
 * receive keys from part q, in the same order: the contract that lets ranks
 * exchange packed blocks without further bookkeeping. */
dg_status dg_halo_plan(const dg_mesh_desc* desc, const int64_t* part_of_elem, int nparts, int part,
                       int64_t* send_faces, int64_t* recv_faces, int64_t* send_keys, int64_t* recv_keys);

/* The part's elements: *n_local (host) and, when not NULL, their global
 * caller indices (host [n_local], ascending) and ghost flags (host
 * [n_local], 1 for a ghost).  The part's state layouts (dg_set_state etc.)
 * hold every local element; only owned elements are computed. */
dg_status dg_part_elements(const dg_mesh* mesh, int64_t* n_local, int64_t* global_of_local, int8_t* is_ghost);

/* Halo sizes: send_faces / recv_faces (host [nparts], may be NULL) the number
 * of face traces this part sends to / receives from each part, and
 * *doubles_per_face (may be NULL) = 5 (N+1)^2.  The send buffer holds the
 * blocks for part 0, then part 1, ...; within a peer the faces are ordered by
 * their global key (owner element, owner's local face), the order in which
 * the peer's receive buffer expects them. */
dg_status dg_halo_counts(const dg_mesh* mesh, int64_t* send_faces, int64_t* recv_faces, int64_t* doubles_per_face);

/* Pack this part's face traces that other parts need into send (device,
 * [sum send_faces][5 (N+1)^2]); unpack the traces received from other parts
 * (device, [sum recv_faces][5 (N+1)^2], same peer grouping) into the ghost
 * side of the shared faces.  Between them the caller moves the blocks (NCCL
 * send/recv, peer copies, or a device copy when two parts share a GPU).
 * Asynchronous. */
dg_status dg_halo_pack(dg_mesh* mesh, double* send, cudaStream_t stream);
dg_status dg_halo_unpack(dg_mesh* mesh, const double* recv, cudaStream_t stream);

/* Navier-Stokes, the second exchange of a stage (BR1: the flux needs the
 * lifted gradient on both sides of a face): the same faces, peers and order
 * as dg_halo_pack / dg_halo_unpack, 15 (N+1)^2 doubles per face (the
 * gradient of the five primitive variables in three directions at the face
 * points), packed from and unpacked into the gradient-trace buffer that
 * dg_rk_stage_lift fills.  DG_ERR_UNSUPPORTED for the Euler equations.
 * Asynchronous. */
dg_status dg_halo_pack_gradients(dg_mesh* mesh, double* send, cudaStream_t stream);
dg_status dg_halo_unpack_gradients(dg_mesh* mesh, const double* recv, cudaStream_t stream);

/* Stage-wise LSERK(5,4) for partitioned runs (Sec. 2, Sec. 3).  dg_rk_prime
 * runs the forward phase of the first stage (state at the points, the
 * element's face traces, the volume term) on Q_store.  dg_rk_stage(stage =
 * 0..4) runs the face phase and the backward phase of that stage with the
 * LSERK update of Q_store and K_store, and -- unless last != 0 -- the forward
 * phase of the next stage on the new state (the next step's first stage
 * after stage 4).  One step: prime (first step only), then for every stage:
 * halo exchange, dg_rk_stage.  Navier-Stokes splits the stage's face phase
 * in two: dg_rk_stage_lift runs the BR1 lifting (face values W*, then the
 * element volume phase: lifted gradient, its face traces, the volume term),
 * the caller exchanges the gradient traces, and dg_rk_stage runs the flux
 * face phase and the backward phase (DG_ERR_ARG if the lifting half has not
 * run for the stage).  Works on any mesh.  Asynchronous. */
dg_status dg_rk_prime(dg_mesh* mesh, const double* Q_store, cudaStream_t stream);
dg_status dg_rk_stage_lift(dg_mesh* mesh, cudaStream_t stream);
dg_status dg_rk_stage(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int stage, int last,
                      cudaStream_t stream);

/* n_dof = 5 * sum_e nM(type_e, N).  slot_of_elem (host, [n_elems], may be
 * NULL) receives the Hilbert slot of every caller element.  counts (host,
 * [6], may be NULL) receives n_elems, n_faces, and the number of hex, prism,
 * pyramid and tet elements. */
dg_status dg_mesh_layout(const dg_mesh* mesh, int64_t* n_dof, int64_t* slot_of_elem, int64_t* counts);

/* Convert a state (or a cotangent) between the caller layout Q_ext and the
 * storage layout: element blocks permuted, hexahedra's modal coefficients Q
 * mapped to W^{1/2} V Q and back by V^T W^{1/2}.  Q_ext and Q_store must not
 * overlap.  is_device = 1: Q_ext is a device pointer and the call is asynchronous;
 * is_device = 0: Q_ext is host memory (pinned or pageable) and the call
 * synchronises `stream` before returning. */
dg_status dg_set_state(dg_mesh* mesh, const double* Q_ext, int is_device, double* Q_store, cudaStream_t stream);
dg_status dg_get_state(const dg_mesh* mesh, const double* Q_store, double* Q_ext, int is_device, cudaStream_t stream);

/* Physical volume quadrature points (collapsed Gauss-Legendre, n^3 per element,
 * n = N+1), caller element order: host [n_elems * n^3][3]; for a batch the
 * instances' arrays concatenated (each with its own n).  Host-only. */
dg_status dg_quad_points(const dg_mesh* mesh, double* xyz_out);

/* Algorithm 1 projection Q = M^{-1} V^T W J q of point values q (device,
 * caller order, [n_elems][5][n^3] at the points of dg_quad_points; for a
 * batch the instances' arrays concatenated) onto the modal space, written to
 * Q_store.  Asynchronous. */
dg_status dg_project(dg_mesh* mesh, const double* q_points, double* Q_store, cudaStream_t stream);

/* The right-hand side of that projection, b = V^T W J q per element:
 * b_i = the volume-rule integral of q times phi_i (with the pointwise J of a
 * curved element), for point values q laid out as dg_project reads them,
 * written to b_store (device, storage layout); dg_project is M^{-1} b.  It is
 * also the gradient of a functional sum_q w_q J_q f(U_q) with respect to the
 * modal state when q = df/dU at the points (the seed of an adjoint).
 * Asynchronous. */
dg_status dg_load_vector(dg_mesh* mesh, const double* q_points, double* b_store, cudaStream_t stream);

/* The inverse direction: the modal expansion of Q_store evaluated at the
 * volume quadrature points, U = V Q (the first step of Eq. 1's residual and
 * of Algorithm 1's nodal form), written to u_points (device, caller order,
 * the layout dg_project reads).  Asynchronous. */
dg_status dg_eval_nodal(dg_mesh* mesh, const double* Q_store, double* u_points, cudaStream_t stream);

/* R = M^{-1}(vol - surf) of Eq. 1 for the state Q_store; R_store (device,
 * storage layout) is overwritten.  Asynchronous. */
dg_status dg_rhs(dg_mesh* mesh, const double* Q_store, double* R_store, cudaStream_t stream);

/* nsteps LSERK(5,4) steps (Carpenter-Kennedy 2N storage, Sec. 2) of size
 * dt, in place on Q_store; K_store is the second register (its input value
 * is ignored, K = 0 at every step start).  The stage loop is replayed from
 * CUDA graphs captured on the first call: one that primes a step, one per
 * step and one for the last step, whose element launches read Q_store,
 * K_store and dt from a device parameter block that the first graph's head
 * node writes.  A new state or register pointer, dt or step count only
 * changes that node's arguments (no capture, no instantiation); a change of
 * scheduler, stage fusion, launch groups, chunk tables or physics captures
 * the graphs again.  With profiling on (dg_set_profiling) the call is one
 * graph with event nodes, captured again whenever an argument changes.
 * Asynchronous. */
dg_status dg_rk_step(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int nsteps, cudaStream_t stream);

/* Host [1]: how many times dg_rk_step has captured (and instantiated) its
 * graphs on this mesh. */
dg_status dg_graph_captures(const dg_mesh* mesh, int64_t* captures);

/* Qbar = (dR/dQ)^T Rbar at Q_store (all device, storage layout); Qbar is
 * overwritten.  No counterpart in the paper.  Asynchronous. */
dg_status dg_rhs_vjp(dg_mesh* mesh, const double* Q_store, const double* Rbar, double* Qbar, cudaStream_t stream);

/* Allocation-free dg_rhs_vjp (the paper has no counterpart; this is a
 * library convenience).  Same arguments, result and asynchrony as
 * dg_rhs_vjp, for callers that must not allocate device memory at call time
 * - for example code whose device memory is budgeted once at start-up, or
 * that runs where calling the CUDA allocator is not allowed.  dg_rhs_vjp
 * allocates its adjoint face buffer with cudaMalloc on first use; this entry
 * point instead uses a fixed scratch array of 64 MiB (8 Mi doubles) that is
 * part of the library image, so every GPU that loads the library holds it
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   - The mesh's face buffer must fit: meshes needing more than 8 Mi doubles
 *     of face scratch (2 * 5 * (N+1)^2 per face) get DG_ERR_ARG with a
 *     message; use dg_rhs_vjp for those.
 *   - The mesh's device must be the current device.  Every call looks up
 *     the array's device address with cudaGetSymbolAddress (which allocates
 *     nothing); the first call on a device can make the runtime load the
 *     library's device code there, so make that first call before any
 *     stream capture.
 *   - All calls on a device share the one array and it keeps the last
 *     call's contents (nothing in it has to start at zero: every slot is
 *     written before it is read).  Calls that overlap on the GPU (different
 *     streams without ordering, or two meshes at once) race on it. */
dg_status dg_rhs_vjp_noalloc(dg_mesh* mesh, const double* Q_store, const double* Rbar, double* Qbar,
                             cudaStream_t stream);

/* Q0bar = (dQ_K/dQ_0)^T QKbar for nsteps LSERK steps of size dt from Q0_store.
 * A forward pass from Q0 keeps the stage data of as many final segments of
 * ckpt_every steps as fit in the mesh's share of the free device memory
 * (half by default; see dg_set_adjoint_storage, dg_set_adjoint_memory) and stores Q at the start of every earlier
 * segment; the reverse sweep uses the kept data directly and recomputes the
 * earlier segments from their checkpoints.  ckpt_every = 0 picks the longest
 * segment whose stage data fit in that memory.  The result does not depend on
 * the segment length.  No counterpart in the paper.  Asynchronous. */
dg_status dg_rk_vjp(dg_mesh* mesh, const double* Q0_store, double dt, int nsteps, int ckpt_every,
                    const double* QKbar, double* Q0bar, cudaStream_t stream);

/* The same split at the checkpoints, for callers that run the forward steps
 * themselves (an autograd forward): dg_rk_step_checkpointed advances Q_store
 * by nsteps steps exactly as dg_rk_step and writes Q at the start of every
 * segment of ckpt_every steps to ckpt_store (device, caller-owned,
 * [ceil(nsteps / ckpt_every)][n_dof] in the storage layout);
 * dg_rk_vjp_checkpointed then computes Q0bar from those checkpoints without
 * the forward pass that dg_rk_vjp runs to place them (bitwise the same result
 * as dg_rk_vjp from the same Q0).  QKbar and Q0bar may alias.
 * Asynchronous. */
dg_status dg_rk_step_checkpointed(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int nsteps,
                                  int ckpt_every, double* ckpt_store, cudaStream_t stream);
dg_status dg_rk_vjp_checkpointed(dg_mesh* mesh, const double* ckpt_store, double dt, int nsteps, int ckpt_every,
                                 const double* QKbar, double* Q0bar, cudaStream_t stream);

/* Memory/time trade-off of dg_rk_vjp.  keep_stages = 1 (default): forward
 * passes keep, per stage, the nodal state and the own-side traces (Euler:
 * (H + F) doubles per stage, H = 5 sum_e n^3 and F = the face buffer,
 * 10 n^2 per face; Navier-Stokes: 4 (H + F), adding the gradient traces and
 * the nodal gradient) -- dg_rk_vjp's first pass for its final segments (up to
 * half of the free device memory), each segment recomputation for its own
 * 5 ckpt_every stages -- so the reverse stages do not recompute them.  The
 * store stays allocated with the mesh.  If that memory cannot be allocated
 * dg_rk_vjp silently recomputes.  keep_stages = 0: always recompute (and free
 * the store).  Results are bitwise identical either way. */
dg_status dg_set_adjoint_storage(dg_mesh* mesh, int keep_stages);

/* Share of the device memory that is free at the call (the mesh's own stage
 * store counted as free) that dg_rk_vjp may fill with kept stage data:
 * 0 < fraction <= 0.95, default 0.5.  A larger share lets the forward pass
 * keep more final steps, so fewer segments are run twice (the self-contained
 * adjoint of a long trajectory); the store stays allocated until
 * dg_set_adjoint_storage(mesh, 0) or dg_mesh_destroy.  When the whole
 * trajectory's stage data do not fit in the share, dg_rk_vjp keeps a compact
 * form instead -- the nodal state per stage (and, Navier-Stokes, the nodal
 * gradient), about half the bytes -- and every reverse stage rebuilds its
 * face traces from them, so more final steps are kept.  Results are bitwise
 * identical for every share and either form. */
dg_status dg_set_adjoint_memory(dg_mesh* mesh, double fraction);

/* Volume term of the hexahedra.  DG_VOLUME_WEAK (default): the weak form of
 * Eq. 1.  DG_VOLUME_SPLIT: the entropy-stable split form that Sec. 2 uses for
 * stabilisation -- Chandrashekar's two-point flux F# in flux-differencing
 * form on the hexahedron's Gauss-Legendre nodes, with the hybridised
 * summation-by-parts operator of Gauss collocation along every coordinate
 * line (antisymmetric part of W D between nodes, coupling of every node to
 * the line's two face states), and entropy-projected traces u(E v(u)) (the
 * entropy variables extrapolated to the face points) on which the surface
 * flux is taken.  Prisms, pyramids and tetrahedra keep the weak form.  With
 * DG_FLUX_EC the semi-discrete entropy of an all-hexahedral periodic mesh is
 * conserved; with DG_FLUX_LF it decays.  Euler equations and affine meshes
 * only (DG_ERR_UNSUPPORTED otherwise, and from the adjoint entry points while
 * it is set).  Synchronous set-up (launch configuration); captured graphs are
 * rebuilt on the next dg_rk_step. */
dg_status dg_set_volume_form(dg_mesh* mesh, int form);

/* Governing equations of dg_rhs / dg_rk_step (a new mesh solves the Euler
 * equations).  DG_NAVIER_STOKES: the Navier-Stokes-Fourier equations that
 * the paper's solver integrates (Sec. 2; Eq. 1 with a flux F(q, grad q); the
 * viscous TGV of Sec. 4), with constant dynamic viscosity mu (>= 0), Prandtl
 * number Pr (> 0), Stokes stress and Fourier heat flux
 * q = -mu gamma / ((gamma - 1) Pr) grad(p / rho).  The paper does not print
 * its viscous scheme; the library uses BR1 lifting of the primitive
 * variables W = (rho, u, v, w, p): per element the modal gradient
 * G_d = M^{-1}(sum_f int phi W* n_d dS - int W dphi/dx_d dx), W* the mean of
 * both traces, and the central viscous face flux (F_v(U-, G-) + F_v(U+, G+)).n/2
 * added to the inviscid Riemann flux.  Per RK stage this adds one face phase
 * (lifting values) and one element phase (gradient, traces, volume term).
 * Allocates the workspace (nodal state, lifting values, gradient traces: 5
 * times the face buffer plus the nodal residual) on first use; DG_ERR_OOM if
 * that fails.  mu and Pr are ignored for DG_EULER.  dg_rhs_vjp and dg_rk_vjp
 * differentiate whichever equations are selected (the viscous adjoint
 * allocates the nodal gradient and gradient-trace cotangents on first use);
 * dg_rhs_vjp_noalloc returns DG_ERR_UNSUPPORTED under Navier-Stokes. */
dg_status dg_set_physics(dg_mesh* mesh, int physics, double mu, double Pr);

/* Scheduler of the element kernels (dg_scheduler above): DG_SCHED_BALANCED
 * (one persistent launch per phase, blocks take cost-weighted
 * Hilbert-contiguous element chunks from an atomic queue), DG_SCHED_NAIVE
 * (one launch per element type and phase, caller element order),
 * DG_SCHED_STATIC (one persistent launch, every block owns one contiguous
 * Hilbert segment of equal element count: the SFC partition without load
 * balancing of Sec. 3) or DG_SCHED_WEIGHTED (the same with segments of equal
 * weight: the load-balanced SFC partition of Sec. 3).  Results are bitwise
 * identical. */
dg_status dg_set_scheduler(dg_mesh* mesh, int scheduler);

/* Tile shape of the element kernels: the number of warps (1..4) that work
 * together on one element (one element per thread block), for every (type,
 * N) table at once.  The default is 2 for N <= 4 and 1 above; dg_autotune
 * picks the fastest.  Rebuilds the chunk tables; results are bitwise
 * identical for every choice. */
dg_status dg_set_element_warps(dg_mesh* mesh, int warps);

/* Tile shape of one (type, N) table (balanced scheduler): tables that share
 * N and warps form one persistent launch per phase, sized for that N.
 * DG_ERR_ARG if the mesh (or batch) holds no element of that type and N. */
dg_status dg_set_table_warps(dg_mesh* mesh, int type, int N, int warps);

/* The tables present and their tile shapes: *n_tables receives the count;
 * type, N, warps (host, [max], may be NULL) the first max entries. */
dg_status dg_tile_shapes(const dg_mesh* mesh, int max, int* n_tables, int* type, int* N, int* warps);

/* Autotuner: times dg_rk_step of size dt for every uniform tile shape
 * (1..4 warps per element) on a scratch copy of Q_store (device, storage
 * layout; library-allocated scratch of 2 n_dof doubles, freed on return),
 * reads each table's time per element from the in-kernel cost probe, and
 * keeps the fastest uniform shape unless per-table shapes (each table at its
 * best resident-blocks-per-time ratio; balanced scheduler only) make the step
 * faster still.  With the environment variable DG_AUTOTUNE_CACHE naming a
 * file, results are read from and appended to it, keyed by device name, N,
 * element counts, scheduler and flux.  best_warps (may be NULL) receives the
 * uniform choice, ms_per_step (host [5], may be NULL) the times of the four
 * uniform shapes and of the per-table shapes (0 when not tried; all zeros
 * when taken from the cache).  Synchronises `stream`. */
dg_status dg_autotune(dg_mesh* mesh, const double* Q_store, double dt, int* best_warps, double* ms_per_step,
                      cudaStream_t stream);

/* Stage fusion of dg_rk_step: fused != 0 (default) runs the backward phase of
 * stage s (lift, projection, LSERK update) and the forward phase of stage s+1
 * in one element launch; fused == 0 uses two launches.  Results are bitwise
 * identical. */
dg_status dg_set_stage_fusion(dg_mesh* mesh, int fused);

/* Per-type element cost measured in the balanced kernels with %globaltimer
 * (Listing 1's per-element attribution, done per element in-kernel):
 * host [4] mean ns per element of each type (0 if none measured) and the
 * current per-SM load imbalance (max/mean - 1).  Synchronises `stream`. */
dg_status dg_cost_table(dg_mesh* mesh, double* ns_per_elem, double* imbalance, cudaStream_t stream);

/* Rebuild the weighted chunk table and the equal-weight partition of
 * DG_SCHED_WEIGHTED from the measured costs when the measured imbalance
 * exceeds the threshold (or always, if force != 0); resets the counters.
 * *rebuilt (may be NULL) tells whether it did.  Synchronises. */
dg_status dg_rebalance(dg_mesh* mesh, int force, int* rebuilt, cudaStream_t stream);

/* The imbalance trigger inside the time loop (Sec. 3: the paper checks the
 * measured imbalance during the run and redistributes when it exceeds the
 * threshold): with nsteps > 0, dg_rk_step runs dg_rebalance(force = 0) once
 * at least nsteps steps have been enqueued since the last check (that call
 * synchronises `stream`, so it must not run inside a stream capture).
 * nsteps = 0 (default) turns it off.  Results do not depend on it (every
 * schedule is bitwise identical). */
dg_status dg_set_rebalance_interval(dg_mesh* mesh, int nsteps);

/* Host [1] counters of the automatic trigger: checks made, tables rebuilt
 * (either may be NULL). */
dg_status dg_rebalance_stats(const dg_mesh* mesh, int64_t* checks, int64_t* rebalances);

/* Phase timing: with profiling on, dg_rhs and the dg_rk_step graph record
 * CUDA events around every element-kernel and face-kernel phase (events
 * inside the captured graph; a few microseconds of overhead per phase).
 * dg_phase_times synchronises `stream` and returns, for the most recent
 * dg_rk_step / dg_rhs call, host [4]: total element-phase ms, total
 * face-phase ms, number of element phases, number of face phases. */
dg_status dg_set_profiling(dg_mesh* mesh, int on);
dg_status dg_phase_times(dg_mesh* mesh, double* out, cudaStream_t stream);
/* Moving meshes, with profiling on: for the most recent dg_rk_step / dg_rhs
 * call, host [4]: total ms of the per-stage geometry kernels, total ms of the
 * stage mass-matrix kernels (products and solves), the number of geometry
 * launches and the number of mass calls (a product or a solve, one launch
 * per element type each; events around each; synchronises `stream`). */
dg_status dg_moving_phase_times(dg_mesh* mesh, double* out, cudaStream_t stream);

/* Synchronise `stream` and report sticky device errors (DG_ERR_NONFINITE). */
dg_status dg_sync(dg_mesh* mesh, cudaStream_t stream);

/* Thread-local description of the last error. */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H_ */
