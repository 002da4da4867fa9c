// C ABI of the modal DG library (include/dg.h): mesh upload, launch
// orchestration of the per-stage phases, CUDA-graph replay of the LSERK stage
// loop, scheduler and cost table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dg.h"
#include "dg_host.h"
#include "dg_kernels.cuh"

namespace {

thread_local std::string g_err;

dg_status fail(dg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

dg_status cuda_fail(cudaError_t e, const char* where) {
  return fail(DG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients.
const double kLsA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kLsB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

}  // namespace

struct dg_mesh {
  int device = 0;
  dgh::HostMesh h;
  int flux = 0;
  int split = 0;      // DG_VOLUME_SPLIT: entropy-stable split form on the hexahedra
  // partition meshes (dg_mesh_create_part): the part's elements (owned and
  // ghosts, ascending global caller index) and the halo lists: per peer part,
  // the face-buffer offsets of the owned traces to send and of the ghost
  // slots to fill, both in the order of the faces' global keys
  int nparts = 0, part = -1;
  std::vector<int64_t> global_of_local;
  std::vector<int64_t> send_count, recv_count, send_off, recv_off;
  int64_t* d_send_off = nullptr;
  int64_t* d_recv_off = nullptr;
  // moving meshes (dg_mesh_create_moving): the geometry coefficients, the
  // mesh time, the mass-weighted state and the stage state of dg_rk_step
  bool moving = false;
  double t_mesh = 0.0;
  int64_t *d_slot_moff = nullptr, *d_slot_mmoff = nullptr;
  double *d_mpool = nullptr, *d_fmot = nullptr, *d_Ut = nullptr, *d_S = nullptr;
  float* d_mk32 = nullptr;
  double* d_lift = nullptr;   // Navier-Stokes on a moving mesh: lifting residuals [3][n_dof]
  double* d_G = nullptr;      // ... and the lifted gradients that solve them [3][n_dof]
  bool G_warm = false;        // d_G holds the previous stage's gradients (this call's)
  // the FP32 factors of the last stage solve, at the offsets of d_mk32
  // ([L][s][rdiag] per prism and pyramid), for the lifting of the same stage
  float* d_fac = nullptr;
  int64_t n_mk32 = 0;
  bool fac_ready = false;
  int lift_phase = 0;
  double gamma = 1.4;
  int scheduler = DG_SCHED_BALANCED;
  double threshold = 0.1;
  int nQmax = 0, wpb = 2, blocks_per_sm = 1, num_sms = 1;
  // Navier-Stokes (BR1): off until dg_set_physics; buffers allocated then
  int ns = 0, blocks_per_sm_ns = 1;
  double mu = 0.0, Pr = 0.72;
  double *d_Unod = nullptr, *d_L = nullptr, *d_Vt = nullptr, *d_fnrm = nullptr;
  double *d_DW = nullptr, *d_Vtb = nullptr;   // Navier-Stokes adjoint workspace
  bool store_dw = false;                      // the volume phase keeps the nodal gradient (adjoint)
  bool keep_stages = true;                    // dg_rk_vjp keeps stage data (dg_set_adjoint_storage)
  double adj_mem_frac = 0.5;                  // share of the free device memory dg_rk_vjp may keep stage data in
  // Stage data kept by the forward pass of dg_rk_vjp for one segment (5 per
  // step): the nodal state and the own-side traces, plus for Navier-Stokes
  // the gradient traces and the nodal gradient.  The reverse stages then skip
  // the forward recomputation.
  double* d_sstore = nullptr;
  size_t sstore_doubles = 0;
  double* d_ckpt_q = nullptr;                 // dg_rk_vjp's own checkpoints (+ work state)
  size_t ckpt_q_doubles = 0;
  double *ov_T = nullptr, *ov_Unod = nullptr, *ov_Vt = nullptr, *ov_DW = nullptr, *ov_Usave = nullptr;
  struct StagePtrs {
    double *U, *T, *Vt, *DW;
  };
  // compact: only the nodal state (and, Navier-Stokes, the nodal gradient)
  // is kept per stage; the reverse stage rebuilds the face traces from them
  // (kTraces).  dg_rk_vjp chooses it when the whole trajectory's full stage
  // data do not fit in the memory share, so more stages are kept.
  bool compact = false;
  bool lift_done = false;   // Navier-Stokes stage-wise stepping: dg_rk_stage_lift ran for the pending stage
  size_t stage_doubles() const {
    const size_t hh = (size_t)std::max<int64_t>(1, h.h_total), tt = (size_t)std::max<int64_t>(1, h.t_total);
    if (compact) return ns ? 4 * hh : hh;
    return ns ? 4 * (hh + tt) : hh + tt;
  }
  StagePtrs stage_ptrs(int g) const {
    const size_t hh = (size_t)std::max<int64_t>(1, h.h_total), tt = (size_t)std::max<int64_t>(1, h.t_total);
    double* b = d_sstore + (size_t)g * stage_doubles();
    if (compact) return StagePtrs{b, nullptr, nullptr, ns ? b + hh : nullptr};
    StagePtrs P{b, b + hh, nullptr, nullptr};
    if (ns) {
      P.Vt = P.T + tt;
      P.DW = P.Vt + 3 * tt;
    }
    return P;
  }
  void clear_overrides() { ov_T = ov_Unod = ov_Vt = ov_DW = ov_Usave = nullptr; }
  // false when the store cannot be allocated: the caller recomputes instead
  bool ensure_stage_store(int nstages) {
    const size_t need = (size_t)nstages * stage_doubles();
    if (need <= sstore_doubles) return true;
    if (d_sstore) cudaFree(d_sstore);
    d_sstore = nullptr;
    sstore_doubles = 0;
    if (cudaMalloc(&d_sstore, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();  // clear the allocation error; fall back to recomputation
      d_sstore = nullptr;
      return false;
    }
    sstore_doubles = need;
    return true;
  }
  // device data
  double* d_dpool = nullptr;
  int* d_ipool = nullptr;
  dgk::TypeTab* d_tabs = nullptr;
  int* d_slot_tab = nullptr;
  int8_t* d_slot_type = nullptr;
  int64_t *d_slot_qoff = nullptr, *d_slot_hoff = nullptr, *d_slot_ftoff = nullptr;
  int64_t *d_elem_of_slot = nullptr, *d_elem_qoff = nullptr, *d_elem_voff = nullptr;
  dgk::ElemGeo* d_geo = nullptr;
  int64_t* d_slot_coff = nullptr;
  double *d_cpool = nullptr, *d_fgeo = nullptr, *d_snrm = nullptr;
  double* d_H = nullptr;
  double* d_T = nullptr;
  double* d_Tv = nullptr;       // adjoint face buffer
  double* d_Kbar = nullptr;     // adjoint LSERK register
  double* d_ckpt = nullptr;     // dg_rk_vjp checkpoints / stage states
  size_t ckpt_doubles = 0;
  dgk::FaceRec* d_faces = nullptr;
  dgk::FaceBlock* d_fblocks = nullptr;
  int16_t* d_perms = nullptr;
  double* d_dense = nullptr;
  unsigned* d_status = nullptr;
  unsigned long long* d_cost = nullptr;
  unsigned long long* d_smns = nullptr;
  unsigned* d_counters = nullptr;
  int64_t* d_type_slots[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t* d_chunks_static = nullptr;
  int64_t nchunks_static = 0;
  int64_t* d_chunks_weighted = nullptr;   // equal-weight Hilbert segments (DG_SCHED_WEIGHTED)
  int64_t nchunks_weighted = 0;
  bool fused = true;  // backward of stage s and forward of stage s+1 in one launch
  // automatic imbalance trigger of dg_rk_step (dg_set_rebalance_interval)
  int rebalance_every = 0, steps_since_check = 0;
  int64_t rebalances = 0, checks = 0;
  double weight[dgk::kMaxTabs] = {};  // chunk weights in use per (type, N) table (ns or modelled)

  std::vector<double> static_weights() const {
    std::vector<double> w(dgk::kMaxTabs, 1.0);
    for (size_t i = 0; i < h.tables.tabs.size() && i < (size_t)dgk::kMaxTabs; ++i) {
      const dgk::TypeTab& t = h.tables.tabs[i];
      w[i] = dgh::static_cost(t);
      // split form: every coordinate line's node pairs and face pairs, each
      // a two-point flux of about 100 FP64 operations
      if (split && t.type == dgk::HEX) w[i] += 3.0 * t.n * t.n * (t.n * (t.n - 1) + 4.0 * t.n) * 100.0;
    }
    return w;
  }
  double* d_stage = nullptr;
  // graph cache for dg_rk_step.  Without profiling: three graphs captured
  // once and replayed for any state, register, dt and step count -- prime
  // (parameter node, forward of stage 1), step (five stages ending in the
  // next step's forward) and last (five stages) -- whose element launches
  // read (Q, K, dt) from d_rkdyn; only the parameter node's arguments change
  // between calls.  With profiling: one graph of the whole call (its event
  // nodes time the phases), captured again when an argument changes.
  cudaStream_t cap = nullptr;
  dgk::RkDyn* d_rkdyn = nullptr;
  struct Captured {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
  };
  Captured gr_prime, gr_step, gr_last;
  cudaGraphNode_t gr_param_node = nullptr;
  int64_t graph_captures = 0;
  cudaGraphExec_t gexec = nullptr;
  const double* g_Q = nullptr;
  const double* g_K = nullptr;
  double g_dt = 0.0;
  int g_nsteps = -1, g_sched = -1, g_fused = -1;
  int r_sched = -1, r_fused = -1;   // configuration of the three replayed graphs

  void drop_graphs() {
    for (Captured* c : {&gr_prime, &gr_step, &gr_last}) {
      if (c->x) cudaGraphExecDestroy(c->x);
      if (c->g) cudaGraphDestroy(c->g);
      c->x = nullptr;
      c->g = nullptr;
    }
    gr_param_node = nullptr;
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }

  template <class F>
  cudaError_t capture(Captured& c, F&& body) {
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    body(cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&c.x, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return e;
    }
    c.g = g;   // kept: the parameter node handle refers to it
    return cudaSuccess;
  }

  // The three replayed graphs of dg_rk_step (profiling off).
  cudaError_t capture_stage_graphs() {
    drop_graphs();
    dgk::StageArgs a{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0, d_rkdyn};
    auto stages = [&](cudaStream_t st, bool last_step) {
      cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
      parity = 0;
      for (int s = 0; s < 5; ++s) {
        face_phase(st);
        const bool last = last_step && s == 4;
        a.a = kLsA[s];
        a.b = kLsB[s];
        if (fused) {
          element_phase(last ? dgk::kBwdRk : dgk::kBwdRkFwd, a, st);
        } else {
          element_phase(dgk::kBwdRk, a, st);
          if (!last) element_phase(dgk::kFwd, a, st);
        }
      }
    };
    cudaError_t e = capture(gr_prime, [&](cudaStream_t st) {
      dgk::launch_rk_params(d_rkdyn, nullptr, nullptr, 0.0, st);
      cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
      parity = 0;
      element_phase(dgk::kFwd, a, st);
    });
    if (e == cudaSuccess) e = capture(gr_step, [&](cudaStream_t st) { stages(st, false); });
    if (e == cudaSuccess) e = capture(gr_last, [&](cudaStream_t st) { stages(st, true); });
    if (e != cudaSuccess) {
      drop_graphs();
      return e;
    }
    size_t n = 0;
    e = cudaGraphGetNodes(gr_prime.g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(gr_prime.g, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n && !gr_param_node; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
      cudaKernelNodeParams kp{};
      if (cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess && dgk::is_rk_params_kernel(kp.func))
        gr_param_node = nodes[i];
    }
    if (e == cudaSuccess && !gr_param_node) e = cudaErrorGraphExecUpdateFailure;
    if (e != cudaSuccess) {
      drop_graphs();
      return e;
    }
    r_sched = scheduler;
    r_fused = (int)fused;
    ++graph_captures;
    return cudaSuccess;
  }
  int parity = 0;
  // phase timing events: pool 0 for captured graphs, pool 1 for direct calls
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool[2];
  int ev_used[2] = {0, 0};
  int pool = 1;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_elem[2], ev_face[2];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_geom, ev_mass;   // moving meshes (direct launches)
  int last_pool = -1;

  cudaEvent_t next_event() {
    if (ev_used[pool] == (int)ev_pool[pool].size()) {
      cudaEvent_t e = nullptr;
      cudaEventCreate(&e);
      ev_pool[pool].push_back(e);
    }
    return ev_pool[pool][ev_used[pool]++];
  }
  void begin_timing(int which) {
    pool = which;
    ev_used[pool] = 0;
    ev_elem[pool].clear();
    ev_face[pool].clear();
    if (which == 1) {
      ev_geom.clear();
      ev_mass.clear();
    }
    last_pool = which;
  }
  template <class F>
  void timed(bool elem, cudaStream_t st, F&& f) {
    if (!profiling) { f(); return; }
    cudaEvent_t a = next_event(), b = next_event();
    // inside a stream capture a plain record is only a dependency marker;
    // the external flag makes it an event-record node of the graph
    const unsigned flags = pool == 0 ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaEventRecordWithFlags(a, st, flags);
    f();
    cudaEventRecordWithFlags(b, st, flags);
    (elem ? ev_elem[pool] : ev_face[pool]).push_back({a, b});
  }
  // the same around a moving mesh's geometry (mass = false) or mass kernels
  template <class F>
  auto timed_moving(bool mass, cudaStream_t st, F&& f) -> decltype(f()) {
    if (!profiling) return f();
    cudaEvent_t a = next_event(), b = next_event();
    cudaEventRecord(a, st);
    auto r = f();
    cudaEventRecord(b, st);
    (mass ? ev_mass : ev_geom).push_back({a, b});
    return r;
  }

  dgk::Ctx ctx() const {
    dgk::Ctx c;
    c.dpool = d_dpool;
    c.ipool = d_ipool;
    c.tabs = d_tabs;
    c.slot_tab = d_slot_tab;
    c.slot_type = d_slot_type;
    c.slot_qoff = d_slot_qoff;
    c.slot_hoff = d_slot_hoff;
    c.slot_ftoff = d_slot_ftoff;
    c.elem_of_slot = d_elem_of_slot;
    c.elem_qoff = d_elem_qoff;
    c.elem_voff = d_elem_voff;
    c.geo = d_geo;
    c.slot_coff = h.n_curved ? d_slot_coff : nullptr;
    c.cpool = d_cpool;
    c.fgeo = d_fgeo;
    c.snrm = d_snrm;
    c.ns = ns;
    c.mu = mu;
    c.kappa = ns ? mu * gamma / ((gamma - 1.0) * Pr) : 0.0;
    c.fnrm = d_fnrm;
    c.Unod = ov_Unod ? ov_Unod : d_Unod;
    c.L = d_L;
    c.Vt = ov_Vt ? ov_Vt : d_Vt;
    c.DW = ov_DW ? ov_DW : (store_dw ? d_DW : nullptr);
    c.Usave = ov_Usave;
    c.Vtb = d_Vtb;
    c.H = d_H;
    c.T = ov_T ? ov_T : d_T;
    c.Tv = d_Tv;
    c.faces = d_faces;
    c.fblocks = d_fblocks;
    c.perms = d_perms;
    c.dense = d_dense;
    c.status = d_status;
    c.cost = d_cost;
    c.sm_ns = d_smns;
    c.gamma = gamma;
    c.flux = flux;
    c.split = split;
    c.nQmax = nQmax;
    if (moving) {
      c.mpool = d_mpool;
      c.slot_moff = d_slot_moff;
      c.fmot = d_fmot;
      c.mk32 = d_mk32;
      c.slot_mmoff = d_slot_mmoff;
      // phase 1 writes the lifting residuals, phase 2 reads the gradients
      c.lift = lift_phase == 2 ? d_G : d_lift;
      c.lift_stride = h.n_dof;
      c.lift_phase = lift_phase;
    }
    return c;
  }

  // ---- moving meshes
  void moving_geometry(double t, cudaStream_t st) {
    timed_moving(false, st, [&] {
      // HBM-bound: enough blocks in flight to cover the loads' latency
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h.n_elems, (int64_t)num_sms * 32));
      dgk::launch_moving_geometry(ctx(), d_cpool, d_fgeo, ns ? d_snrm : nullptr, h.n_elems, h.n_faces, h.n, t, grid,
                                  st);
      return 0;
    });
  }
  // one launch per element type, each with the shared memory its own mass
  // matrices need
  cudaError_t moving_mass(const double* in, double* out, const double tau[4], int weight, cudaStream_t st,
                          const double* x0 = nullptr, bool dense_only = false, int nblk = 1,
                          float* fac_out = nullptr, const float* fac_in = nullptr) {
    return timed_moving(true, st, [&] {
      return moving_mass_launches(in, out, x0, tau, weight, st, dense_only, nblk, fac_out, fac_in);
    });
  }
  cudaError_t moving_mass_launches(const double* in, double* out, const double* x0, const double tau[4], int weight,
                                   cudaStream_t st, bool dense_only, int nblk, float* fac_out, const float* fac_in) {
    const dgk::Ctx c = ctx();
    for (int t = dense_only ? 1 : 0; t < 3; ++t) {
      const int64_t cnt = (int64_t)h.type_slots[t].size();
      if (!cnt) continue;
      int nM = 0, nQ = 0;
      if (t != dgk::HEX)
        for (const auto& T : h.tables.tabs)
          if (T.type == t) {
            nM = std::max(nM, T.nM);
            nQ = std::max(nQ, T.nQ);
          }
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(cnt, (int64_t)num_sms * 8));
      cudaError_t e = dgk::launch_moving_mass(c, d_type_slots[t], cnt, in, out, x0, tau, weight, nM, nQ, grid, st,
                                              nblk, h.n_dof, fac_out, fac_in);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static void powers(double t, double tau[4]) {
    tau[0] = 1.0;
    tau[1] = t;
    tau[2] = t * t;
    tau[3] = t * t * t;
  }
  // Whether the stage values y_k lie within tol of t^k (relative to
  // max(1, |t|)^k).  1e-6: a factor of M^ built from y_k can stand in for
  // one of M(t) in the lifting solves (M^ - M(t) stays near the factor's
  // FP32 rounding for mesh velocity gradients up to about 10, and two
  // corrections from the previous stage's gradients still reach FP64
  // rounding).  1e-14: the Ut a step leaves can be carried into the next
  // step in place of M(t + dt) Q (the scheme integrates t^k exactly up to
  // the accuracy of its published coefficients, about 1e-15 at the
  // benchmark's dt but 1e-11 at dt = 0.05, t = 1).
  static bool stage_values_near(const double y[4], double t, double tol) {
    double tau[4];
    powers(t, tau);
    const double sc = std::max(1.0, std::fabs(t));
    double s = 1.0;
    for (int k = 1; k < 4; ++k) {
      s *= sc;
      if (!(std::fabs(y[k] - tau[k]) <= tol * s)) return false;
    }
    return true;
  }
  // The face phase of a moving mesh at time ts.  Navier-Stokes: the lifting
  // values, then the volume phase in two halves around the lifting's
  // M(ts)^{-1} for prisms and pyramids (three solves of five variables, the
  // lifting residual of direction d in d_lift + d n_dof), then the flux.
  cudaError_t moving_face_phase(double ts, cudaStream_t st) {
    if (!ns) {
      face_phase(st);
      return cudaSuccess;
    }
    const int64_t nb = (int64_t)h.face_blocks.size();
    timed(false, st, [&] { dgk::launch_faces_ns(ctx(), nb, h.n, 0, st); });
    dgk::StageArgs none{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
    lift_phase = 1;
    element_phase(dgk::kNsVolume, none, st);
    double tau[4];
    powers(ts, tau);
    // the three directions with one factor of M(ts) per element -- the one
    // the stage's state solve kept, whose matrix M^ of the stage values y_k
    // differs from M(ts) by the stages' error in integrating t^k (about
    // dt^2, far below the factor's FP32 rounding) -- started from the
    // previous stage's gradients (one correction fewer) once this call has
    // them
    cudaError_t e = moving_mass(d_lift, d_G, tau, 0, st, G_warm ? d_G : nullptr, true, 3, nullptr,
                                fac_ready ? d_fac : nullptr);
    G_warm = true;
    lift_phase = 2;
    element_phase(dgk::kNsVolume, none, st);
    lift_phase = 0;
    timed(false, st, [&] { dgk::launch_faces_ns(ctx(), nb, h.n, 1, st); });
    return e;
  }
  // Residual at the mesh time: M(t)^{-1} (vol - surf).
  cudaError_t moving_rhs(const double* Q, double* R, cudaStream_t st) {
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
    parity = 0;
    G_warm = false;
    fac_ready = false;
    moving_geometry(t_mesh, st);
    dgk::StageArgs a{Q, R, nullptr, 0.0, 0.0, 0.0};
    element_phase(dgk::kFwd, a, st);
    cudaError_t e = moving_face_phase(t_mesh, st);
    if (e != cudaSuccess) return e;
    element_phase(dgk::kBwdRhs, a, st);
    double tau[4];
    powers(t_mesh, tau);
    return moving_mass(R, R, tau, 0, st);
  }
  // LSERK(5,4) steps of the mass-weighted state Ut = M Q (K: its register).
  // Stage s evaluates the residual at t_s = t + c_s dt on the geometry of
  // t_s, from the stage state M^_s^{-1} Ut with M^_s built from the stage
  // values y_k of t^k, which run through the same 2N-storage recursion
  // (dy_k/dt = k t^(k-1)).  The product Ut = M(t) Q runs at the first step
  // of a call and after any step whose y_k end away from the powers of
  // t + dt: a fourth-order scheme integrates k t^(k-1) (degree <= 2)
  // exactly, so otherwise the Ut a step leaves is M(t + dt) Q_{n+1} up to
  // the rounding of the end-of-step solve -- the next step's product would
  // only reproduce it.
  cudaError_t moving_rk(double* Q, double* K, double dt, int nsteps, cudaStream_t st) {
    static const double kLsC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363183857.0,
                                   2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
    cudaError_t e = cudaSuccess;
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
    parity = 0;
    G_warm = false;   // a caller may change the state between calls
    fac_ready = false;
    float* keep = ns ? d_fac : nullptr;
    bool carry = false;   // d_Ut holds M(t) Q of the step about to start
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
      const double t = t_mesh;
      double y[4], Ky[4] = {0.0, 0.0, 0.0, 0.0};
      powers(t, y);
      if (!carry && (e = moving_mass(Q, d_Ut, y, 1, st)) != cudaSuccess) return e;
      for (int s = 0; s < 5; ++s) {
        const double ts = t + kLsC[s] * dt;
        moving_geometry(ts, st);
        // the first stage's state is Q itself (its solve would undo the
        // product above up to rounding)
        // later stages start their solve from the previous stage's state
        if (s > 0) {
          if ((e = moving_mass(d_Ut, d_S, y, 0, st, s == 1 ? Q : d_S, false, 1, keep)) != cudaSuccess) return e;
          fac_ready = keep != nullptr && stage_values_near(y, ts, 1e-6);
        }
        dgk::StageArgs f{s > 0 ? d_S : Q, nullptr, nullptr, 0.0, 0.0, 0.0};
        element_phase(dgk::kFwd, f, st);
        if ((e = moving_face_phase(ts, st)) != cudaSuccess) return e;
        dgk::StageArgs a{d_Ut, d_Ut, K, kLsA[s], kLsB[s], dt};
        element_phase(dgk::kBwdRk, a, st);
        const double dp[4] = {0.0, 1.0, 2.0 * ts, 3.0 * ts * ts};
        for (int k = 0; k < 4; ++k) {
          Ky[k] = kLsA[s] * Ky[k] + dt * dp[k];
          y[k] += kLsB[s] * Ky[k];
        }
      }
      // the step's end: y_k are the powers of t + dt, so its factor serves
      // the next step's first lifting as well
      if ((e = moving_mass(d_Ut, Q, y, 0, st, d_S, false, 1, keep)) != cudaSuccess) return e;
      fac_ready = keep != nullptr && stage_values_near(y, t + dt, 1e-6);
      carry = stage_values_near(y, t + dt, 1e-14);
      t_mesh = t + dt;
    }
    return cudaGetLastError();
  }

  bool ghost_slot(int64_t s) const { return !h.slot_ghost.empty() && h.slot_ghost[s]; }

  int grid_balanced() const { return num_sms * blocks_per_sm; }
  int grid_ns() const { return num_sms * blocks_per_sm_ns; }

  // Launch groups of the balanced scheduler: the (type, N) tables present in
  // the mesh, grouped by (n, warps per element).  Every group is one
  // persistent launch per phase with its own block size, shared memory
  // (n^3-sized buffers) and grid, so the tile shape can differ per table
  // (dg_autotune chooses it per table).
  struct Group {
    int n = 0, wpb = 1, bpsm = 1, bpsm_ns = 1;
    std::vector<int> tabs;
    int64_t* d_chunks = nullptr;
    int64_t* d_list = nullptr;
    int64_t nchunks = 0;
  };
  std::vector<Group> groups;
  int tab_wpb[dgk::kMaxTabs] = {};

  void free_groups() {
    for (auto& G : groups) {
      if (G.d_chunks) cudaFree(G.d_chunks);
      if (G.d_list) cudaFree(G.d_list);
    }
    groups.clear();
  }

  cudaError_t build_groups() {
    free_groups();
    std::vector<int64_t> count(h.tables.tabs.size(), 0);
    for (int64_t s = 0; s < h.n_elems; ++s)
      if (!ghost_slot(s)) ++count[h.slot_tab[s]];
    for (size_t t = 0; t < h.tables.tabs.size(); ++t) {
      if (!count[t]) continue;
      const int n = h.tables.tabs[t].n, w = tab_wpb[t];
      auto it = std::find_if(groups.begin(), groups.end(), [&](const Group& G) { return G.n == n && G.wpb == w; });
      if (it == groups.end()) {
        Group G;
        G.n = n;
        G.wpb = w;
        groups.push_back(G);
        it = groups.end() - 1;
      }
      it->tabs.push_back((int)t);
    }
    for (auto& G : groups) {
      cudaError_t e = dgk::element_kernel_attributes(G.n * G.n * G.n, G.wpb, &G.bpsm, h.n_curved > 0, split != 0);
      if (e != cudaSuccess) return e;
      if (G.bpsm < 1) G.bpsm = 1;
      if (ns) {
        e = dgk::element_kernel_attributes_ns(G.n * G.n * G.n, G.wpb, &G.bpsm_ns, h.n_curved > 0);
        if (e != cudaSuccess) return e;
        if (G.bpsm_ns < 1) G.bpsm_ns = 1;
      }
    }
    // restore the mesh-wide attributes used by the static and naive launches
    cudaError_t e = dgk::element_kernel_attributes(nQmax, wpb, &blocks_per_sm, h.n_curved > 0, split != 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    std::vector<double> w(weight, weight + dgk::kMaxTabs);
    return build_chunks(w.data());
  }

  // Balanced work list of every group: the Hilbert order grouped by (type,
  // N) table (every table's elements stay in Hilbert order), tables in
  // decreasing cost per element, cut into contiguous chunks by guided
  // self-scheduling on the measured (or modelled) cost: each chunk takes a
  // fixed fraction of the group's work still unassigned, so chunks are large
  // at first and single elements at the end, where they set the length of
  // the tail.  A chunk never spans two tables.
  cudaError_t build_chunks(const double* tab_weight) {
    const int64_t E = h.n_elems;
    for (int t = 0; t < dgk::kMaxTabs; ++t) weight[t] = tab_weight[t];
    for (auto& G : groups) {
      std::vector<int> order = G.tabs;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tab_weight[x] > tab_weight[y]; });
      std::vector<int64_t> list;
      for (int t : order)
        for (int64_t s = 0; s < E; ++s)
          if (h.slot_tab[s] == t && !ghost_slot(s)) list.push_back(s);
      const int64_t L = (int64_t)list.size();
      double remaining = 0.0;
      for (int64_t s : list) remaining += tab_weight[h.slot_tab[s]];
      const double blocks = (double)std::max(1, num_sms * G.bpsm);
      std::vector<int64_t> starts;
      starts.push_back(0);
      double acc = 0.0, target = remaining / (2.0 * blocks);
      for (int64_t i = 0; i < L; ++i) {
        const double w = tab_weight[h.slot_tab[list[i]]];
        acc += w;
        remaining -= w;
        bool tab_end = i + 1 < L && h.slot_tab[list[i + 1]] != h.slot_tab[list[i]];
        if (i + 1 < L && (acc >= target || tab_end)) {
          starts.push_back(i + 1);
          acc = 0.0;
          target = remaining / (2.0 * blocks);
        }
      }
      starts.push_back(L);
      G.nchunks = (int64_t)starts.size() - 1;
      if (G.d_chunks) cudaFree(G.d_chunks);
      if (G.d_list) cudaFree(G.d_list);
      G.d_chunks = G.d_list = nullptr;
      cudaError_t e = upload(&G.d_chunks, starts);
      if (e != cudaSuccess) return e;
      e = upload(&G.d_list, list);
      if (e != cudaSuccess) return e;
    }
    return build_static_chunks();
  }

  // Static partitions, one contiguous Hilbert segment per resident block:
  // of equal element count (the paper's partition without load balancing,
  // DG_SCHED_STATIC), and of equal weight with the current per-(type, N)
  // weights (the paper's load-balanced partition, Sec. 3: weights from the
  // timers once dg_rebalance has read them, DG_SCHED_WEIGHTED).
  cudaError_t build_static_chunks() {
    const int64_t E = h.n_elems;
    int64_t W = std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)grid_balanced()));
    std::vector<int64_t> starts(W + 1);
    for (int64_t w = 0; w <= W; ++w) starts[w] = w * E / W;
    nchunks_static = W;
    if (d_chunks_static) cudaFree(d_chunks_static);
    d_chunks_static = nullptr;
    cudaError_t e = upload(&d_chunks_static, starts);
    if (e != cudaSuccess) return e;
    // equal-weight cuts of the prefix sum of the slots' weights
    double total = 0.0;
    for (int64_t s = 0; s < E; ++s) total += weight[h.slot_tab[s]];
    std::vector<int64_t> ws(1, 0);
    double acc = 0.0;
    for (int64_t s = 0; s < E && (int64_t)ws.size() < W; ++s) {
      acc += weight[h.slot_tab[s]];
      if (acc >= total * (double)ws.size() / (double)W) ws.push_back(s + 1);
    }
    ws.push_back(E);
    nchunks_weighted = (int64_t)ws.size() - 1;
    if (d_chunks_weighted) cudaFree(d_chunks_weighted);
    d_chunks_weighted = nullptr;
    return upload(&d_chunks_weighted, ws);
  }

  // Hexahedra are stored as scaled nodal values W^{1/2} V Q (an orthogonal
  // change of basis; the other types hold their modal coefficients): after
  // the permutation of every element block, kGather / kScatter rewrite the
  // hexahedra's blocks with the converted values.
  void convert_hex(int mode, const double* src, double* dst, cudaStream_t st) const {
    if (h.type_slots[dgk::HEX].empty()) return;
    dgk::StageArgs a{src, dst, nullptr, 0.0, 0.0, 0.0};
    dgk::Sched s{d_type_slots[dgk::HEX], (int64_t)h.type_slots[dgk::HEX].size(), nullptr, nullptr, nullptr};
    dgk::launch_element(ctx(), mode, a, s, false, 0, wpb, st);
  }

  void element_phase(int mode, const dgk::StageArgs& a, cudaStream_t st) {
    dgk::Ctx c = ctx();
    timed(true, st, [&] {
      const bool per_elem = mode == dgk::kProject || mode == dgk::kEval || mode == dgk::kLoad ||
                            mode == dgk::kTraces;   // one-shot maps
      if (scheduler == DG_SCHED_BALANCED && !per_elem) {
        for (const auto& G : groups) {
          dgk::Ctx cg = c;
          cg.nQmax = G.n * G.n * G.n;
          dgk::Sched s{G.d_list, G.nchunks, G.d_chunks, d_counters + parity, d_counters + (parity ^ 1)};
          dgk::launch_element(cg, mode, a, s, true, num_sms * (mode == dgk::kNsVolume ? G.bpsm_ns : G.bpsm), G.wpb,
                              st);
          parity ^= 1;
        }
      } else if ((scheduler == DG_SCHED_STATIC || scheduler == DG_SCHED_WEIGHTED) && !per_elem) {
        const bool wt = scheduler == DG_SCHED_WEIGHTED;
        dgk::Sched s{nullptr, wt ? nchunks_weighted : nchunks_static, wt ? d_chunks_weighted : d_chunks_static,
                     d_counters + parity, d_counters + (parity ^ 1)};
        dgk::launch_element(c, mode, a, s, true, mode == dgk::kNsVolume ? grid_ns() : grid_balanced(), wpb, st);
        parity ^= 1;
      } else {
        for (int t = 0; t < 4; ++t) {
          if (h.type_slots[t].empty()) continue;
          dgk::Sched s{d_type_slots[t], (int64_t)h.type_slots[t].size(), nullptr, nullptr, nullptr};
          dgk::launch_element(c, mode, a, s, false, 0, wpb, st);
        }
      }
    });
  }

  // Face phase of one residual evaluation.  Navier-Stokes inserts the BR1
  // lifting (face values of W*, then the element volume phase that lifts the
  // gradient and forms the volume residual) before the flux face kernel.
  void face_phase(cudaStream_t st) {
    const int64_t nb = (int64_t)h.face_blocks.size();
    if (ns) {
      timed(false, st, [&] { dgk::launch_faces_ns(ctx(), nb, h.n, 0, st); });
      dgk::StageArgs none{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
      element_phase(dgk::kNsVolume, none, st);
      timed(false, st, [&] { dgk::launch_faces_ns(ctx(), nb, h.n, 1, st); });
      return;
    }
    timed(false, st, [&] { dgk::launch_faces(ctx(), nb, h.n, st); });
  }

  // Enqueue nsteps LSERK steps (no synchronisation).
  // Adjoint workspace (allocated on first use).
  cudaError_t ensure_adjoint(size_t ckpt_needed) {
    cudaError_t e = cudaSuccess;
    if (ns) {
      const size_t hb = sizeof(double) * (size_t)std::max<int64_t>(1, h.h_total);
      const size_t tb = sizeof(double) * (size_t)std::max<int64_t>(1, h.t_total);
      if (!d_DW && (e = cudaMalloc(&d_DW, 3 * hb)) != cudaSuccess) return e;
      if (!d_Vtb && (e = cudaMalloc(&d_Vtb, 3 * tb)) != cudaSuccess) return e;
    }
    if (!d_Tv && (e = cudaMalloc(&d_Tv, sizeof(double) * std::max<int64_t>(1, h.t_total))) != cudaSuccess) return e;
    if (!d_Kbar && (e = cudaMalloc(&d_Kbar, sizeof(double) * std::max<int64_t>(1, h.n_dof))) != cudaSuccess) return e;
    if (ckpt_needed > ckpt_doubles) {
      if (d_ckpt) cudaFree(d_ckpt);
      d_ckpt = nullptr;
      ckpt_doubles = 0;
      if ((e = cudaMalloc(&d_ckpt, sizeof(double) * ckpt_needed)) != cudaSuccess) return e;
      ckpt_doubles = ckpt_needed;
    }
    return e;
  }

  // One RHS VJP (rk == 0) or one reverse LSERK stage (rk == 1) at state Q.
  // stage >= 0: the forward data of that stage of the store are used instead
  // of recomputing them from va.Q.
  void enqueue_vjp(dgk::VjpArgs va, cudaStream_t st, int stage = -1) {
    if (stage >= 0) {
      const StagePtrs P = stage_ptrs(stage);
      ov_T = P.T;
      ov_Unod = P.U;
      ov_Vt = P.Vt;
      ov_DW = P.DW;
      va.stored = 1;
      if (compact) {
        // traces into the mesh's own face buffers (T, and Vt for Navier-Stokes)
        dgk::StageArgs none{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
        element_phase(dgk::kTraces, none, st);
      }
    }
    const int64_t nb = (int64_t)h.face_blocks.size();
    if (ns) {
      if (stage < 0) {
        // forward state at Q (traces, nodal state, lifting values, gradient
        // traces and the nodal gradient), then the transposed phases
        dgk::StageArgs fa{va.Q, nullptr, nullptr, 0.0, 0.0, 0.0};
        store_dw = true;
        element_phase(dgk::kFwd, fa, st);
        dgk::launch_faces_ns(ctx(), nb, h.n, 0, st);
        element_phase(dgk::kNsVolume, fa, st);
      }
      dgk::Ctx c = ctx();
      store_dw = false;
      dgk::launch_vjp(c, 10, va, h.n_elems, wpb, st);
      dgk::launch_faces_ns_vjp(c, nb, h.n, 1, st);
      dgk::launch_vjp(c, 11, va, h.n_elems, wpb, st);
      dgk::launch_faces_ns_vjp(c, nb, h.n, 0, st);
      dgk::launch_vjp(c, 2, va, h.n_elems, wpb, st);
      clear_overrides();
      return;
    }
    dgk::Ctx c = ctx();
    dgk::launch_vjp(c, 0, va, h.n_elems, wpb, st);
    dgk::launch_faces_vjp(c, nb, h.n, st);
    dgk::launch_vjp(c, 2, va, h.n_elems, wpb, st);
    clear_overrides();
  }

  // Forward LSERK steps from Q (in place) with the stage inputs copied to
  // `stages` (5 per step) when non-null.  Non-captured launches.
  // keep: fill the stage store (stage g = 5 step + s) for enqueue_vjp.
  // final_update = false: the state after the last stage is not needed (a
  // segment pass of the reverse sweep), so the last stage stops once its
  // stage data exist.
  void enqueue_rk_stages(double* Q, double* K, double dt, int nsteps, double* stages, cudaStream_t st,
                         bool keep = false, bool final_update = true) {
    const size_t bytes = sizeof(double) * h.n_dof;
    const size_t tbytes = sizeof(double) * (size_t)std::max<int64_t>(1, h.t_total);
    auto keep_forward = [&](int g) {
      if (!keep) return;
      if (ns) ov_Unod = stage_ptrs(g).U;
      else ov_Usave = stage_ptrs(g).U;
    };
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
    parity = 0;
    dgk::StageArgs a{Q, Q, K, 0.0, 0.0, dt};
    keep_forward(0);
    element_phase(dgk::kFwd, a, st);
    clear_overrides();
    for (int step = 0; step < nsteps; ++step)
      for (int s = 0; s < 5; ++s) {
        const int g = 5 * step + s;
        if (stages) cudaMemcpyAsync(stages + (size_t)g * h.n_dof, Q, bytes, cudaMemcpyDeviceToDevice, st);
        if (keep) {
          const StagePtrs P = stage_ptrs(g);
          if (P.T) cudaMemcpyAsync(P.T, d_T, tbytes, cudaMemcpyDeviceToDevice, st);
          if (ns) {
            ov_Unod = P.U;
            ov_Vt = P.Vt;
            ov_DW = P.DW;
          }
        }
        bool last = step == nsteps - 1 && s == 4;
        if (last && !final_update) {
          // only the Navier-Stokes stage data of the volume phase are still
          // missing (with kept stage data); nothing else is read later
          if (ns && keep) {
            timed(false, st, [&] { dgk::launch_faces_ns(ctx(), (int64_t)h.face_blocks.size(), h.n, 0, st); });
            dgk::StageArgs none{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
            element_phase(dgk::kNsVolume, none, st);
          }
          clear_overrides();
          return;
        }
        face_phase(st);
        clear_overrides();
        a.a = kLsA[s];
        a.b = kLsB[s];
        if (!last) keep_forward(g + 1);
        element_phase(last ? dgk::kBwdRk : dgk::kBwdRkFwd, a, st);
        clear_overrides();
      }
  }

  void enqueue_rk(double* Q, double* K, double dt, int nsteps, cudaStream_t st) {
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned), st);
    parity = 0;
    dgk::StageArgs a{Q, Q, K, 0.0, 0.0, dt};
    element_phase(dgk::kFwd, a, st);
    for (int step = 0; step < nsteps; ++step)
      for (int s = 0; s < 5; ++s) {
        face_phase(st);
        bool last = step == nsteps - 1 && s == 4;
        a.a = kLsA[s];
        a.b = kLsB[s];
        if (fused) {
          element_phase(last ? dgk::kBwdRk : dgk::kBwdRkFwd, a, st);
        } else {
          element_phase(dgk::kBwdRk, a, st);
          if (!last) element_phase(dgk::kFwd, a, st);
        }
      }
  }

  void release() {
    void* ptrs[] = {d_dpool, d_ipool, d_tabs, d_slot_tab, d_slot_type, d_slot_qoff, d_slot_hoff, d_slot_ftoff,
                    d_elem_of_slot, d_elem_qoff, d_elem_voff, d_geo, d_H, d_T, d_faces, d_fblocks, d_perms, d_dense, d_status,
                    d_cost, d_smns, d_counters, d_chunks_static, d_chunks_weighted, d_stage,
                    d_Tv, d_Kbar, d_ckpt, d_Unod, d_L, d_Vt, d_fnrm, d_DW, d_Vtb, d_sstore, d_ckpt_q,
                    d_slot_coff, d_cpool, d_fgeo, d_snrm, d_slot_moff, d_mpool, d_fmot, d_Ut, d_S, d_slot_mmoff,
                    d_mk32, d_lift, d_G, d_fac};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    for (auto& p : d_type_slots)
      if (p) cudaFree(p);
    free_groups();
    for (auto& pl : ev_pool)
      for (auto e : pl) cudaEventDestroy(e);
    drop_graphs();
    if (d_rkdyn) cudaFree(d_rkdyn);
    if (d_send_off) cudaFree(d_send_off);
    if (d_recv_off) cudaFree(d_recv_off);
    if (cap) cudaStreamDestroy(cap);
  }
};

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// Calls that evaluate a whole residual in one go cannot run on a partition
// mesh (its ghost traces need the halo exchange between phases).
bool part_mesh(const dg_mesh* m) { return m && m->nparts > 0; }

dg_status check_desc(const dg_mesh_desc* desc) {
  if (desc->flux != DG_FLUX_LF && desc->flux != DG_FLUX_ROE && desc->flux != DG_FLUX_EC)
    return fail(DG_ERR_ARG, "unknown flux");
  if (desc->scheduler < DG_SCHED_BALANCED || desc->scheduler > DG_SCHED_WEIGHTED) return fail(DG_ERR_ARG, "unknown scheduler");
  if (!(desc->gamma > 1.0)) return fail(DG_ERR_ARG, "gamma must exceed 1");
  return DG_OK;
}

dgh::MeshInput input_of(const dg_mesh_desc* d) {
  return dgh::MeshInput{d->n_vertices, d->xyz, d->n_elems, d->type, d->elem_vert_off, d->elem_verts, d->period, d->N,
                        d->geometry};
}

dg_status create_device_mesh(dg_mesh* m, const dg_mesh_desc* desc, cudaStream_t stream, dg_mesh** out);

}  // namespace

extern "C" {

dg_status dg_mesh_create(const dg_mesh_desc* desc, cudaStream_t stream, dg_mesh** out) {
  if (!desc || !out) return fail(DG_ERR_ARG, "null argument");
  *out = nullptr;
  dg_status st = check_desc(desc);
  if (st != DG_OK) return st;
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) return fail(DG_ERR_CUDA, "no CUDA device available (the library has no CPU path)");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  std::string err;
  int r = dgh::build_mesh(input_of(desc), &m->h, &err);
  if (r != 0) {
    delete m;
    return fail((dg_status)r, err);
  }
  return create_device_mesh(m, desc, stream, out);
}

dg_status dg_mesh_create_moving(const dg_mesh_desc* desc, const double* vertex_velocity, cudaStream_t stream,
                                dg_mesh** out) {
  if (!desc || !vertex_velocity || !out) return fail(DG_ERR_ARG, "null argument");
  *out = nullptr;
  dg_status st = check_desc(desc);
  if (st != DG_OK) return st;
  if (desc->flux != DG_FLUX_LF) return fail(DG_ERR_UNSUPPORTED, "a moving mesh takes the LF flux");
  for (int64_t v = 0; v < 3 * desc->n_vertices; ++v)
    if (!std::isfinite(vertex_velocity[v])) return fail(DG_ERR_ARG, "vertex velocities must be finite");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) return fail(DG_ERR_CUDA, "no CUDA device available (the library has no CPU path)");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  dgh::MeshInput in = input_of(desc);
  in.force_curved = 1;
  std::string err;
  int r = dgh::build_mesh(in, &m->h, &err);
  dgh::Motion mo;
  if (r == 0) r = dgh::build_motion(m->h, in, vertex_velocity, &mo, &err);
  size_t max_nM = 0;
  for (const auto& T : m->h.tables.tabs)
    if (T.type == dgk::PRISM || T.type == dgk::PYR) max_nM = std::max<size_t>(max_nM, (size_t)T.nM);
  if (r == 0 && max_nM > 128) {
    err = "the stage mass solve covers prisms and pyramids of up to 128 modes (N <= 5)";
    r = DG_ERR_UNSUPPORTED;
  }
  if (r != 0) {
    delete m;
    return fail((dg_status)r, err);
  }
  dg_mesh* made = nullptr;
  st = create_device_mesh(m, desc, stream, &made);
  if (st != DG_OK) return st;
  made->moving = true;
  const size_t bytes = sizeof(double) * (size_t)std::max<int64_t>(1, made->h.n_dof);
  // the FP32 preconditioner's coefficients: per prism and pyramid the four
  // lower triangles, packed row by row
  std::vector<float> mk32;
  std::vector<int64_t> slot_m32off(made->h.n_elems, -1);
  for (int64_t sl = 0; sl < made->h.n_elems; ++sl) {
    if (mo.slot_mmoff[sl] < 0) continue;
    const int nM = made->h.tables.tabs[made->h.slot_tab[sl]].nM;
    slot_m32off[sl] = (int64_t)mk32.size();
    for (int k = 0; k < 4; ++k) {
      const double* Mc = mo.mmat.data() + mo.slot_mmoff[sl] + (size_t)k * nM * nM;
      for (int a = 0; a < nM; ++a)
        for (int b = 0; b <= a; ++b) mk32.push_back((float)Mc[(size_t)a * nM + b]);
    }
  }
  if (mk32.empty()) mk32.push_back(0.0f);
  made->n_mk32 = (int64_t)mk32.size();
  cudaError_t e = upload(&made->d_slot_moff, mo.slot_moff);
  if (e == cudaSuccess) e = upload(&made->d_slot_mmoff, slot_m32off);
  if (e == cudaSuccess) e = upload(&made->d_mk32, mk32);
  if (e == cudaSuccess) e = upload(&made->d_mpool, mo.mpool);
  if (e == cudaSuccess) e = upload(&made->d_fmot, mo.fpool);
  if (e == cudaSuccess) e = cudaMalloc(&made->d_Ut, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&made->d_S, bytes);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    made->release();
    delete made;
    return cuda_fail(e, "moving-mesh geometry");
  }
  *out = made;
  return DG_OK;
}

dg_status dg_geometry_at(const dg_mesh_desc* desc, const double* vertex_velocity, double t, int64_t* n_elem_doubles,
                         int64_t* n_face_doubles, double* elem_geo, double* face_geo) {
  if (!desc || !n_elem_doubles || !n_face_doubles) return fail(DG_ERR_ARG, "null argument");
  if (!std::isfinite(t)) return fail(DG_ERR_ARG, "t must be finite");
  dgh::MeshInput in = input_of(desc);
  in.force_curved = 1;
  dgh::HostMesh h;
  std::string err;
  int r = dgh::build_mesh(in, &h, &err);
  if (r != 0) return fail((dg_status)r, err);
  std::vector<double> cp, fg;
  if (vertex_velocity) {
    dgh::Motion mo;
    r = dgh::build_motion(h, in, vertex_velocity, &mo, &err);
    if (r == 0) r = dgh::motion_geometry_at(h, mo, t, &cp, &fg, &err);
    if (r != 0) return fail((dg_status)r, err);
  } else {
    cp = h.cpool;
    fg = h.fgeo;
  }
  *n_elem_doubles = (int64_t)cp.size();
  *n_face_doubles = (int64_t)fg.size();
  // caller order: elements by caller index, faces by (owner, owner's local face)
  if (elem_geo) {
    size_t o = 0;
    for (int64_t e = 0; e < h.n_elems; ++e) {
      const int64_t sl = h.slot_of_elem[e];
      const size_t len = (size_t)dgh::curved_block_doubles(h.tables.tabs[h.slot_tab[sl]]);
      std::memcpy(elem_geo + o, cp.data() + h.slot_coff[sl], sizeof(double) * len);
      o += len;
    }
  }
  if (face_geo) {
    std::vector<std::tuple<int64_t, int, int64_t>> key;
    for (int64_t f = 0; f < h.n_faces; ++f)
      if (h.faces[f].cgeo >= 0) key.emplace_back(h.face_e0[f], (int)h.face_l0[f], f);
    std::sort(key.begin(), key.end());
    const size_t per = (size_t)4 * h.n * h.n;
    for (size_t k = 0; k < key.size(); ++k)
      std::memcpy(face_geo + k * per, fg.data() + h.faces[std::get<2>(key[k])].cgeo, sizeof(double) * per);
  }
  return DG_OK;
}

dg_status dg_mesh_time(const dg_mesh* mesh, double* t) {
  if (!mesh || !t) return fail(DG_ERR_ARG, "null argument");
  *t = mesh->t_mesh;
  return DG_OK;
}

dg_status dg_set_mesh_time(dg_mesh* mesh, double t) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (!mesh->moving) return fail(DG_ERR_UNSUPPORTED, "only a moving mesh has a time");
  if (!std::isfinite(t)) return fail(DG_ERR_ARG, "t must be finite");
  mesh->t_mesh = t;
  return DG_OK;
}

dg_status dg_batch_create(const dg_mesh_desc* descs, int n_instances, cudaStream_t stream, dg_mesh** out) {
  if (!descs || !out || n_instances < 1) return fail(DG_ERR_ARG, "null argument or empty batch");
  *out = nullptr;
  for (int i = 0; i < n_instances; ++i) {
    dg_status st = check_desc(descs + i);
    if (st != DG_OK) return st;
    if (descs[i].flux != descs[0].flux || descs[i].gamma != descs[0].gamma)
      return fail(DG_ERR_ARG, "all instances of a batch must share flux and gamma");
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) return fail(DG_ERR_CUDA, "no CUDA device available (the library has no CPU path)");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  std::vector<dgh::MeshInput> ins;
  for (int i = 0; i < n_instances; ++i) ins.push_back(input_of(descs + i));
  std::string err;
  int r = dgh::build_batch(ins, &m->h, &err);
  if (r != 0) {
    delete m;
    return fail((dg_status)r, err);
  }
  return create_device_mesh(m, descs, stream, out);
}

dg_status dg_mesh_geometry(const dg_mesh* mesh, int64_t* n_curved_elems, int64_t* n_curved_faces, int64_t* geometry_doubles) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (n_curved_elems) *n_curved_elems = mesh->h.n_curved;
  if (n_curved_faces) *n_curved_faces = mesh->h.n_curved_faces;
  if (geometry_doubles) *geometry_doubles = (int64_t)(mesh->h.cpool.size() + mesh->h.fgeo.size());
  return DG_OK;
}

dg_status dg_batch_layout(const dg_mesh* mesh, int64_t* instance_elem_off, int64_t* instance_dof_off) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  const size_t k = mesh->h.inst_elem_off.size();
  if (instance_elem_off) std::memcpy(instance_elem_off, mesh->h.inst_elem_off.data(), sizeof(int64_t) * k);
  if (instance_dof_off) std::memcpy(instance_dof_off, mesh->h.inst_dof_off.data(), sizeof(int64_t) * k);
  return DG_OK;
}

}  // extern "C"

namespace {

dg_status create_device_mesh(dg_mesh* m, const dg_mesh_desc* desc, cudaStream_t stream, dg_mesh** out) {
  m->flux = desc->flux;
  m->gamma = desc->gamma;
  m->scheduler = desc->scheduler;
  m->threshold = desc->imbalance_threshold > 0 ? desc->imbalance_threshold : 0.1;
  cudaGetDevice(&m->device);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  const dgh::HostMesh& h = m->h;
  m->nQmax = h.n * h.n * h.n;
  m->wpb = m->nQmax >= 216 ? 1 : 2;  // warps cooperating on one element
  auto fail_cuda = [&](cudaError_t e, const char* what) {
    m->release();
    delete m;
    return cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = dgk::element_kernel_attributes(m->nQmax, m->wpb, &m->blocks_per_sm, m->h.n_curved > 0)) != cudaSuccess) return fail_cuda(e, "kernel attributes");
  if (m->blocks_per_sm < 1) m->blocks_per_sm = 1;
  std::vector<int> slot_tab(h.slot_tab);
  if ((e = upload(&m->d_dpool, h.tables.dpool)) != cudaSuccess) return fail_cuda(e, "upload tables");
  if ((e = upload(&m->d_ipool, h.tables.ipool)) != cudaSuccess) return fail_cuda(e, "upload tables");
  if ((e = upload(&m->d_tabs, h.tables.tabs)) != cudaSuccess) return fail_cuda(e, "upload tables");
  if ((e = upload(&m->d_slot_tab, slot_tab)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_slot_type, h.slot_type)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_slot_qoff, h.slot_qoff)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_slot_hoff, h.slot_hoff)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_slot_ftoff, h.slot_ftoff)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_elem_of_slot, h.elem_of_slot)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_elem_qoff, h.elem_qoff)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_elem_voff, h.elem_voff)) != cudaSuccess) return fail_cuda(e, "upload slots");
  if ((e = upload(&m->d_geo, h.slot_geo)) != cudaSuccess) return fail_cuda(e, "upload geometry");
  if (h.n_curved) {
    if ((e = upload(&m->d_slot_coff, h.slot_coff)) != cudaSuccess) return fail_cuda(e, "upload geometry");
    if ((e = upload(&m->d_cpool, h.cpool)) != cudaSuccess) return fail_cuda(e, "upload geometry");
    if ((e = upload(&m->d_fgeo, h.fgeo)) != cudaSuccess) return fail_cuda(e, "upload geometry");
    if ((e = upload(&m->d_snrm, h.snrm)) != cudaSuccess) return fail_cuda(e, "upload geometry");
  }
  if ((e = upload(&m->d_fnrm, h.slot_fnrm)) != cudaSuccess) return fail_cuda(e, "upload geometry");
  if ((e = upload(&m->d_faces, h.faces)) != cudaSuccess) return fail_cuda(e, "upload faces");
  if ((e = upload(&m->d_fblocks, h.face_blocks)) != cudaSuccess) return fail_cuda(e, "upload faces");
  if ((e = upload(&m->d_perms, h.perms)) != cudaSuccess) return fail_cuda(e, "upload maps");
  if ((e = upload(&m->d_dense, h.dense)) != cudaSuccess) return fail_cuda(e, "upload maps");
  for (int t = 0; t < 4; ++t)
    if ((e = upload(&m->d_type_slots[t], h.type_slots[t])) != cudaSuccess) return fail_cuda(e, "upload type lists");
  if ((e = cudaMalloc(&m->d_H, sizeof(double) * std::max<int64_t>(1, h.h_total))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_T, sizeof(double) * std::max<int64_t>(1, h.t_total))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_stage, sizeof(double) * std::max<int64_t>(1, h.n_dof))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_status, sizeof(unsigned))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_counters, 2 * sizeof(unsigned))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_cost, 2 * dgk::kMaxTabs * sizeof(unsigned long long))) != cudaSuccess) return fail_cuda(e, "workspace");
  if ((e = cudaMalloc(&m->d_smns, (size_t)m->num_sms * sizeof(unsigned long long))) != cudaSuccess) return fail_cuda(e, "workspace");
  cudaMemset(m->d_status, 0, sizeof(unsigned));
  cudaMemset(m->d_counters, 0, 2 * sizeof(unsigned));
  cudaMemset(m->d_cost, 0, 2 * dgk::kMaxTabs * sizeof(unsigned long long));
  cudaMemset(m->d_smns, 0, (size_t)m->num_sms * sizeof(unsigned long long));
  {
    const std::vector<double> w0 = m->static_weights();
    for (int t = 0; t < dgk::kMaxTabs; ++t) {
      m->weight[t] = w0[t];
      m->tab_wpb[t] = m->wpb;
    }
  }
  if ((e = m->build_groups()) != cudaSuccess) return fail_cuda(e, "chunk table");
  if ((e = m->build_static_chunks()) != cudaSuccess) return fail_cuda(e, "chunk table");
  if ((e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking)) != cudaSuccess) return fail_cuda(e, "stream");
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return fail_cuda(e, "synchronise");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail_cuda(e, "synchronise");
  *out = m;
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_mesh_check(const dg_mesh_desc* desc, int64_t* counts, double* quad_xyz, int64_t* slot_of_elem) {
  if (!desc) return fail(DG_ERR_ARG, "null argument");
  dgh::HostMesh h;
  dgh::MeshInput in = input_of(desc);
  std::string err;
  int r = dgh::build_mesh(in, &h, &err);
  if (r != 0) return fail((dg_status)r, err);
  if (counts) {
    counts[0] = h.n_elems;
    counts[1] = h.n_faces;
    for (int t = 0; t < 4; ++t) counts[2 + t] = h.type_count[t];
    counts[6] = h.n_perm;
    counts[7] = h.n_dense;
  }
  if (quad_xyz) std::memcpy(quad_xyz, h.quad_xyz.data(), sizeof(double) * h.quad_xyz.size());
  if (slot_of_elem) std::memcpy(slot_of_elem, h.slot_of_elem.data(), sizeof(int64_t) * h.n_elems);
  return DG_OK;
}

dg_status dg_partition_plan(const dg_mesh_desc* desc, int nparts, const double* type_weight, int64_t* part_of_elem,
                            int64_t* halo_off, int64_t* halo_elems) {
  if (!desc || !part_of_elem || !halo_off) return fail(DG_ERR_ARG, "null argument");
  dgh::HostMesh h;
  std::string err;
  int r = dgh::build_mesh(input_of(desc), &h, &err);
  if (r != 0) return fail((dg_status)r, err);
  std::vector<int64_t> part, off, halo;
  r = dgh::partition_plan(h, nparts, type_weight, &part, &off, &halo, &err);
  if (r != 0) return fail((dg_status)r, err);
  std::memcpy(part_of_elem, part.data(), sizeof(int64_t) * part.size());
  std::memcpy(halo_off, off.data(), sizeof(int64_t) * off.size());
  if (halo_elems) std::memcpy(halo_elems, halo.data(), sizeof(int64_t) * halo.size());
  return DG_OK;
}

}  // extern "C"

namespace {

// The part mesh of `part` (owned elements and their ghosts, ascending
// global caller index) and its halo lists, on the host.  A face with one
// ghost side is sent (the owned side's trace) to, and received (the ghost
// side's slot) from, the ghost's part; both lists are ordered by (peer,
// global owner element, owner's local face), an order the peer's lists of
// the same faces share.
struct PartPlan {
  dgh::HostMesh h;
  std::vector<int64_t> glob, send_count, recv_count, send_off, recv_off, send_key, recv_key;
};

dg_status plan_part(const dg_mesh_desc* desc, const int64_t* part_of_elem, int nparts, int part, PartPlan* P) {
  if (!desc || !part_of_elem) return fail(DG_ERR_ARG, "null argument");
  if (nparts < 1 || part < 0 || part >= nparts) return fail(DG_ERR_ARG, "part must lie in [0, nparts)");
  dg_status st = check_desc(desc);
  if (st != DG_OK) return st;
  const int64_t E = desc->n_elems;
  for (int64_t e = 0; e < E; ++e)
    if (part_of_elem[e] < 0 || part_of_elem[e] >= nparts) return fail(DG_ERR_ARG, "part_of_elem out of range");
  // the whole mesh's faces give the ghosts: every element of another part
  // that shares a face with an element of this part
  std::string err;
  dgh::HostMesh G;
  int r = dgh::build_mesh(input_of(desc), &G, &err);
  if (r != 0) return fail((dg_status)r, err);
  std::vector<uint8_t> keep(E, 0);
  for (int64_t e = 0; e < E; ++e) keep[e] = part_of_elem[e] == part ? 1 : 0;
  for (int64_t f = 0; f < G.n_faces; ++f) {
    const int64_t a = G.face_e0[f], b = G.face_e1[f];
    if (part_of_elem[a] == part && part_of_elem[b] != part) keep[b] = 2;
    if (part_of_elem[b] == part && part_of_elem[a] != part) keep[a] = 2;
  }
  std::vector<int8_t> type;
  std::vector<int64_t> off(1, 0), verts;
  std::vector<uint8_t> ghost;
  P->glob.clear();
  for (int64_t e = 0; e < E; ++e) {
    if (!keep[e]) continue;
    P->glob.push_back(e);
    type.push_back(desc->type[e]);
    for (int64_t k = desc->elem_vert_off[e]; k < desc->elem_vert_off[e + 1]; ++k) verts.push_back(desc->elem_verts[k]);
    off.push_back((int64_t)verts.size());
    ghost.push_back(keep[e] == 2 ? 1 : 0);
  }
  if (P->glob.empty() || std::find(ghost.begin(), ghost.end(), 0) == ghost.end())
    return fail(DG_ERR_ARG, "the part owns no element");
  dgh::MeshInput in = input_of(desc);
  in.n_elems = (int64_t)P->glob.size();
  in.type = type.data();
  in.off = off.data();
  in.verts = verts.data();
  in.ghost = ghost.data();
  r = dgh::build_mesh(in, &P->h, &err);
  if (r != 0) return fail((dg_status)r, err);
  const dgh::HostMesh& h = P->h;
  const int64_t per = 5 * (int64_t)h.n * h.n;
  struct Entry { int64_t peer, key0, key1, off; };
  std::vector<Entry> snd, rcv;
  for (int64_t f = 0; f < h.n_faces; ++f) {
    const int64_t a = h.face_e0[f], b = h.face_e1[f];
    const bool ga = ghost[a] != 0, gb = ghost[b] != 0;
    if (ga == gb) continue;
    const int own_side = ga ? 1 : 0;
    const int64_t peer = part_of_elem[P->glob[ga ? a : b]];
    const int64_t toff = h.faces[f].toff;
    snd.push_back({peer, P->glob[a], h.face_l0[f], toff + own_side * per});
    rcv.push_back({peer, P->glob[a], h.face_l0[f], toff + (1 - own_side) * per});
  }
  auto by_key = [](const Entry& x, const Entry& y) { return std::tie(x.peer, x.key0, x.key1) < std::tie(y.peer, y.key0, y.key1); };
  std::sort(snd.begin(), snd.end(), by_key);
  std::sort(rcv.begin(), rcv.end(), by_key);
  P->send_count.assign(nparts, 0);
  P->recv_count.assign(nparts, 0);
  P->send_off.clear();
  P->recv_off.clear();
  P->send_key.clear();
  P->recv_key.clear();
  for (const auto& x : snd) {
    P->send_count[x.peer]++;
    P->send_off.push_back(x.off);
    P->send_key.push_back(x.key0 * 8 + x.key1);
  }
  for (const auto& x : rcv) {
    P->recv_count[x.peer]++;
    P->recv_off.push_back(x.off);
    P->recv_key.push_back(x.key0 * 8 + x.key1);
  }
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_halo_plan(const dg_mesh_desc* desc, const int64_t* part_of_elem, int nparts, int part,
                       int64_t* send_faces, int64_t* recv_faces, int64_t* send_keys, int64_t* recv_keys) {
  if (!send_faces || !recv_faces) return fail(DG_ERR_ARG, "null argument");
  PartPlan P;
  dg_status st = plan_part(desc, part_of_elem, nparts, part, &P);
  if (st != DG_OK) return st;
  for (int q = 0; q < nparts; ++q) {
    send_faces[q] = P.send_count[q];
    recv_faces[q] = P.recv_count[q];
  }
  if (send_keys) std::memcpy(send_keys, P.send_key.data(), sizeof(int64_t) * P.send_key.size());
  if (recv_keys) std::memcpy(recv_keys, P.recv_key.data(), sizeof(int64_t) * P.recv_key.size());
  return DG_OK;
}

dg_status dg_mesh_create_part(const dg_mesh_desc* desc, const int64_t* part_of_elem, int nparts, int part,
                              cudaStream_t stream, dg_mesh** out) {
  if (!out) return fail(DG_ERR_ARG, "null argument");
  *out = nullptr;
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) return fail(DG_ERR_CUDA, "no CUDA device available (the library has no CPU path)");
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ERR_OOM, "host allocation failed");
  {
    PartPlan P;
    dg_status st = plan_part(desc, part_of_elem, nparts, part, &P);
    if (st != DG_OK) {
      delete m;
      return st;
    }
    m->h = std::move(P.h);
    m->global_of_local = std::move(P.glob);
    m->send_count = std::move(P.send_count);
    m->recv_count = std::move(P.recv_count);
    m->send_off = std::move(P.send_off);
    m->recv_off = std::move(P.recv_off);
  }
  m->nparts = nparts;
  m->part = part;
  dg_mesh* made = nullptr;
  dg_status st = create_device_mesh(m, desc, stream, &made);
  if (st != DG_OK) return st;
  if (!made->send_off.empty()) {
    cudaError_t e = upload(&made->d_send_off, made->send_off);
    if (e == cudaSuccess) e = upload(&made->d_recv_off, made->recv_off);
    if (e != cudaSuccess) {
      made->release();
      delete made;
      return cuda_fail(e, "upload halo lists");
    }
  }
  *out = made;
  return DG_OK;
}

dg_status dg_part_elements(const dg_mesh* mesh, int64_t* n_local, int64_t* global_of_local, int8_t* is_ghost) {
  if (!mesh || !n_local) return fail(DG_ERR_ARG, "null argument");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  *n_local = (int64_t)mesh->global_of_local.size();
  for (int64_t e = 0; e < *n_local; ++e) {
    if (global_of_local) global_of_local[e] = mesh->global_of_local[e];
    if (is_ghost) is_ghost[e] = (int8_t)mesh->h.slot_ghost[mesh->h.slot_of_elem[e]];
  }
  return DG_OK;
}

dg_status dg_halo_counts(const dg_mesh* mesh, int64_t* send_faces, int64_t* recv_faces, int64_t* doubles_per_face) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  for (int p = 0; p < mesh->nparts; ++p) {
    if (send_faces) send_faces[p] = mesh->send_count[p];
    if (recv_faces) recv_faces[p] = mesh->recv_count[p];
  }
  if (doubles_per_face) *doubles_per_face = 5 * (int64_t)mesh->h.n * mesh->h.n;
  return DG_OK;
}

dg_status dg_halo_pack(dg_mesh* mesh, double* send, cudaStream_t stream) {
  if (!mesh || (!send && !mesh->send_off.empty())) return fail(DG_ERR_ARG, "null argument");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  if (mesh->send_off.empty()) return DG_OK;
  dgk::launch_halo_copy(mesh->d_T, send, mesh->d_send_off, (int64_t)mesh->send_off.size(),
                        5 * mesh->h.n * mesh->h.n, true, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_halo_unpack(dg_mesh* mesh, const double* recv, cudaStream_t stream) {
  if (!mesh || (!recv && !mesh->recv_off.empty())) return fail(DG_ERR_ARG, "null argument");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  if (mesh->recv_off.empty()) return DG_OK;
  dgk::launch_halo_copy(recv, mesh->d_T, mesh->d_recv_off, (int64_t)mesh->recv_off.size(),
                        5 * mesh->h.n * mesh->h.n, false, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_halo_pack_gradients(dg_mesh* mesh, double* send, cudaStream_t stream) {
  if (!mesh || (!send && !mesh->send_off.empty())) return fail(DG_ERR_ARG, "null argument");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  if (!mesh->ns) return fail(DG_ERR_UNSUPPORTED, "gradient traces exist for the Navier-Stokes equations");
  if (mesh->send_off.empty()) return DG_OK;
  dgk::launch_halo_copy(mesh->d_Vt, send, mesh->d_send_off, (int64_t)mesh->send_off.size(),
                        15 * mesh->h.n * mesh->h.n, true, stream, 3);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_halo_unpack_gradients(dg_mesh* mesh, const double* recv, cudaStream_t stream) {
  if (!mesh || (!recv && !mesh->recv_off.empty())) return fail(DG_ERR_ARG, "null argument");
  if (mesh->nparts == 0) return fail(DG_ERR_ARG, "not a partition mesh");
  if (!mesh->ns) return fail(DG_ERR_UNSUPPORTED, "gradient traces exist for the Navier-Stokes equations");
  if (mesh->recv_off.empty()) return DG_OK;
  dgk::launch_halo_copy(recv, mesh->d_Vt, mesh->d_recv_off, (int64_t)mesh->recv_off.size(),
                        15 * mesh->h.n * mesh->h.n, false, stream, 3);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_rk_stage_lift(dg_mesh* mesh, cudaStream_t stream) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "a moving mesh steps with dg_rk_step: every stage needs the geometry of its time and a mass solve");
  if (!mesh->ns) return fail(DG_ERR_UNSUPPORTED, "the lifting half-stage belongs to the Navier-Stokes equations");
  DG_CUDA(cudaMemsetAsync(mesh->d_counters, 0, 2 * sizeof(unsigned), stream));
  mesh->parity = 0;
  mesh->begin_timing(1);
  mesh->timed(false, stream, [&] { dgk::launch_faces_ns(mesh->ctx(), (int64_t)mesh->h.face_blocks.size(), mesh->h.n, 0, stream); });
  dgk::StageArgs none{nullptr, nullptr, nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kNsVolume, none, stream);
  mesh->lift_done = true;
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_rk_prime(dg_mesh* mesh, const double* Q_store, cudaStream_t stream) {
  if (!mesh || !Q_store) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "a moving mesh steps with dg_rk_step: every stage needs the geometry of its time and a mass solve");
  mesh->lift_done = false;
  DG_CUDA(cudaMemsetAsync(mesh->d_counters, 0, 2 * sizeof(unsigned), stream));
  mesh->parity = 0;
  mesh->begin_timing(1);
  dgk::StageArgs a{Q_store, const_cast<double*>(Q_store), nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kFwd, a, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_rk_stage(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int stage, int last,
                      cudaStream_t stream) {
  if (!mesh || !Q_store || !K_store) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "a moving mesh steps with dg_rk_step: every stage needs the geometry of its time and a mass solve");
  if (stage < 0 || stage > 4) return fail(DG_ERR_ARG, "stage must lie in 0..4");
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be finite");
  if (mesh->ns && !mesh->lift_done)
    return fail(DG_ERR_ARG, "Navier-Stokes: dg_rk_stage_lift (and the gradient-trace exchange) first");
  DG_CUDA(cudaMemsetAsync(mesh->d_counters, 0, 2 * sizeof(unsigned), stream));
  mesh->parity = 0;
  if (!mesh->ns) mesh->begin_timing(1);
  if (mesh->ns) {
    // the inviscid and viscous flux of the stage (the lifting half ran in
    // dg_rk_stage_lift, before the gradient traces were exchanged)
    mesh->timed(false, stream, [&] { dgk::launch_faces_ns(mesh->ctx(), (int64_t)mesh->h.face_blocks.size(), mesh->h.n, 1, stream); });
    mesh->lift_done = false;
  } else {
    mesh->face_phase(stream);
  }
  dgk::StageArgs a{Q_store, Q_store, K_store, kLsA[stage], kLsB[stage], dt};
  if (mesh->fused) {
    mesh->element_phase(last ? dgk::kBwdRk : dgk::kBwdRkFwd, a, stream);
  } else {
    mesh->element_phase(dgk::kBwdRk, a, stream);
    if (!last) mesh->element_phase(dgk::kFwd, a, stream);
  }
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_mesh_destroy(dg_mesh* mesh) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  cudaDeviceSynchronize();
  mesh->release();
  delete mesh;
  return DG_OK;
}

dg_status dg_mesh_layout(const dg_mesh* mesh, int64_t* n_dof, int64_t* slot_of_elem, int64_t* counts) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (n_dof) *n_dof = mesh->h.n_dof;
  if (slot_of_elem) std::memcpy(slot_of_elem, mesh->h.slot_of_elem.data(), sizeof(int64_t) * mesh->h.n_elems);
  if (counts) {
    counts[0] = mesh->h.n_elems;
    counts[1] = mesh->h.n_faces;
    for (int t = 0; t < 4; ++t) counts[2 + t] = mesh->h.type_count[t];
  }
  return DG_OK;
}

dg_status dg_set_state(dg_mesh* mesh, const double* Q_ext, int is_device, double* Q_store, cudaStream_t stream) {
  if (!mesh || !Q_ext || !Q_store) return fail(DG_ERR_ARG, "null argument");
  const double* src = Q_ext;
  if (!is_device) {
    DG_CUDA(cudaMemcpyAsync(mesh->d_stage, Q_ext, sizeof(double) * mesh->h.n_dof, cudaMemcpyHostToDevice, stream));
    src = mesh->d_stage;
  }
  dgk::launch_permute(mesh->ctx(), src, Q_store, mesh->h.n_elems, 1, stream);
  mesh->convert_hex(dgk::kGather, src, Q_store, stream);
  DG_CUDA(cudaGetLastError());
  if (!is_device) DG_CUDA(cudaStreamSynchronize(stream));
  return DG_OK;
}

dg_status dg_get_state(const dg_mesh* mesh, const double* Q_store, double* Q_ext, int is_device, cudaStream_t stream) {
  if (!mesh || !Q_ext || !Q_store) return fail(DG_ERR_ARG, "null argument");
  double* dst = is_device ? Q_ext : mesh->d_stage;
  dgk::launch_permute(mesh->ctx(), Q_store, dst, mesh->h.n_elems, 0, stream);
  mesh->convert_hex(dgk::kScatter, Q_store, dst, stream);
  DG_CUDA(cudaGetLastError());
  if (!is_device) {
    DG_CUDA(cudaMemcpyAsync(Q_ext, mesh->d_stage, sizeof(double) * mesh->h.n_dof, cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
  }
  return DG_OK;
}

dg_status dg_quad_points(const dg_mesh* mesh, double* xyz_out) {
  if (!mesh || !xyz_out) return fail(DG_ERR_ARG, "null argument");
  std::memcpy(xyz_out, mesh->h.quad_xyz.data(), sizeof(double) * mesh->h.quad_xyz.size());
  return DG_OK;
}

dg_status dg_project(dg_mesh* mesh, const double* q_points, double* Q_store, cudaStream_t stream) {
  if (!mesh || !q_points || !Q_store) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) {
    // Algorithm 1 at the mesh time: the load vector on the geometry of t,
    // then the solve with M(t)
    mesh->moving_geometry(mesh->t_mesh, stream);
    dgk::StageArgs b{q_points, Q_store, nullptr, 0.0, 0.0, 0.0};
    mesh->element_phase(dgk::kLoad, b, stream);
    double tau[4];
    dg_mesh::powers(mesh->t_mesh, tau);
    DG_CUDA(mesh->moving_mass(Q_store, Q_store, tau, 0, stream));
    return DG_OK;
  }
  dgk::StageArgs a{q_points, Q_store, nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kProject, a, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_load_vector(dg_mesh* mesh, const double* q_points, double* b_store, cudaStream_t stream) {
  if (!mesh || !q_points || !b_store) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) mesh->moving_geometry(mesh->t_mesh, stream);
  dgk::StageArgs a{q_points, b_store, nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kLoad, a, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_eval_nodal(dg_mesh* mesh, const double* Q_store, double* u_points, cudaStream_t stream) {
  if (!mesh || !Q_store || !u_points) return fail(DG_ERR_ARG, "null argument");
  dgk::StageArgs a{Q_store, u_points, nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kEval, a, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_rhs(dg_mesh* mesh, const double* Q_store, double* R_store, cudaStream_t stream) {
  if (!mesh || !Q_store || !R_store) return fail(DG_ERR_ARG, "null argument");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "a partition mesh steps with dg_rk_prime / dg_rk_stage and the halo exchange");
  if (mesh->moving) {
    mesh->begin_timing(1);
    DG_CUDA(mesh->moving_rhs(Q_store, R_store, stream));
    return DG_OK;
  }
  DG_CUDA(cudaMemsetAsync(mesh->d_counters, 0, 2 * sizeof(unsigned), stream));
  mesh->parity = 0;
  mesh->begin_timing(1);
  dgk::StageArgs a{Q_store, R_store, nullptr, 0.0, 0.0, 0.0};
  mesh->element_phase(dgk::kFwd, a, stream);
  mesh->face_phase(stream);
  mesh->element_phase(dgk::kBwdRhs, a, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status dg_rk_step(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int nsteps, cudaStream_t stream) {
  if (!mesh || !Q_store || !K_store) return fail(DG_ERR_ARG, "null argument");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "a partition mesh steps with dg_rk_prime / dg_rk_stage and the halo exchange");
  if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return DG_OK;
  if (!(std::isfinite(dt))) return fail(DG_ERR_ARG, "dt must be finite");
  if (mesh->moving) {
    // direct launches: every stage's geometry and mass matrix depend on the
    // mesh time, passed by value
    mesh->begin_timing(1);
    DG_CUDA(mesh->moving_rk(Q_store, K_store, dt, nsteps, stream));
  } else if (!mesh->profiling) {
    // replay the three captured graphs; a new state, register, dt or step
    // count only changes the arguments of the parameter node
    if (!mesh->gr_prime.x || mesh->r_sched != mesh->scheduler || mesh->r_fused != (int)mesh->fused) {
      if (!mesh->d_rkdyn && cudaMalloc(&mesh->d_rkdyn, sizeof(dgk::RkDyn)) != cudaSuccess)
        return fail(DG_ERR_OOM, "step parameter block");
      mesh->begin_timing(0);
      cudaError_t e = mesh->capture_stage_graphs();
      if (e != cudaSuccess) return cuda_fail(e, "stage graph capture");
    }
    dgk::RkDyn* d = mesh->d_rkdyn;
    double* Qp = Q_store;
    double* Kp = K_store;
    double dtv = dt;
    void* args[] = {&d, &Qp, &Kp, &dtv};
    cudaKernelNodeParams kp{};
    dgk::rk_params_node(&kp, args);
    DG_CUDA(cudaGraphExecKernelNodeSetParams(mesh->gr_prime.x, mesh->gr_param_node, &kp));
    mesh->last_pool = 0;
    DG_CUDA(cudaGraphLaunch(mesh->gr_prime.x, stream));
    for (int k = 0; k + 1 < nsteps; ++k) DG_CUDA(cudaGraphLaunch(mesh->gr_step.x, stream));
    DG_CUDA(cudaGraphLaunch(mesh->gr_last.x, stream));
  } else {
    if (!mesh->gexec || mesh->g_Q != Q_store || mesh->g_K != K_store || mesh->g_dt != dt ||
        mesh->g_nsteps != nsteps || mesh->g_sched != mesh->scheduler || mesh->g_fused != (int)mesh->fused) {
      if (mesh->gexec) {
        cudaGraphExecDestroy(mesh->gexec);
        mesh->gexec = nullptr;
      }
      cudaGraph_t g;
      mesh->begin_timing(0);
      DG_CUDA(cudaStreamBeginCapture(mesh->cap, cudaStreamCaptureModeThreadLocal));
      mesh->enqueue_rk(Q_store, K_store, dt, nsteps, mesh->cap);
      cudaError_t e = cudaStreamEndCapture(mesh->cap, &g);
      if (e != cudaSuccess) return cuda_fail(e, "graph capture");
      e = cudaGraphInstantiate(&mesh->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
      mesh->g_Q = Q_store;
      mesh->g_K = K_store;
      mesh->g_dt = dt;
      mesh->g_nsteps = nsteps;
      mesh->g_sched = mesh->scheduler;
      mesh->g_fused = (int)mesh->fused;
      ++mesh->graph_captures;
    }
    mesh->last_pool = 0;
    DG_CUDA(cudaGraphLaunch(mesh->gexec, stream));
  }
  if (mesh->rebalance_every > 0) {
    // the imbalance trigger of Sec. 3 in the time loop: every
    // rebalance_every steps compare the measured SM load imbalance with the
    // threshold and rebuild the chunk tables from the measured costs
    mesh->steps_since_check += nsteps;
    if (mesh->steps_since_check >= mesh->rebalance_every) {
      mesh->steps_since_check = 0;
      int rebuilt = 0;
      dg_status st = dg_rebalance(mesh, 0, &rebuilt, stream);
      if (st != DG_OK) return st;
      mesh->checks++;
      mesh->rebalances += rebuilt;
    }
  }
  return DG_OK;
}

dg_status dg_graph_captures(const dg_mesh* mesh, int64_t* captures) {
  if (!mesh || !captures) return fail(DG_ERR_ARG, "null argument");
  *captures = mesh->graph_captures;
  return DG_OK;
}

dg_status dg_set_rebalance_interval(dg_mesh* mesh, int nsteps) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (nsteps < 0) return fail(DG_ERR_ARG, "the interval must be >= 0");
  mesh->rebalance_every = nsteps;
  mesh->steps_since_check = 0;
  return DG_OK;
}

dg_status dg_rebalance_stats(const dg_mesh* mesh, int64_t* checks, int64_t* rebalances) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (checks) *checks = mesh->checks;
  if (rebalances) *rebalances = mesh->rebalances;
  return DG_OK;
}

dg_status dg_rhs_vjp(dg_mesh* mesh, const double* Q_store, const double* Rbar, double* Qbar, cudaStream_t stream) {
  if (!mesh || !Q_store || !Rbar || !Qbar) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers static meshes");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers whole meshes");
  if (mesh->split || mesh->flux == DG_FLUX_EC)
    return fail(DG_ERR_UNSUPPORTED, "the adjoint covers the weak form with the LF or Roe flux");
  DG_CUDA(mesh->ensure_adjoint(0));
  dgk::VjpArgs va{Q_store, Rbar, nullptr, Qbar, 0.0, 0.0, 0.0, 0, 0};
  mesh->enqueue_vjp(va, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of dg_rhs_vjp.  dg_rhs_vjp allocates its adjoint
// face buffer with cudaMalloc the first time it runs on a mesh; this variant
// takes that scratch from a fixed-size array in device global memory that is
// part of the library image instead, so the call itself never allocates.
namespace {

constexpr size_t kNoAllocScratchDoubles = size_t(8) << 20;  // 64 MiB of FP64 per device
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;

// Device address of the scratch array for the current device, looked up on
// every call (cheap, allocates nothing, and stays right if the device's
// primary context was reset and the module loaded again); in host code the
// symbol itself is only a host-side stand-in, never a device address.
cudaError_t noalloc_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" {

dg_status dg_rhs_vjp_noalloc(dg_mesh* mesh, const double* Q_store, const double* Rbar, double* Qbar,
                             cudaStream_t stream) {
  if (!mesh || !Q_store || !Rbar || !Qbar) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers static meshes");
  if (mesh->split || mesh->flux == DG_FLUX_EC)
    return fail(DG_ERR_UNSUPPORTED, "the adjoint covers the weak form with the LF or Roe flux");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers whole meshes");
  if (mesh->ns)
    return fail(DG_ERR_UNSUPPORTED, "dg_rhs_vjp_noalloc covers the Euler equations (the viscous adjoint needs "
                                    "workspace that dg_rhs_vjp allocates); use dg_rhs_vjp");
  const size_t need = (size_t)std::max<int64_t>(1, mesh->h.t_total);
  if (need > kNoAllocScratchDoubles)
    return fail(DG_ERR_ARG, "dg_rhs_vjp_noalloc: the mesh needs " + std::to_string(need) +
                                " doubles of face scratch, more than the fixed " +
                                std::to_string(kNoAllocScratchDoubles) + " (64 MiB); use dg_rhs_vjp");
  int dev = -1;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev != mesh->device) return fail(DG_ERR_ARG, "dg_rhs_vjp_noalloc: the mesh's device is not the current device");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(DG_ERR_UNSUPPORTED, "device ordinal beyond 63");
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  dgk::Ctx c = mesh->ctx();
  c.Tv = scratch;  // every face side slot is written (seed) before it is read
  dgk::VjpArgs va{Q_store, Rbar, nullptr, Qbar, 0.0, 0.0, 0.0, 0, 0};
  dgk::launch_vjp(c, 0, va, mesh->h.n_elems, mesh->wpb, stream);
  dgk::launch_faces_vjp(c, (int64_t)mesh->h.face_blocks.size(), mesh->h.n, stream);
  dgk::launch_vjp(c, 2, va, mesh->h.n_elems, mesh->wpb, stream);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// Reverse LSERK through nsteps steps (2N storage, K = 0 at every step start),
// per stage s = 5..1 at the stage input state Q_{s-1}:
//   Kbar <- Kbar + B_s Qbar;  Qbar <- Qbar + dt J(Q_{s-1})^T Kbar;  Kbar <- A_s Kbar.
// Stage inputs are recomputed segment by segment from checkpoints of Q taken
// every ckpt_every steps (the last segment's forward pass is not needed).
}  // extern "C"

namespace {
// Reverse sweep of dg_rk_vjp over the checkpoints ck[seg] (Q at the start of
// segment seg of c steps); Q0bar already holds QKbar.
// Segments starting at or after step `tail0` (a multiple of c) already have
// their stage data in the stage store, stage g = 5 (step - tail0) + s (kept by
// dg_rk_vjp's own forward pass); earlier segments are recomputed from their
// checkpoints ck[seg].
dg_status rk_vjp_reverse(dg_mesh* mesh, const double* ck, double dt, int nsteps, int c, double* Q0bar,
                         cudaStream_t stream, int tail0) {
  const size_t n = (size_t)mesh->h.n_dof, bytes = sizeof(double) * n;
  const int nseg = (nsteps + c - 1) / c;
  // forward data of one segment's stages kept for the reverse pass when the
  // device has room (else each reverse stage recomputes them from copies of
  // the stage states)
  const bool keep = mesh->keep_stages && mesh->ensure_stage_store(5 * c);
  DG_CUDA(mesh->ensure_adjoint((size_t)(keep ? 2 : 2 + 5 * c) * n));
  double* Qw = mesh->d_ckpt;
  double* Kw = Qw + n;
  double* stages = Kw + n;
  DG_CUDA(cudaMemsetAsync(mesh->d_Kbar, 0, bytes, stream));
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int steps = std::min(c, nsteps - seg * c);
    const bool kept = keep && seg * c >= tail0;
    const int g0 = kept ? 5 * (seg * c - tail0) : 0;
    if (!kept) {
      DG_CUDA(cudaMemcpyAsync(Qw, ck + (size_t)seg * n, bytes, cudaMemcpyDeviceToDevice, stream));
      mesh->enqueue_rk_stages(Qw, Kw, dt, steps, keep ? nullptr : stages, stream, keep, false);
    }
    for (int step = steps - 1; step >= 0; --step)
      for (int s = 4; s >= 0; --s) {
        const int g = g0 + 5 * step + s;
        dgk::VjpArgs va{keep ? nullptr : stages + (size_t)g * n, nullptr, mesh->d_Kbar, Q0bar, kLsA[s], kLsB[s], dt,
                        1, 0};
        mesh->enqueue_vjp(va, stream, keep ? g : -1);
      }
  }
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status rk_vjp_args(dg_mesh* mesh, const void* a, const void* b, const void* c, int nsteps, int ckpt_every,
                      double dt) {
  if (!mesh || !a || !b || !c) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers static meshes");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "the adjoint covers whole meshes");
  if (mesh->split || mesh->flux == DG_FLUX_EC)
    return fail(DG_ERR_UNSUPPORTED, "the adjoint covers the weak form with the LF or Roe flux");
  if (nsteps < 0 || ckpt_every < 0) return fail(DG_ERR_ARG, "nsteps and ckpt_every must be >= 0");
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be finite");
  return DG_OK;
}

// ckpt_every == 0: the longest segment whose kept stage data (5 stages per
// step) fit in the mesh's share (dg_set_adjoint_memory, half by default) of
// the device memory that is free now (the mesh's own stage store counting as
// free: it is reused or replaced), at least 1 step.
int auto_ckpt(const dg_mesh* mesh, int nsteps) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const double per_step = 5.0 * sizeof(double) * (double)mesh->stage_doubles();
  const double avail = (double)free_b + sizeof(double) * (double)mesh->sstore_doubles;
  const double fit = mesh->adj_mem_frac * avail / per_step;
  return (int)std::max(1.0, std::min((double)nsteps, std::floor(fit)));
}
}  // namespace

extern "C" {

// Reverse LSERK through nsteps steps (2N storage, K = 0 at every step start),
// per stage s = 5..1 at the stage input state Q_{s-1}:
//   Kbar <- Kbar + B_s Qbar;  Qbar <- Qbar + dt J(Q_{s-1})^T Kbar;  Kbar <- A_s Kbar.
// Stage inputs are recomputed segment by segment from checkpoints of Q taken
// every ckpt_every steps (placed by a first forward pass here, or by
// dg_rk_step_checkpointed for dg_rk_vjp_checkpointed).
dg_status dg_rk_vjp(dg_mesh* mesh, const double* Q0_store, double dt, int nsteps, int ckpt_every,
                    const double* QKbar, double* Q0bar, cudaStream_t stream) {
  dg_status st = rk_vjp_args(mesh, Q0_store, QKbar, Q0bar, nsteps, ckpt_every, dt);
  if (st != DG_OK) return st;
  const size_t n = (size_t)mesh->h.n_dof, bytes = sizeof(double) * n;
  if (Q0bar != QKbar) DG_CUDA(cudaMemcpyAsync(Q0bar, QKbar, bytes, cudaMemcpyDeviceToDevice, stream));
  if (nsteps == 0) return DG_OK;
  const int c = ckpt_every == 0 ? auto_ckpt(mesh, nsteps) : std::min(ckpt_every, nsteps);
  const int nseg = (nsteps + c - 1) / c;
  // The forward pass keeps the stage data of the final steps itself, as many
  // whole segments as fit in half of the free device memory: those segments
  // are reversed without being recomputed.  The steps before tail0 only
  // place checkpoints.
  int tail0 = nsteps;
  mesh->compact = false;
  if (mesh->keep_stages && auto_ckpt(mesh, nsteps) < nsteps) mesh->compact = true;   // keep more stages
  if (mesh->keep_stages) {
    const int fit = auto_ckpt(mesh, nsteps);
    int t0 = std::max(0, nsteps - fit);
    t0 = ((t0 + c - 1) / c) * c;
    if (t0 < nsteps && mesh->ensure_stage_store(5 * std::max(c, nsteps - t0))) tail0 = t0;
  }
  const int nseg0 = (tail0 + c - 1) / c;   // segments that get checkpoints
  if (!mesh->d_ckpt_q || mesh->ckpt_q_doubles < (size_t)(nseg + 2) * n) {
    if (mesh->d_ckpt_q) cudaFree(mesh->d_ckpt_q);
    mesh->d_ckpt_q = nullptr;
    mesh->ckpt_q_doubles = 0;
    DG_CUDA(cudaMalloc(&mesh->d_ckpt_q, sizeof(double) * (size_t)(nseg + 2) * n));
    mesh->ckpt_q_doubles = (size_t)(nseg + 2) * n;
  }
  double* Qw = mesh->d_ckpt_q;
  double* Kw = Qw + n;
  double* ck = Kw + n;
  DG_CUDA(cudaMemcpyAsync(Qw, Q0_store, bytes, cudaMemcpyDeviceToDevice, stream));
  for (int seg = 0; seg < nseg0; ++seg) {
    DG_CUDA(cudaMemcpyAsync(ck + (size_t)seg * n, Qw, bytes, cudaMemcpyDeviceToDevice, stream));
    const int steps = std::min(c, tail0 - seg * c);
    if (seg < nseg0 - 1 || tail0 < nsteps) mesh->enqueue_rk_stages(Qw, Kw, dt, steps, nullptr, stream);
  }
  if (tail0 < nsteps) mesh->enqueue_rk_stages(Qw, Kw, dt, nsteps - tail0, nullptr, stream, true, false);
  return rk_vjp_reverse(mesh, ck, dt, nsteps, c, Q0bar, stream, tail0);
}

dg_status dg_rk_vjp_checkpointed(dg_mesh* mesh, const double* ckpt_store, double dt, int nsteps, int ckpt_every,
                                 const double* QKbar, double* Q0bar, cudaStream_t stream) {
  dg_status st = rk_vjp_args(mesh, ckpt_store, QKbar, Q0bar, nsteps, ckpt_every, dt);
  if (st != DG_OK) return st;
  if (ckpt_every < 1) return fail(DG_ERR_ARG, "ckpt_every must be >= 1 (the checkpoints' spacing)");
  mesh->compact = false;   // one segment's full stage data at a time
  const size_t bytes = sizeof(double) * (size_t)mesh->h.n_dof;
  if (Q0bar != QKbar) DG_CUDA(cudaMemcpyAsync(Q0bar, QKbar, bytes, cudaMemcpyDeviceToDevice, stream));
  if (nsteps == 0) return DG_OK;
  return rk_vjp_reverse(mesh, ckpt_store, dt, nsteps, std::min(ckpt_every, nsteps), Q0bar, stream, nsteps);
}

dg_status dg_rk_step_checkpointed(dg_mesh* mesh, double* Q_store, double* K_store, double dt, int nsteps,
                                  int ckpt_every, double* ckpt_store, cudaStream_t stream) {
  if (!mesh || !Q_store || !K_store || !ckpt_store) return fail(DG_ERR_ARG, "null argument");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "checkpointed steps serve the adjoint, which covers static meshes");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "a partition mesh steps with dg_rk_prime / dg_rk_stage and the halo exchange");
  if (nsteps < 0 || ckpt_every < 1) return fail(DG_ERR_ARG, "nsteps must be >= 0 and ckpt_every >= 1");
  if (!std::isfinite(dt)) return fail(DG_ERR_ARG, "dt must be finite");
  const size_t bytes = sizeof(double) * (size_t)mesh->h.n_dof;
  const int c = std::max(1, std::min(ckpt_every, nsteps));
  for (int seg = 0, done = 0; done < nsteps; ++seg, done += c) {
    DG_CUDA(cudaMemcpyAsync(ckpt_store + (size_t)seg * mesh->h.n_dof, Q_store, bytes, cudaMemcpyDeviceToDevice,
                            stream));
    dg_status r = dg_rk_step(mesh, Q_store, K_store, dt, std::min(c, nsteps - done), stream);
    if (r != DG_OK) return r;
  }
  return DG_OK;
}

}  // extern "C"

extern "C" {

dg_status dg_set_adjoint_storage(dg_mesh* mesh, int keep_stages) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  mesh->keep_stages = keep_stages != 0;
  if (!mesh->keep_stages && mesh->d_sstore) {
    DG_CUDA(cudaFree(mesh->d_sstore));
    mesh->d_sstore = nullptr;
    mesh->sstore_doubles = 0;
  }
  return DG_OK;
}

dg_status dg_set_adjoint_memory(dg_mesh* mesh, double fraction) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (!(fraction > 0.0 && fraction <= 0.95)) return fail(DG_ERR_ARG, "the memory fraction must lie in (0, 0.95]");
  mesh->adj_mem_frac = fraction;
  return DG_OK;
}

dg_status dg_set_volume_form(dg_mesh* mesh, int form) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (form != DG_VOLUME_WEAK && form != DG_VOLUME_SPLIT) return fail(DG_ERR_ARG, "unknown volume form");
  if (form == DG_VOLUME_SPLIT) {
    if (mesh->ns) return fail(DG_ERR_UNSUPPORTED, "the split form covers the Euler equations");
    if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "the split form covers static affine meshes");
    if (mesh->h.n_curved > 0) return fail(DG_ERR_UNSUPPORTED, "the split form covers affine meshes");
  }
  mesh->split = form == DG_VOLUME_SPLIT;
  {
    // the modelled chunk weights of the new volume form (dg_rebalance
    // replaces them with measured ones)
    const std::vector<double> w0 = mesh->static_weights();
    for (int t = 0; t < dgk::kMaxTabs; ++t) mesh->weight[t] = w0[t];
  }
  DG_CUDA(mesh->build_groups());
  DG_CUDA(mesh->build_static_chunks());
  mesh->drop_graphs();
  return DG_OK;
}

dg_status dg_set_physics(dg_mesh* mesh, int physics, double mu, double Pr) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (physics != DG_EULER && physics != DG_NAVIER_STOKES) return fail(DG_ERR_ARG, "unknown physics");
  if (physics == DG_NAVIER_STOKES && (mesh->split || mesh->flux == DG_FLUX_EC))
    return fail(DG_ERR_UNSUPPORTED, "Navier-Stokes runs with the weak form and the LF or Roe flux");
  if (physics == DG_NAVIER_STOKES) {
    if (!(mu >= 0.0) || !std::isfinite(mu)) return fail(DG_ERR_ARG, "mu must be finite and >= 0");
    if (!(Pr > 0.0) || !std::isfinite(Pr)) return fail(DG_ERR_ARG, "Pr must be finite and > 0");
    const size_t hb = sizeof(double) * (size_t)std::max<int64_t>(1, mesh->h.h_total);
    const size_t tb = sizeof(double) * (size_t)std::max<int64_t>(1, mesh->h.t_total);
    if (!mesh->d_Unod && cudaMalloc(&mesh->d_Unod, hb) != cudaSuccess) return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    if (!mesh->d_L && cudaMalloc(&mesh->d_L, tb) != cudaSuccess) return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    if (!mesh->d_Vt && cudaMalloc(&mesh->d_Vt, 3 * tb) != cudaSuccess) return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    const size_t lb = 3 * sizeof(double) * (size_t)std::max<int64_t>(1, mesh->h.n_dof);
    if (mesh->moving && !mesh->d_lift && cudaMalloc(&mesh->d_lift, lb) != cudaSuccess)
      return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    if (mesh->moving && !mesh->d_G && cudaMalloc(&mesh->d_G, lb) != cudaSuccess)
      return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    if (mesh->moving && !mesh->d_fac &&
        cudaMalloc(&mesh->d_fac, sizeof(float) * (size_t)std::max<int64_t>(1, mesh->n_mk32)) != cudaSuccess)
      return fail(DG_ERR_OOM, "Navier-Stokes workspace");
    DG_CUDA(dgk::element_kernel_attributes_ns(mesh->nQmax, mesh->wpb, &mesh->blocks_per_sm_ns, mesh->h.n_curved > 0));
    if (mesh->blocks_per_sm_ns < 1) mesh->blocks_per_sm_ns = 1;
    mesh->mu = mu;
    mesh->Pr = Pr;
  }
  mesh->ns = physics == DG_NAVIER_STOKES;
  DG_CUDA(mesh->build_groups());
  mesh->drop_graphs();
  return DG_OK;
}

dg_status dg_set_scheduler(dg_mesh* mesh, int scheduler) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (scheduler < DG_SCHED_BALANCED || scheduler > DG_SCHED_WEIGHTED) return fail(DG_ERR_ARG, "unknown scheduler");
  if (part_mesh(mesh) && (scheduler == DG_SCHED_STATIC || scheduler == DG_SCHED_WEIGHTED))
    return fail(DG_ERR_UNSUPPORTED, "a partition mesh runs the balanced or naive scheduler");
  mesh->scheduler = scheduler;
  return DG_OK;
}

namespace {
// Per-table cost bins (ns, count) and the per-SM busy times since the last reset.
cudaError_t read_cost(dg_mesh* mesh, unsigned long long* cost, std::vector<unsigned long long>* sm,
                      cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(cost, mesh->d_cost, 2 * dgk::kMaxTabs * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  sm->assign(mesh->num_sms, 0ull);
  return cudaMemcpy(sm->data(), mesh->d_smns, sizeof(unsigned long long) * sm->size(), cudaMemcpyDeviceToHost);
}

double busy_imbalance(const std::vector<unsigned long long>& sm) {
  double mx = 0.0, sum = 0.0;
  for (auto v : sm) { mx = std::max(mx, (double)v); sum += (double)v; }
  double mean = sum / std::max<size_t>(1, sm.size());
  return mean > 0 ? mx / mean - 1.0 : 0.0;
}
}  // namespace

dg_status dg_cost_table(dg_mesh* mesh, double* ns_per_elem, double* imbalance, cudaStream_t stream) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  unsigned long long cost[2 * dgk::kMaxTabs];
  std::vector<unsigned long long> sm;
  DG_CUDA(read_cost(mesh, cost, &sm, stream));
  if (ns_per_elem) {
    // per element type, over every N the mesh (or batch) holds
    double ns[4] = {0, 0, 0, 0}, cnt[4] = {0, 0, 0, 0};
    const auto& tabs = mesh->h.tables.tabs;
    for (size_t t = 0; t < tabs.size(); ++t) {
      ns[tabs[t].type] += (double)cost[2 * t];
      cnt[tabs[t].type] += (double)cost[2 * t + 1];
    }
    for (int t = 0; t < 4; ++t) ns_per_elem[t] = cnt[t] > 0 ? ns[t] / cnt[t] : 0.0;
  }
  if (imbalance) *imbalance = busy_imbalance(sm);
  return DG_OK;
}

dg_status dg_rebalance(dg_mesh* mesh, int force, int* rebuilt, cudaStream_t stream) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  unsigned long long cost[2 * dgk::kMaxTabs];
  std::vector<unsigned long long> sm;
  DG_CUDA(read_cost(mesh, cost, &sm, stream));
  const double imb = busy_imbalance(sm);
  const auto& tabs = mesh->h.tables.tabs;
  // Every table that holds elements must have been timed; otherwise the
  // modelled weights stay.
  bool measured = false, complete = true;
  for (size_t t = 0; t < tabs.size(); ++t) {
    if (cost[2 * t + 1]) measured = true;
    else complete = false;
  }
  bool doit = force || (measured && imb > mesh->threshold);
  if (rebuilt) *rebuilt = doit ? 1 : 0;
  if (doit) {
    std::vector<double> w = mesh->static_weights();
    if (measured && complete)
      for (size_t t = 0; t < tabs.size(); ++t) w[t] = (double)cost[2 * t] / (double)cost[2 * t + 1];
    DG_CUDA(mesh->build_chunks(w.data()));
    mesh->drop_graphs();
  }
  // on the caller's stream: the next launch there is ordered after the reset
  DG_CUDA(cudaMemsetAsync(mesh->d_cost, 0, 2 * dgk::kMaxTabs * sizeof(unsigned long long), stream));
  DG_CUDA(cudaMemsetAsync(mesh->d_smns, 0, (size_t)mesh->num_sms * sizeof(unsigned long long), stream));
  return DG_OK;
}

dg_status dg_set_element_warps(dg_mesh* mesh, int warps) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (warps < 1 || warps > 4) return fail(DG_ERR_ARG, "warps per element must be 1..4");
  mesh->wpb = warps;
  for (int t = 0; t < dgk::kMaxTabs; ++t) mesh->tab_wpb[t] = warps;
  if (mesh->ns) {
    DG_CUDA(dgk::element_kernel_attributes_ns(mesh->nQmax, mesh->wpb, &mesh->blocks_per_sm_ns, mesh->h.n_curved > 0));
    if (mesh->blocks_per_sm_ns < 1) mesh->blocks_per_sm_ns = 1;
  }
  DG_CUDA(mesh->build_groups());
  DG_CUDA(mesh->build_static_chunks());
  mesh->drop_graphs();
  return DG_OK;
}

namespace {

// Cache line: "<device name>|N=<N>|E=<elements>|h<hex>p<prism>y<pyr>t<tet>|s<sched>|f<flux> <warps>"
std::string autotune_key(const dg_mesh* m) {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, m->device);
  std::string k = std::string(p.name) + "|N=" + std::to_string(m->h.N) + "|E=" + std::to_string(m->h.n_elems) + "|h" +
                  std::to_string(m->h.type_count[0]) + "p" + std::to_string(m->h.type_count[1]) + "y" +
                  std::to_string(m->h.type_count[2]) + "t" + std::to_string(m->h.type_count[3]) + "|s" +
                  std::to_string(m->scheduler) + "|f" + std::to_string(m->flux);
  for (auto& ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

// Cache line: "<key> <uniform warps> <warps of table 0>,<table 1>,...".
bool autotune_lookup(const char* path, const std::string& key, int* uniform, std::vector<int>* per_table) {
  FILE* f = path ? std::fopen(path, "r") : nullptr;
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[480], list[480];
    int w = 0;
    if (std::sscanf(line, "%479s %d %479s", k, &w, list) == 3 && key == k && w >= 1 && w <= 4) {
      std::vector<int> v;
      for (char* p = std::strtok(list, ","); p; p = std::strtok(nullptr, ",")) v.push_back(std::atoi(p));
      *uniform = w;
      *per_table = v;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void autotune_store(const char* path, const std::string& key, int warps, const int* tab_wpb, int ntab) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d ", key.c_str(), warps);
  for (int t = 0; t < ntab; ++t) std::fprintf(f, "%s%d", t ? "," : "", tab_wpb[t]);
  std::fprintf(f, "\n");
  std::fclose(f);
}

// Apply per-table warps (values outside 1..4 keep the uniform choice).
dg_status apply_table_warps(dg_mesh* mesh, int uniform, const std::vector<int>& per_table) {
  dg_status s = dg_set_element_warps(mesh, uniform);
  if (s != DG_OK) return s;
  bool differs = false;
  for (size_t t = 0; t < per_table.size() && t < (size_t)dgk::kMaxTabs; ++t)
    if (per_table[t] >= 1 && per_table[t] <= 4 && per_table[t] != uniform) {
      mesh->tab_wpb[t] = per_table[t];
      differs = true;
    }
  if (differs) {
    cudaError_t e = mesh->build_groups();
    if (e != cudaSuccess) return cuda_fail(e, "launch groups");
    mesh->drop_graphs();
  }
  return DG_OK;
}

}  // namespace

// Tile shape per (type, N) table.  For every uniform choice of warps per
// element (1..4) a few steps are timed, and the in-kernel cost probe gives
// each table's time per element at that shape; a table's throughput is its
// resident blocks per SM over that time.  The uniform shape with the fastest
// step is kept unless the per-table best shapes (balanced scheduler only,
// one persistent launch per (N, warps) group) make the step faster still.
dg_status dg_autotune(dg_mesh* mesh, const double* Q_store, double dt, int* best_warps, double* ms_per_step,
                      cudaStream_t stream) {
  if (!mesh || !Q_store) return fail(DG_ERR_ARG, "null argument");
  if (part_mesh(mesh)) return fail(DG_ERR_UNSUPPORTED, "the autotuner times dg_rk_step, which a partition mesh cannot run");
  if (mesh->moving) return fail(DG_ERR_UNSUPPORTED, "the autotuner times the static stage graphs; set the tile shape with dg_set_element_warps");
  const char* cache = std::getenv("DG_AUTOTUNE_CACHE");
  const std::string key = autotune_key(mesh);
  const int ntab = (int)mesh->h.tables.tabs.size();
  {
    int cached = 0;
    std::vector<int> per;
    if (autotune_lookup(cache, key, &cached, &per)) {
      dg_status s = apply_table_warps(mesh, cached, per);
      if (s != DG_OK) return s;
      if (best_warps) *best_warps = cached;
      if (ms_per_step) for (int g = 0; g < 5; ++g) ms_per_step[g] = 0.0;
      return DG_OK;
    }
  }
  double *Qs = nullptr, *Ks = nullptr;
  const size_t bytes = sizeof(double) * mesh->h.n_dof;
  DG_CUDA(cudaMalloc(&Qs, bytes));
  if (cudaMalloc(&Ks, bytes) != cudaSuccess) {
    cudaFree(Qs);
    return fail(DG_ERR_OOM, "autotune scratch");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = 3;
  auto time_steps = [&](double* per) -> dg_status {
    cudaMemcpyAsync(Qs, Q_store, bytes, cudaMemcpyDeviceToDevice, stream);
    dg_status st = dg_rk_step(mesh, Qs, Ks, dt, 1, stream);  // captures this shape's graph
    if (st != DG_OK) return st;
    cudaMemsetAsync(mesh->d_cost, 0, 2 * dgk::kMaxTabs * sizeof(unsigned long long), stream);
    cudaEventRecord(e0, stream);
    for (int r = 0; r < reps && st == DG_OK; ++r) st = dg_rk_step(mesh, Qs, Ks, dt, 1, stream);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *per = ms / reps;
    return st;
  };
  double best = 1e300;
  int bestg = mesh->wpb;
  std::vector<std::vector<double>> score(5, std::vector<double>(ntab, 0.0));
  dg_status st = DG_OK;
  for (int g = 1; g <= 4 && st == DG_OK; ++g) {
    st = dg_set_element_warps(mesh, g);
    if (st != DG_OK) break;
    double per = 0.0;
    st = time_steps(&per);
    if (st != DG_OK) break;
    if (ms_per_step) ms_per_step[g - 1] = per;
    if (per < best) {
      best = per;
      bestg = g;
    }
    unsigned long long cost[2 * dgk::kMaxTabs];
    if (cudaMemcpy(cost, mesh->d_cost, sizeof(cost), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = fail(DG_ERR_CUDA, "cost table");
      break;
    }
    for (const auto& G : mesh->groups)
      for (int t : G.tabs)
        if (cost[2 * t + 1] && cost[2 * t]) score[g][t] = (double)G.bpsm * (double)cost[2 * t + 1] / (double)cost[2 * t];
  }
  std::vector<int> per_table(ntab, bestg);
  double mixed = 0.0;
  if (st == DG_OK && mesh->scheduler == DG_SCHED_BALANCED) {
    bool differs = false;
    for (int t = 0; t < ntab; ++t) {
      int bw = bestg;
      for (int g = 1; g <= 4; ++g)
        if (score[g][t] > score[bw][t] * 1.02) bw = g;
      per_table[t] = bw;
      differs |= bw != bestg;
    }
    if (differs) {
      st = apply_table_warps(mesh, bestg, per_table);
      if (st == DG_OK) st = time_steps(&mixed);
      if (st == DG_OK && !(mixed < best)) {
        per_table.assign(ntab, bestg);   // keep the uniform shape
      }
    }
  }
  if (ms_per_step) ms_per_step[4] = mixed;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Qs);
  cudaFree(Ks);
  if (st != DG_OK) return st;
  dg_status s = apply_table_warps(mesh, bestg, per_table);
  if (s != DG_OK) return s;
  autotune_store(cache, key, bestg, per_table.data(), ntab);
  if (best_warps) *best_warps = bestg;
  return DG_OK;
}

dg_status dg_tile_shapes(const dg_mesh* mesh, int max, int* n_tables, int* type, int* N, int* warps) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  int k = 0;
  for (const auto& G : mesh->groups)
    for (int t : G.tabs) {
      if (k < max) {
        if (type) type[k] = mesh->h.tables.tabs[t].type;
        if (N) N[k] = mesh->h.tables.tabs[t].N;
        if (warps) warps[k] = G.wpb;
      }
      ++k;
    }
  if (n_tables) *n_tables = k;
  return DG_OK;
}

dg_status dg_set_table_warps(dg_mesh* mesh, int type, int N, int warps) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  if (warps < 1 || warps > 4) return fail(DG_ERR_ARG, "warps per element must be 1..4");
  const int t = mesh->h.tables.find(type, N);
  if (t < 0) return fail(DG_ERR_ARG, "no such (type, N) table in the mesh");
  mesh->tab_wpb[t] = warps;
  DG_CUDA(mesh->build_groups());
  mesh->drop_graphs();
  return DG_OK;
}

dg_status dg_set_stage_fusion(dg_mesh* mesh, int fused) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  mesh->fused = fused != 0;
  return DG_OK;
}

dg_status dg_set_profiling(dg_mesh* mesh, int on) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  mesh->profiling = on != 0;
  return DG_OK;
}

dg_status dg_phase_times(dg_mesh* mesh, double* out, cudaStream_t stream) {
  if (!mesh || !out) return fail(DG_ERR_ARG, "null argument");
  DG_CUDA(cudaStreamSynchronize(stream));
  for (int i = 0; i < 4; ++i) out[i] = 0.0;
  if (mesh->last_pool < 0) return DG_OK;
  const int p = mesh->last_pool;
  for (int k = 0; k < 2; ++k) {
    const auto& v = k == 0 ? mesh->ev_elem[p] : mesh->ev_face[p];
    for (const auto& ab : v) {
      float ms = 0.f;
      DG_CUDA(cudaEventElapsedTime(&ms, ab.first, ab.second));
      out[k] += ms;
    }
    out[2 + k] = (double)v.size();
  }
  return DG_OK;
}

dg_status dg_moving_phase_times(dg_mesh* mesh, double* out, cudaStream_t stream) {
  if (!mesh || !out) return fail(DG_ERR_ARG, "null argument");
  DG_CUDA(cudaStreamSynchronize(stream));
  for (int i = 0; i < 4; ++i) out[i] = 0.0;
  for (int k = 0; k < 2; ++k) {
    const auto& v = k == 0 ? mesh->ev_geom : mesh->ev_mass;
    for (const auto& ab : v) {
      float ms = 0.f;
      DG_CUDA(cudaEventElapsedTime(&ms, ab.first, ab.second));
      out[k] += ms;
    }
    out[2 + k] = (double)v.size();
  }
  return DG_OK;
}

dg_status dg_sync(dg_mesh* mesh, cudaStream_t stream) {
  if (!mesh) return fail(DG_ERR_ARG, "null mesh");
  DG_CUDA(cudaStreamSynchronize(stream));
  unsigned st = 0;
  DG_CUDA(cudaMemcpy(&st, mesh->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  // the flag is cleared on the caller's stream, so the next launch there
  // starts from a clean status
  if (st & 4u) {
    DG_CUDA(cudaMemsetAsync(mesh->d_status, 0, sizeof(unsigned), stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return fail(DG_ERR_MESH, "the moving mesh turned an element inside out (J or the face area reached zero)");
  }
  if (st & 1u) {
    DG_CUDA(cudaMemsetAsync(mesh->d_status, 0, sizeof(unsigned), stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return fail(DG_ERR_NONFINITE, "a non-finite state value was produced");
  }
  return DG_OK;
}

}  // extern "C"
