"""Benchmark of the modal DG hot path on GB300.

Workload (one "step" = one LSERK(5,4) time step = 5 RHS evaluations + stage
updates): periodic [-pi, pi]^3 box of 16^3 cubes, mixed hexahedra / prisms /
pyramids (seeded recipe of dg_inputs, seed 2), N = 4, compressible Euler,
Taylor-Green vortex state, LF flux, dt from CFL 0.5, FP64.  The inputs are
resident in HBM; the working set (state, register, nodal residual, face
buffers: ~180 MB) exceeds the 129 MB L2, so no flush is needed between steps.

Metric: FP64 DOF-updates/s per RK stage (DOF = sum of modal coefficients per
variable, the paper's performance-index denominator, Sec. 4), for the
SFC-balanced persistent scheduler; the naive per-type scheduler, the Roe flux,
the end-to-end rate through host buffers and the roofline of the dominant
kernel are reported beside it.  --impl reference times the CPU oracle (the
reference arm of this benchmark) on a bounded sample of the same workload.

Under torchrun (N > 1) every rank advances its own independent copy of the
workload (instance-parallel replicas; no data-path collective), the timed
region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

# The CPU legs (oracle timing) run single-threaded; set before NumPy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dg_inputs as di  # noqa: E402

MESH_M, MESH_SEED, N_DEG, CFL = 16, 2, 4, 0.5
GAMMA = 1.4
WORKLOAD = "16^3-cube periodic box, mixed hex/prism/pyramid (seed 2), N=4, Euler TGV (Ma 0.1), LF, CFL 0.5, FP64"
METRIC = "FP64 RHS DOF-updates/s per RK stage (balanced vs naive); adjoint/forward cost"


def workload_config(box, faces, dof, dt, flux, ws):
    """The workload part of the JSON line's config (the same for both arms)."""
    counts = [int((box.etype == t).sum()) for t in range(4)]
    return {"workload": WORKLOAD, "elements": box.n_elems,
            "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), counts)), "faces": faces,
            "dof_per_var": dof, "dt": dt, "flux": flux,
            "l2": "working set ~180 MB > 129 MB L2 (no flush)", "parallelism": f"replicas x{ws}"}


# ----------------------------------------------------------------------------- model
def n_modes(t, N):
    n = N + 1
    return {0: n ** 3, 1: n * n * (n + 1) // 2, 2: n * (n + 1) * (2 * n + 1) // 6, 3: n * (n + 1) * (n + 2) // 6}[t]


def element_flops(t, N):
    """Algorithmic FP64 flops of one element for one stage in the schedule the
    kernels implement (FMA = 2 flops; division and square root count 1):
    modal->nodal and nodal->modal sum-factorised passes, collocation volume
    derivative (3 n^4 per variable), face traces and lifts (n^3 per face and
    variable each), contravariant flux per volume point, diagonal mass
    projection and the LSERK update.  A hexahedron is stored in scaled nodal
    values, so its two transforms are pointwise scales (one multiply per
    point and variable each) instead of sum-factorised passes."""
    n = N + 1
    nM = n_modes(t, N)
    fwd, bwd = transform_macs(t, N)
    nf = (6, 5, 5, 4)[t]
    macs_per_var = fwd + bwd + 3 * n ** 4 + 2 * nf * n ** 3
    metric = (9, 15, 21, 27)[t]
    pointwise = n ** 3 * (61 + metric) + (2 * 5 * n ** 3 if t == 0 else 0)
    epilogue = 5 * nM * (2 + 5)
    return 2 * 5 * macs_per_var + pointwise + epilogue


def transform_macs(t, N):
    """MACs per variable of the storage -> nodal and nodal -> storage
    transforms: the c, b, a passes and their transposes for prism, pyramid
    and tetrahedron (modal storage); none for the hexahedron, whose storage
    W^{1/2} V Q turns both into pointwise scales."""
    if t == 0:
        return 0, 0
    n = N + 1
    nM = n_modes(t, N)
    T = n * (n + 1) // 2
    ncols = n * n if t == 2 else T
    bsum = n * n * (n * n if t == 2 else T)               # sum_p blen(p) n^2
    fwd = n * nM + bsum + n ** 4                            # c, b, a passes
    bwd = n ** 4 + ncols * n * n + nM * n                   # a^T, b^T, c^T
    return fwd, bwd


FACE_POINT_FLOPS = {"lf": 101, "roe": 214}


def curved_element_flops(t, N):
    """element_flops of a curved element: the pointwise metric is read
    instead of formed (no metric flops), a hexahedron scales its nodal
    residual by 1/J_q (5 n^3), a prism or pyramid applies its dense inverse
    mass matrix (2 * 5 nM^2) instead of the diagonal one; tetrahedra stay
    affine."""
    if t == 3:
        return element_flops(t, N)
    n = N + 1
    nM = n_modes(t, N)
    metric = (9, 15, 21, 27)[t]
    base = element_flops(t, N) - n ** 3 * metric
    return base + (5 * n ** 3 if t == 0 else 2 * 5 * nM * nM)


def curved_element_bytes(t, N):
    """element_bytes plus the curved element's pointwise geometry: metric,
    J and 1/J per volume point, and for prism / pyramid the dense inverse
    mass matrix."""
    if t == 3:
        return element_bytes(t, N)
    n = N + 1
    nM = n_modes(t, N)
    return element_bytes(t, N) - 8 * 10 + 8 * (9 * n ** 3 + (n ** 3 if t == 0 else nM * nM))


def ns_element_flops(t, N):
    """Algorithmic FP64 flops of one element for one Navier-Stokes stage:
    the fused backward + forward launch (no volume term there) and the BR1
    volume launch (per direction: lifting volume term, face lift, V^T, V and
    gradient traces; then the total flux and the volume residual)."""
    n = N + 1
    nM = n_modes(t, N)
    fwd, bwd = transform_macs(t, N)
    nf = (6, 5, 5, 4)[t]
    metric = (9, 15, 21, 27)[t]
    nQ = n ** 3
    fused = 2 * 5 * (fwd + bwd + 2 * nf * n ** 3) + 5 * nM * 7 + (2 * 5 * nQ if t == 0 else 0)
    # per direction: lifting volume term, face lift, projection V M^-1 V^T
    # (pointwise 1/w for the hexahedron, whose V is square) and gradient traces
    proj = 5 * nQ if t == 0 else 2 * 5 * (bwd + fwd)
    per_dir = 2 * 5 * (2 * nf * n ** 3) + proj
    # lifting volume terms through the reference directions: one directional
    # pass per structurally nonzero entry of d(a,b,c)/dxi (3/4/5/6 for
    # hex/prism/pyramid/tet), then the 3x3 metric combination per point
    nz = (3, 4, 5, 6)[t]
    lift_volume = 2 * 5 * nz * n ** 4 + nQ * (13 + 5 * nz + 2 * 5 * 9)
    volume = lift_volume + 3 * per_dir + 2 * 5 * 3 * n ** 4 + nQ * (61 + metric + 13 + 66 + 72)
    return fused + volume


# per face point: lifting values (two primitive conversions and the mean) and
# the Navier-Stokes flux (inviscid Riemann flux plus two viscous fluxes and
# their normal components)
FACE_POINT_FLOPS_NS = {"lift": 36, "lf": 101 + 2 * (13 + 66 + 30) + 10, "roe": 214 + 2 * (13 + 66 + 30) + 10}

# dram__bytes_read.sum + dram__bytes_write.sum of one fused element launch
# (backward + LSERK + forward) of this workload, from the ncu capture
# summarised in profiles/element_kernel_16cube_N4.md; set to None whenever
# the element kernel changes until it is captured again.
NCU_TRAFFIC_FUSED_LAUNCH = (186.212096 + 145.397760) * 1e6


def element_bytes(t, N):
    """Algorithmic HBM bytes of one element for one stage: Q, K read and
    written, the nodal residual H written and read back, own-face traces
    written and face fluxes read back, geometry."""
    n = N + 1
    nM = n_modes(t, N)
    nf = (6, 5, 5, 4)[t]
    return 8 * (4 * 5 * nM + 2 * 5 * n ** 3 + 2 * nf * 5 * n * n + 10)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def build_workload(flux="lf"):
    box = di.box_mesh(MESH_M, "mixed", seed=MESH_SEED)
    return box


def h_min(m):
    """Smallest element size h_e = 6 Vol / Area(boundary) of the m^3-cube box:
    all cubes have the same size, so it is the pyramid's (a cube face as base,
    the cube centre as apex)."""
    h_cube = 2 * math.pi / m
    vol = h_cube ** 3 / 6.0
    slant = 0.5 * h_cube * math.sqrt(h_cube ** 2 / 4 + h_cube ** 2 / 4)
    area = h_cube ** 2 + 4 * slant
    return 6 * vol / area


def tgv_smax(mesh_xyz):
    rho, u, v, w, p = di.tgv_primitive(mesh_xyz)
    return float(np.max(np.sqrt(u * u + v * v + w * w) + np.sqrt(GAMMA * p / rho)))


def tgv_dt(box, mesh_xyz, N, m=MESH_M):
    """dt = CFL * min_e h_e / ((2N+1) max_q(|u| + c)), evaluated once from the
    initial state."""
    return CFL * h_min(m) / ((2 * N + 1) * tgv_smax(mesh_xyz))


def dist_helpers(ws, dev):
    """barrier() and max_over_ranks(x) of the replica run (torch.distributed
    already initialised when ws > 1; CPU tensors on the gloo backend)."""
    import torch

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        if ws == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def replica_value(ws, dof, steps, ms):
    """Whole-job DOF-updates/s: every rank advanced its own copy of `dof`
    modal coefficients per variable for `steps` LSERK steps (5 stages), and
    `ms` is the slowest rank's time."""
    return ws * dof * 5 * steps / (ms * 1e-3)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- reference arm
class OracleSample:
    """The CPU oracle on a fixed seeded sample of elements of the workload
    (the TGV projected on the sample and its face neighbours): one 'step' is 5
    residual evaluations of the sample (one LSERK step's worth)."""

    def __init__(self, flux, size):
        from oracle.dg import Oracle
        from oracle.mesh import from_box
        box = build_workload()
        self.box = box
        self.n_elems = box.n_elems
        self.o = o = Oracle(from_box(box, N_DEG), flux=flux)
        self.dof_total = int(o.mesh.nM.sum())
        xyz = np.concatenate([o.quad_points(e) for e in range(box.n_elems)])
        self.dt = tgv_dt(box, xyz, N_DEG)
        rng = np.random.default_rng(0)
        self.sample = np.sort(rng.choice(box.n_elems, size=size, replace=False))
        self.Q = np.zeros(o.mesh.n_dof())
        touched = set(self.sample.tolist())
        for e in self.sample:
            for f, _ in o.mesh.elem_faces[e]:
                e0, _, e1, _ = o.mesh.faces[f]
                touched.update((e0, e1))
        for e in touched:
            op = o.ops[o.mesh.etype[e]]
            q = di.tgv_state(o.quad_points(e))
            r = o.mesh.J[e] * (q * op.w) @ op.V
            self.Q[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = o.apply_minv(e, r).ravel()
        self.dof = int(sum(o.mesh.nM[e] for e in self.sample))

    def step(self):
        for _ in range(5):
            self.o.rhs(self.Q, elems=self.sample)

    def describe(self):
        return f"{len(self.sample)} of {self.n_elems} elements (seeded), 5 residual evaluations per step, 1 thread"


def run_reference(args):
    """The CPU oracle timed on this host on a bounded sample of the workload."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    smp = OracleSample(args.flux, args.ref_sample)
    for _ in range(args.warmup):
        smp.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.step()
    dt = time.perf_counter() - t0
    value = smp.dof * 5 * args.steps / dt
    sample_txt = smp.describe()
    cfg = workload_config(smp.box, len(smp.o.mesh.faces), smp.dof_total, smp.dt, args.flux, ws)
    cfg["sample"] = sample_txt
    line = {"metric": METRIC, "value": value, "unit": "DOF-updates/s",
            "impl": "reference", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle", "sample": sample_txt},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(flux, seconds=12.0, size=48):
    """Oracle throughput on the same bounded sample as the reference arm
    (one warm-up step, then steps for about `seconds` of CPU work)."""
    smp = OracleSample(flux, size)
    smp.step()
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        smp.step()
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": smp.dof * 5 * steps / dt, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{smp.describe()}, {steps} steps in {dt:.1f} s"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_2511_08020_gb300 as dg
    dg.load()
    box = build_workload()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    barrier, max_over_ranks = dist_helpers(ws, dev)
    if args.curved_only:
        # profiling aid: the curved-geometry leg alone (its affine ratio is omitted)
        cv = curved_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, None)
        if rank == 0:
            print(json.dumps({"metric": "FP64 RHS DOF-updates/s per RK stage (curved mesh)",
                              "value": cv["balanced"]["value"], "unit": "DOF-updates/s", "curved": cv,
                              "curved_only": True}), flush=True)
        return

    def make(flux, sched):
        mesh = dg.Mesh(box, N_DEG, flux=flux, scheduler=sched)
        n = N_DEG + 1
        xyz = mesh.quad_points()
        vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
        Q0 = mesh.project(torch.from_numpy(vals).to(dev))
        return mesh, Q0, xyz

    mesh, Q0, xyz = make(args.flux, "balanced")
    dt = tgv_dt(box, xyz, N_DEG)
    dof = int(sum(n_modes(int(t), N_DEG) for t in box.etype))
    counts = mesh.type_counts


    def timed_steps(m, Q, K, steps, warmup, profile=False):
        m.set_profiling(profile)
        for _ in range(warmup):
            m.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        elem_ms = face_ms = 0.0
        nel = nfa = 0
        e0.record(stream)
        for _ in range(steps):
            m.rk_step(Q, K, dt, 1)
            if profile:
                a, b, c, d = m.phase_times()
                elem_ms += a
                face_ms += b
                nel += c
                nfa += d
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1))
        return ms, (elem_ms, face_ms, nel, nfa)

    # tile shape (warps per element) chosen by the library's autotuner per scheduler
    tuned = {}
    for sched in ("naive", "static", "balanced"):
        mesh.set_scheduler(sched)
        if args.warps:
            mesh.set_element_warps(args.warps)
            tuned[sched] = (args.warps, np.zeros(4))
        else:
            tuned[sched] = mesh.autotune(Q0, dt)
    tuned_ms = {k: [round(x, 3) for x in v[1].tolist()] for k, v in tuned.items()}
    shapes_main = mesh.tile_shapes()      # the balanced configuration the main leg times

    # main measurement: balanced scheduler, LF
    Q = Q0.clone()
    K = torch.empty_like(Q)
    clocks = ClockSampler(local)
    clocks.start()
    ms, _ = timed_steps(mesh, Q, K, args.steps, args.warmup)
    clk = clocks.stop()
    mesh.sync()
    value = replica_value(ws, dof, args.steps, ms)

    # kernel split (events inside the replayed graph), same workload
    Qp = Q0.clone()
    msp, (elem_ms, face_ms, nel, nfa) = timed_steps(mesh, Qp, K, max(2, args.steps // 2), 1, profile=True)
    mesh.set_profiling(False)
    steps_p = max(2, args.steps // 2)
    el_flops_stage = sum(element_flops(int(t), N_DEG) for t in box.etype)
    face_flops_stage = mesh.n_faces * (N_DEG + 1) ** 2 * FACE_POINT_FLOPS[args.flux]
    el_bytes_stage = sum(element_bytes(int(t), N_DEG) for t in box.etype)
    # element work per step is exactly 5 stages (a forward-only prime, 4 fused
    # backward+forward phases and a backward-only last phase)
    elem_tflops = el_flops_stage * 5 * steps_p / (elem_ms * 1e-3) / 1e12
    face_tflops = face_flops_stage * 5 * steps_p / (face_ms * 1e-3) / 1e12
    total_tflops = (el_flops_stage + face_flops_stage) * 5 * args.steps / (ms * 1e-3) / 1e12 / ws

    if args.only_main:
        # profiling aid: the main measurement (and the Navier-Stokes and curved legs) only
        line = {"metric": METRIC, "value": value, "unit": "DOF-updates/s",
                "ms_per_step": ms / args.steps, "element_ms_per_step": elem_ms / steps_p,
                "face_ms_per_step": face_ms / steps_p, "element_tflops": elem_tflops, "only_main": True}
        if args.ns_steps > 0:
            line["navier_stokes"] = ns_leg(dg, dev, stream, args, barrier, max_over_ranks, ws)
        if args.curved_steps > 0:
            line["curved"] = curved_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, value)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    dfma, dmma = dg.probe_fp64_peak()
    fp64_mixed = dg.probe_fp64_mixed()
    # ALU roofline: FP64 peak from unit counts and clocks -- every SM retires
    # 2 DFMA per clock (the sm__inst_executed_pipe_fp64 peak ncu reports for
    # this part), 2 flops each, at the maximum SM clock seen during the run
    props = torch.cuda.get_device_properties(dev)
    sm_max_ghz = (clk.get("sm_max_mhz") or 2070.0) / 1e3
    peak_derived = props.multi_processor_count * 2 * 2 * sm_max_ghz / 1e3

    # naive scheduler and Roe flux, same workload and state
    mesh.set_scheduler("naive")
    mesh.set_element_warps(tuned["naive"][0])
    Qn = Q0.clone()
    ms_naive, _ = timed_steps(mesh, Qn, K, args.steps, args.warmup)
    mesh.set_scheduler("static")
    mesh.set_element_warps(tuned["static"][0])
    Qst = Q0.clone()
    ms_static, _ = timed_steps(mesh, Qst, K, args.steps, args.warmup)
    # the paper's balanced partition: equal-weight Hilbert segments with the
    # per-type weights the in-kernel timers measured (dg_rebalance reads them)
    _, imb_static = mesh.cost_table()
    mesh.rebalance(force=True)
    mesh.set_scheduler("weighted")
    Qwt = Q0.clone()
    ms_weighted, _ = timed_steps(mesh, Qwt, K, args.steps, args.warmup)
    _, imb_weighted = mesh.cost_table()
    mesh.set_scheduler("balanced")
    mesh.set_element_warps(tuned["balanced"][0])
    mesh.set_stage_fusion(False)
    Qsp = Q0.clone()
    ms_split, _ = timed_steps(mesh, Qsp, K, args.steps, args.warmup)
    mesh.set_stage_fusion(True)
    split_value = ws * dof * 5 * args.steps / (ms_split * 1e-3)
    naive_value = ws * dof * 5 * args.steps / (ms_naive * 1e-3)
    static_value = ws * dof * 5 * args.steps / (ms_static * 1e-3)
    weighted_value = ws * dof * 5 * args.steps / (ms_weighted * 1e-3)
    same_bits = (bool(torch.equal(Qn, Q)) and bool(torch.equal(Qst, Q)) and bool(torch.equal(Qsp, Q))
                 and bool(torch.equal(Qwt, Q)))

    roe_mesh, Q0r, _ = make("roe", "naive")
    roe_mesh.autotune(Q0r, dt)
    Qrn = Q0r.clone()
    ms_roe_naive, _ = timed_steps(roe_mesh, Qrn, torch.empty_like(Qrn), args.steps, args.warmup)
    roe_naive_value = ws * dof * 5 * args.steps / (ms_roe_naive * 1e-3)
    roe_mesh.set_scheduler("balanced")
    roe_mesh.autotune(Q0r, dt)
    Qr = Q0r.clone()
    ms_roe, _ = timed_steps(roe_mesh, Qr, torch.empty_like(Qr), args.steps, args.warmup)
    roe_value = ws * dof * 5 * args.steps / (ms_roe * 1e-3)

    # adjoint / forward cost: dg_rk_vjp over K steps (checkpoints every 5 steps,
    # and one segment) against K forward steps, same workload, LF, balanced
    Kadj = 10
    Qa = Q0.clone()
    Ka = torch.empty_like(Qa)
    wbar = torch.ones_like(Qa)
    mesh.rk_step(Qa, Ka, dt, Kadj)          # capture the K-step graph
    mesh.rk_vjp(Q0, dt, Kadj, 5, wbar)      # allocate the adjoint workspace
    torch.cuda.synchronize()

    def device_ms(fn, reps=2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    fwd_ms = device_ms(lambda: mesh.rk_step(Qa, Ka, dt, Kadj))
    adj5_ms = device_ms(lambda: mesh.rk_vjp(Q0, dt, Kadj, 5, wbar))
    adjK_ms = device_ms(lambda: mesh.rk_vjp(Q0, dt, Kadj, Kadj, wbar))
    mesh.set_adjoint_storage(False)
    adj5r_ms = device_ms(lambda: mesh.rk_vjp(Q0, dt, Kadj, 5, wbar))
    mesh.set_adjoint_storage(True)
    # autograd split: the forward keeps the segment-start checkpoints, the
    # backward recomputes the segments from them
    Qc = Q0.clone()
    ck = mesh.rk_step_checkpointed(Qc, Ka, dt, Kadj, 5)
    fwdc_ms = device_ms(lambda: mesh.rk_step_checkpointed(Qc, Ka, dt, Kadj, 5, ck))
    adjc_ms = device_ms(lambda: mesh.rk_vjp_checkpointed(ck, dt, Kadj, 5, wbar))
    rhs_ms = device_ms(lambda: mesh.rhs(Q0), reps=5)
    vjp_ms = device_ms(lambda: mesh.rhs_vjp(Q0, wbar), reps=5)
    mesh.sync()

    # measured per-type cost table from the balanced kernels
    ns_type, imb = mesh.cost_table()

    # end to end through the C ABI with host buffers: every step uploads its
    # input state from pinned host memory, permutes it into the storage layout
    # (dg_set_state), advances it (dg_rk_step), permutes it back (dg_get_state)
    # and reads the result to pinned host memory.  The copies run on their own
    # streams, double-buffered, so the upload of step k+1 and the read-back of
    # step k-1 overlap the compute of step k.
    host_in = torch.from_numpy(mesh.get_state(Q0)).pin_memory()
    host_out = [torch.empty(mesh.n_dof, dtype=torch.float64).pin_memory() for _ in range(2)]
    dev_in = [torch.empty(mesh.n_dof, dtype=torch.float64, device=dev) for _ in range(2)]
    dev_out = [torch.empty(mesh.n_dof, dtype=torch.float64, device=dev) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    Qe = mesh.empty()
    Ke = torch.empty_like(Qe)

    def e2e_steps(nsteps):
        ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in_ready", "in_used", "out_ready", "out_done")}
        used = {k: [False, False] for k in ev}
        for k in range(nsteps):
            b = k % 2
            if used["in_used"][b]:
                h2d.wait_event(ev["in_used"][b])
            with torch.cuda.stream(h2d):
                dev_in[b].copy_(host_in, non_blocking=True)
            ev["in_ready"][b].record(h2d)
            stream.wait_event(ev["in_ready"][b])
            mesh.set_state(dev_in[b], Qe, stream=stream)
            ev["in_used"][b].record(stream)
            used["in_used"][b] = True
            mesh.rk_step(Qe, Ke, dt, 1, stream=stream)
            if used["out_done"][b]:
                stream.wait_event(ev["out_done"][b])
            mesh.get_state(Qe, out=dev_out[b], stream=stream)
            ev["out_ready"][b].record(stream)
            d2h.wait_event(ev["out_ready"][b])
            with torch.cuda.stream(d2h):
                host_out[b].copy_(dev_out[b], non_blocking=True)
            ev["out_done"][b].record(d2h)
            used["out_done"][b] = True
        torch.cuda.synchronize()

    e2e_steps(args.warmup)
    barrier()
    t0 = time.perf_counter()
    e2e_steps(args.steps)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = ws * dof * 5 * args.steps / e2e_s
    e2e_ok = bool(torch.equal(torch.from_numpy(mesh.get_state(Qe)), host_out[(args.steps - 1) % 2]))

    # per step: a forward prime and 5 element phases per launch group
    # (tables sharing N and tile shape), and 5 face phases
    n_groups = len({(N, w) for _, N, w in shapes_main})
    gpu_launches = args.steps * (6 * n_groups + 5)

    # the batch and Navier-Stokes legs time every rank's replica (barriers and
    # the max over ranks inside), so every rank runs them
    batch = batch_leg(dg, dev, stream, args, barrier, max_over_ranks, ws) if args.batch_steps > 0 else None
    nsl = ns_leg(dg, dev, stream, args, barrier, max_over_ranks, ws) if args.ns_steps > 0 else None
    cvl = curved_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, value) if args.curved_steps > 0 else None
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": value, "unit": "DOF-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(box, mesh.n_faces, dof, dt, args.flux, ws), scheduler="balanced"),
        "naive": {"value": naive_value, "ms_per_step": ms_naive / args.steps},
        "static": {"value": static_value, "ms_per_step": ms_static / args.steps, "sm_load_imbalance": imb_static},
        "static_weighted": {"value": weighted_value, "ms_per_step": ms_weighted / args.steps,
                            "sm_load_imbalance": imb_weighted,
                            "what": "equal-weight Hilbert segments, measured per-type weights (the paper's partition)"},
        "balanced_unfused_stages": {"value": split_value, "ms_per_step": ms_split / args.steps},
        "schedulers_bitwise_equal": same_bits,
        "balanced_over_naive": value / naive_value,
        "balanced_over_static": value / static_value,
        "weighted_over_static": weighted_value / static_value,
        "roe": {"balanced": roe_value, "naive": roe_naive_value, "balanced_over_naive": roe_value / roe_naive_value},
        "pid_ns_per_dof_stage": 1e9 / (value / ws),
        # the same rate in the other usual units: all five variables, and
        # volume quadrature points (n^3 per element, the nodal DGSEM count)
        "dof_updates_all_variables": 5 * value,
        "quad_point_updates": value * box.n_elems * (N_DEG + 1) ** 3 / dof,
        "roofline": {"bound": "alu", "kernel": "element kernel (balanced, fused backward+LSERK+forward)",
                     "achieved": elem_tflops, "peak": peak_derived, "unit": "TFLOP/s",
                     "frac": elem_tflops / peak_derived,
                     "peak_kind": f"derived: {props.multi_processor_count} SMs x 2 DFMA/clk x 2 flop x "
                                  f"{sm_max_ghz:.3f} GHz (max SM clock of the run)",
                     "dfma_loop_measured": dfma, "frac_of_dfma_loop": elem_tflops / dfma,
                     "traffic": NCU_TRAFFIC_FUSED_LAUNCH,
                     "traffic_source": "dram read+write of one fused element launch, profiles/element_kernel_16cube_N4.md",
                     "algorithmic_bytes_per_stage": el_bytes_stage, "algorithmic_flops_per_stage": el_flops_stage,
                     "element_ms_per_step": elem_ms / steps_p, "face_ms_per_step": face_ms / steps_p,
                     "face_kernel_tflops": face_tflops, "whole_step_tflops": total_tflops,
                     "dmma_peak_measured": dmma, "dfma_plus_dmma_concurrent_measured": fp64_mixed},
        "cost_table_ns_per_elem": dict(zip(("hex", "prism", "pyramid", "tet"), [round(x, 1) for x in ns_type])),
        "sm_load_imbalance": imb,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 8 * mesh.n_dof,
                "d2h_bytes_per_step": 8 * mesh.n_dof, "read_back_matches": e2e_ok,
                "pipeline": "uploads and read-backs on their own streams, double-buffered"},
        "gpu_launches": gpu_launches, "launch_groups": n_groups,
        "autotune_warps_per_element": {k: v[0] for k, v in tuned.items()},
        "tile_shapes": {f"{('hex', 'prism', 'pyramid', 'tet')[t]}/N{N}": w for t, N, w in shapes_main},
        "autotune_ms_per_step_by_warps": tuned_ms,
        "adjoint_over_forward": adj5_ms / fwd_ms,
        "adjoint": {"steps": Kadj, "forward_ms": fwd_ms, "rk_vjp_ckpt5_ms": adj5_ms, "rk_vjp_one_segment_ms": adjK_ms,
                    "ratio_ckpt5": adj5_ms / fwd_ms, "ratio_one_segment": adjK_ms / fwd_ms,
                    "rk_vjp_ckpt5_recompute_ms": adj5r_ms, "ratio_ckpt5_recompute": adj5r_ms / fwd_ms,
                    "forward_checkpointed_ms": fwdc_ms, "rk_vjp_checkpointed_ms": adjc_ms,
                    "ratio_backward_given_forward_checkpoints": adjc_ms / fwdc_ms,
                    "rhs_ms": rhs_ms, "rhs_vjp_ms": vjp_ms, "rhs_vjp_over_rhs": vjp_ms / rhs_ms},
    }
    if batch is not None:
        line["batch"] = batch
    if nsl is not None:
        line["navier_stokes"] = nsl
    if cvl is not None:
        line["curved"] = cvl
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.flux, args.cpu_seconds)
    print(json.dumps(line), flush=True)


BATCH_WORKLOAD = ("64 independent periodic mixed hex/prism/pyramid boxes, m uniform on 4..20 cubes per "
                  "direction, N uniform on {2,3,4,5} (dg_inputs.batch_workload seed 5), Euler TGV, LF, one "
                  "dt (CFL 0.5 of the finest instance), FP64")


NS_WORKLOAD = ("24^3-cube periodic box, mixed hex/prism/pyramid (prism columns 1/4, pyramid cubes 1/9 of hex "
               "columns, seed 4), N=4, Navier-Stokes TGV Re=1600 (mu=1/1600, Pr=0.72, BR1), LF, CFL 0.5, FP64")


def ns_leg(dg, dev, stream, args, barrier, max_over_ranks, ws):
    """Viscous TGV: one handle in Navier-Stokes mode, balanced and naive."""
    import torch
    m, N = 24, 4
    box = di.box_mesh(m, "mixed", seed=4, p_prism=0.25, p_pyr=1.0 / 9.0)
    mesh = dg.Mesh(box, N, flux=args.flux, scheduler="balanced")
    mesh.set_physics("navier_stokes", 1.0 / 1600.0, 0.72)
    n = N + 1
    xyz = mesh.quad_points()
    vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Q0 = mesh.project(torch.from_numpy(vals).to(dev))
    dt = tgv_dt(box, xyz, N, m)
    del vals, xyz
    dof = int(sum(n_modes(int(t), N) for t in box.etype))
    steps = args.ns_steps

    def timed(Q, K, profile=False):
        mesh.set_profiling(profile)
        for _ in range(args.warmup):
            mesh.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = fa = 0.0
        e0.record(stream)
        for _ in range(steps):
            mesh.rk_step(Q, K, dt, 1)
            if profile:
                a, b, _, _ = mesh.phase_times()
                el += a
                fa += b
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        mesh.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1)), el, fa

    out = {"workload": NS_WORKLOAD, "elements": box.n_elems, "faces": mesh.n_faces, "dof_per_var": dof,
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), mesh.type_counts)), "steps": steps, "dt": dt,
           "unit": "DOF-updates/s"}
    res = {}
    for sched in (("balanced",) if args.only_main else ("naive", "balanced")):
        mesh.set_scheduler(sched)
        if args.warps:
            mesh.set_element_warps(args.warps)
            warps = args.warps
        else:
            warps, _ = mesh.autotune(Q0, dt)
        Q = Q0.clone()
        ms, _, _ = timed(Q, torch.empty_like(Q))
        res[sched] = Q
        out[sched] = {"value": ws * dof * 5 * steps / (ms * 1e-3), "ms_per_step": ms / steps, "warps": warps}
    Qp = Q0.clone()
    _, el_ms, fa_ms = timed(Qp, torch.empty_like(Qp), profile=True)
    el_flops = sum(ns_element_flops(int(t), N) for t in box.etype) * 5 * steps
    fa_flops = mesh.n_faces * n * n * (FACE_POINT_FLOPS_NS["lift"] + FACE_POINT_FLOPS_NS[args.flux]) * 5 * steps
    out["element_kernels_tflops"] = el_flops / (el_ms * 1e-3) / 1e12
    out["face_kernels_tflops"] = fa_flops / (fa_ms * 1e-3) / 1e12
    out["element_ms_per_step"] = el_ms / steps
    out["face_ms_per_step"] = fa_ms / steps
    if "naive" in out:
        out["balanced_over_naive"] = out["balanced"]["value"] / out["naive"]["value"]
        out["schedulers_bitwise_equal"] = bool(torch.equal(res["naive"], res["balanced"]))
    if args.ns_adj_steps > 0:
        # adjoint through K steps (checkpoints every 5 steps) against K
        # forward steps; the seed is all ones (the cost does not depend on it)
        Ka = args.ns_adj_steps
        Qa = Q0.clone()
        Kr = torch.empty_like(Qa)
        seed = torch.ones_like(Qa)
        mesh.rk_step(Qa, Kr, dt, Ka)
        mesh.rk_vjp(Q0, dt, Ka, 5, seed)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.rk_step(Qa, Kr, dt, Ka)
        e1.record(stream)
        mesh.rk_vjp(Q0, dt, Ka, 5, seed)
        e2.record(stream)
        torch.cuda.synchronize()
        fwd_ms, adj_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        ck = mesh.rk_step_checkpointed(Qa, Kr, dt, Ka, 5)
        mesh.rk_vjp_checkpointed(ck, dt, Ka, 5, seed)
        torch.cuda.synchronize()
        e0.record(stream)
        mesh.rk_step_checkpointed(Qa, Kr, dt, Ka, 5, ck)
        e1.record(stream)
        mesh.rk_vjp_checkpointed(ck, dt, Ka, 5, seed)
        e2.record(stream)
        torch.cuda.synchronize()
        fwdc_ms, adjc_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        # automatic segment length (as long as half the free memory allows)
        mesh.rk_vjp(Q0, dt, Ka, 0, seed)
        torch.cuda.synchronize()
        e0.record(stream)
        mesh.rk_vjp(Q0, dt, Ka, 0, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        auto_ms = e0.elapsed_time(e1)
        out["adjoint"] = {"steps": Ka, "ckpt_every": 5, "forward_ms": fwd_ms, "rk_vjp_ms": adj_ms,
                          "adjoint_over_forward": adj_ms / fwd_ms, "forward_checkpointed_ms": fwdc_ms,
                          "rk_vjp_checkpointed_ms": adjc_ms,
                          "backward_given_forward_checkpoints_over_forward": adjc_ms / fwdc_ms,
                          "rk_vjp_auto_segment_ms": auto_ms, "auto_segment_over_forward": auto_ms / fwd_ms}
    if args.ns_ke_adjoint:
        # the adjoint of the final kinetic energy with respect to the initial
        # modal state through all the leg's steps (checkpoints every 5 steps,
        # segments recomputed): seed = dE_k/dQ_K = V^T W J (dke/dU)(U_K)
        mesh.set_scheduler("balanced")
        Qf = Q0.clone()
        Kf = torch.empty_like(Qf)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mesh.rk_step(Qf, Kf, dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        fwd_full = e0.elapsed_time(e1)
        U = mesh.eval_nodal(Qf).view(box.n_elems, 5, n ** 3)
        rho, mom = U[:, 0], U[:, 1:4]
        g = torch.zeros_like(U)
        g[:, 0] = -0.5 * (mom * mom).sum(1) / (rho * rho)
        g[:, 1:4] = mom / rho[:, None]
        seed = mesh.load_vector(g.reshape(-1))
        del U, g
        e0.record(stream)
        grad = mesh.rk_vjp(Q0, dt, steps, 5, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        adj_full = e0.elapsed_time(e1)
        # the autograd split: the forward keeps Q at every segment start, the
        # backward recomputes the segments from them
        Qc = Q0.clone()
        e0.record(stream)
        ck = mesh.rk_step_checkpointed(Qc, Kf, dt, steps, 5)
        e1.record(stream)
        torch.cuda.synchronize()
        fwdc_full = e0.elapsed_time(e1)
        e0.record(stream)
        gradc = mesh.rk_vjp_checkpointed(ck, dt, steps, 5, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        adjc_full = e0.elapsed_time(e1)
        del ck
        out["ke_adjoint"] = {"steps": steps, "ckpt_every": 5, "forward_ms": fwd_full, "rk_vjp_ms": adj_full,
                             "adjoint_over_forward": adj_full / fwd_full,
                             "forward_checkpointed_ms": fwdc_full, "rk_vjp_checkpointed_ms": adjc_full,
                             "backward_given_forward_checkpoints_over_forward": adjc_full / fwdc_full,
                             "gradients_equal": bool(torch.equal(grad, gradc)),
                             "gradient_finite": bool(torch.isfinite(grad).all()),
                             "what": "d E_k(Q_K) / d Q_0 through all steps: dg_rk_vjp from Q_0 (its own forward pass "
                                     "places the checkpoints, segments are recomputed with kept stage data), and "
                                     "the split where the forward keeps the checkpoints"}
    mesh.sync()
    mesh.close()
    return out


CURVED_WORKLOAD = ("16^3-cube periodic box, mixed hex/prism/pyramid (seed 2) with every vertex moved by up to "
                   "0.1 h per coordinate (dg_inputs.perturb_vertices, seed 11): trilinear hexahedra, prisms and "
                   "pyramids with pointwise J and dense per-element M^-1; N=4, Euler TGV, LF, FP64")


def curved_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, affine_value):
    """Curved (non-affine) geometry: the main workload's mesh with perturbed
    vertices, so the projection of Algorithm 1 differs per element (a dense
    M_e^-1 for every prism and pyramid, 1/J_q for every hexahedron)."""
    import torch
    box = di.perturb_vertices(di.box_mesh(MESH_M, "mixed", seed=MESH_SEED), 0.1, seed=11)
    mesh = dg.Mesh(box, N_DEG, flux=args.flux, scheduler="balanced", geometry="vertex")
    n = N_DEG + 1
    xyz = mesh.quad_points()
    vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Q0 = mesh.project(torch.from_numpy(vals).to(dev))
    dt = 0.8 * tgv_dt(box, xyz, N_DEG)
    dof = int(sum(n_modes(int(t), N_DEG) for t in box.etype))
    steps = args.curved_steps
    out = {"workload": CURVED_WORKLOAD, "elements": box.n_elems, "curved_elements": mesh.n_curved,
           "curved_faces": mesh.n_curved_faces, "geometry_mb": mesh.geometry_doubles * 8 / 1e6,
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), mesh.type_counts)), "dof_per_var": dof,
           "steps": steps, "dt": dt, "unit": "DOF-updates/s"}

    def timed(Q, K, profile=False):
        mesh.set_profiling(profile)
        for _ in range(args.warmup):
            mesh.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = fa = 0.0
        e0.record(stream)
        for _ in range(steps):
            mesh.rk_step(Q, K, dt, 1)
            if profile:
                a, b_, _, _ = mesh.phase_times()
                el += a
                fa += b_
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        mesh.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1)), el, fa

    res = {}
    for sched in ("naive", "static", "weighted", "balanced"):
        if sched == "weighted":
            mesh.rebalance(force=True)          # per-type weights measured by the in-kernel timers
        mesh.set_scheduler(sched)
        if args.warps:
            mesh.set_element_warps(args.warps)
            warps = args.warps
        else:
            warps, _ = mesh.autotune(Q0, dt)
        Q = Q0.clone()
        ms, _, _ = timed(Q, torch.empty_like(Q))
        res[sched] = Q
        out[sched] = {"value": ws * dof * 5 * steps / (ms * 1e-3), "ms_per_step": ms / steps, "warps": warps}
    Qp = Q0.clone()
    _, el_ms, fa_ms = timed(Qp, torch.empty_like(Qp), profile=True)
    el_flops = sum(curved_element_flops(int(t), N_DEG) for t in box.etype)
    el_bytes = sum(curved_element_bytes(int(t), N_DEG) for t in box.etype)
    out["balanced_over_naive"] = out["balanced"]["value"] / out["naive"]["value"]
    out["balanced_over_static"] = out["balanced"]["value"] / out["static"]["value"]
    out["weighted_over_static"] = out["weighted"]["value"] / out["static"]["value"]
    out["schedulers_bitwise_equal"] = all(bool(torch.equal(res["naive"], res[k])) for k in res)
    out["curved_over_affine"] = out["balanced"]["value"] / affine_value if affine_value else None
    out["element_ms_per_step"] = el_ms / steps
    out["face_ms_per_step"] = fa_ms / steps
    out["element_kernel_tflops"] = el_flops * 5 * steps / (el_ms * 1e-3) / 1e12
    out["element_kernel_gbs"] = el_bytes * 5 * steps / (el_ms * 1e-3) / 1e9
    out["algorithmic_flops_per_stage"] = el_flops
    out["algorithmic_bytes_per_stage"] = el_bytes
    ns, imb = mesh.cost_table()
    out["cost_table_ns_per_elem"] = dict(zip(("hex", "prism", "pyramid", "tet"), [round(x, 1) for x in ns]))
    out["sm_load_imbalance"] = imb
    out["finite"] = bool(torch.isfinite(res["balanced"]).all())

    def device_ms(fn, reps=2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # adjoint / forward on the curved mesh: dg_rk_vjp through K steps,
    # checkpoints every 5, against K forward steps
    Kadj = 10
    Qa, Ka = Q0.clone(), torch.empty_like(Q0)
    wbar = torch.ones_like(Qa)
    mesh.rk_step(Qa, Ka, dt, Kadj)
    mesh.rk_vjp(Q0, dt, Kadj, 5, wbar)
    torch.cuda.synchronize()
    fwd_ms = device_ms(lambda: mesh.rk_step(Qa, Ka, dt, Kadj))
    adj_ms = device_ms(lambda: mesh.rk_vjp(Q0, dt, Kadj, 5, wbar))
    out["adjoint"] = {"steps": Kadj, "forward_ms": fwd_ms, "rk_vjp_ckpt5_ms": adj_ms, "ratio_ckpt5": adj_ms / fwd_ms}

    # Navier-Stokes (BR1, Re 1600) on the same curved mesh and on its affine
    # original, balanced, tile shapes from the autotuner
    nsteps = max(2, steps // 5)
    ns_out = {"steps": nsteps, "mu": 1.0 / 1600, "Pr": 0.72}
    for name, m in (("curved", mesh),
                    ("affine", dg.Mesh(di.box_mesh(MESH_M, "mixed", seed=MESH_SEED), N_DEG, flux=args.flux))):
        m.set_scheduler("balanced")
        m.set_physics("navier_stokes", 1.0 / 1600, 0.72)
        if name == "affine":
            xa = m.quad_points()
            va = di.tgv_state(xa).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
            Qn0 = m.project(torch.from_numpy(va).to(dev))
        else:
            Qn0 = Q0
        if args.warps:
            m.set_element_warps(args.warps)
        else:
            m.autotune(Qn0, dt)
        Qn = Qn0.clone()
        Kn = torch.empty_like(Qn)
        for _ in range(args.warmup):
            m.rk_step(Qn, Kn, dt, 1)
        torch.cuda.synchronize()
        barrier()
        ms_ns = max_over_ranks(device_ms(lambda: m.rk_step(Qn, Kn, dt, nsteps), reps=1))
        ns_out[name] = {"value": ws * dof * 5 * nsteps / (ms_ns * 1e-3), "ms_per_step": ms_ns / nsteps}
        if name == "affine":
            m.sync()
            m.close()
    ns_out["curved_over_affine"] = ns_out["curved"]["value"] / ns_out["affine"]["value"]
    out["navier_stokes"] = ns_out
    mesh.sync()
    mesh.close()
    return out


def batch_leg(dg, dev, stream, args, barrier, max_over_ranks, ws):
    """Serving-style batch: all instances advance in one handle (one persistent
    element launch and one face launch per phase, one CUDA graph per step)."""
    import torch
    work = di.batch_workload(64, seed=5)
    boxes = [di.box_mesh(m, "mixed", seed=sd) for m, N, sd in work]
    Ns = [N for m, N, sd in work]
    b = dg.Batch(boxes, Ns, flux=args.flux, scheduler="balanced")
    xyz = b.quad_points()
    chunks, off = [], 0
    for box, N in zip(boxes, Ns):
        P = box.n_elems * (N + 1) ** 3
        chunks.append(di.tgv_state(xyz[off:off + P]).reshape(5, box.n_elems, (N + 1) ** 3)
                      .transpose(1, 0, 2).reshape(-1))
        off += P
    Q0 = b.project(torch.from_numpy(np.concatenate(chunks)).to(dev))
    del chunks
    smax = tgv_smax(xyz)
    dt = min(CFL * h_min(m) / ((2 * N + 1) * smax) for m, N, _ in work)
    dof = sum(int(sum(n_modes(int(t), N) for t in box.etype)) for box, N in zip(boxes, Ns))
    el_flops_stage = sum(sum(element_flops(int(t), N) for t in box.etype) for box, N in zip(boxes, Ns))
    steps = args.batch_steps

    def timed(Q, K, profile=False):
        b.set_profiling(profile)
        for _ in range(args.warmup):
            b.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = 0.0
        e0.record(stream)
        for _ in range(steps):
            b.rk_step(Q, K, dt, 1)
            if profile:
                el += b.phase_times()[0]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        b.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1)), el

    out = {"workload": BATCH_WORKLOAD, "instances": len(work), "elements": b.n_elems, "faces": b.n_faces,
           "dof_per_var": dof, "degrees": {str(k): Ns.count(k) for k in sorted(set(Ns))},
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), b.type_counts)), "steps": steps, "dt": dt}
    res = {}
    for sched in ("naive", "balanced"):
        b.set_scheduler(sched)
        warps, tms = b.autotune(Q0, dt)
        Q = Q0.clone()
        K = torch.empty_like(Q)
        ms, _ = timed(Q, K)
        res[sched] = Q
        out[sched] = {"value": ws * dof * 5 * steps / (ms * 1e-3), "ms_per_step": ms / steps, "warps": warps,
                      "autotune_ms_per_step": [round(x, 3) for x in tms.tolist()]}
        if sched == "balanced":
            names = ("hex", "prism", "pyramid", "tet")
            out[sched]["tile_shapes"] = {f"{names[t]}/N{N}": w for t, N, w in b.tile_shapes()}
    Qp = Q0.clone()
    _, el_ms = timed(Qp, torch.empty_like(Qp), profile=True)
    out["unit"] = "DOF-updates/s"
    out["balanced_over_naive"] = out["balanced"]["value"] / out["naive"]["value"]
    out["schedulers_bitwise_equal"] = bool(torch.equal(res["naive"], res["balanced"]))
    out["element_kernel_tflops"] = el_flops_stage * 5 * steps / (el_ms * 1e-3) / 1e12
    ns, imb = b.cost_table()
    out["cost_table_ns_per_elem"] = dict(zip(("hex", "prism", "pyramid", "tet"), [round(x, 1) for x in ns]))
    out["sm_load_imbalance"] = imb
    b.sync()
    b.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--flux", default="lf", choices=["lf", "roe"])
    ap.add_argument("--ref-sample", type=int, default=48)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=10,
                    help="steps of the 64-instance batch leg (0 skips it)")
    ap.add_argument("--warps", type=int, default=0,
                    help="warps per element for every scheduler instead of the autotuner (0: autotune)")
    ap.add_argument("--only-main", action="store_true",
                    help="profiling aid: run the main measurement and the Navier-Stokes leg only")
    ap.add_argument("--ns-steps", type=int, default=200,
                    help="steps of the 24^3 Navier-Stokes TGV leg (0 skips it)")
    ap.add_argument("--ns-adj-steps", type=int, default=20,
                    help="steps of the Navier-Stokes adjoint timing (0 skips it)")
    ap.add_argument("--ns-ke-adjoint", type=int, default=1,
                    help="time the adjoint of the final kinetic energy through all NS steps (0 skips it)")
    ap.add_argument("--curved-steps", type=int, default=100,
                    help="steps of the curved-geometry leg (0 skips it)")
    ap.add_argument("--curved-only", action="store_true",
                    help="profiling aid: run the curved-geometry leg only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
