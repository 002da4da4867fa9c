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


def mass_flops(t, N, weight):
    """FP64 flops of one stage mass-matrix call of one element (weight: the
    product M^ q, else the solve): J^ = sum_k tau_k J_k per point (7), its
    weight (1); hexahedra a pointwise scale per point and variable; prisms
    and pyramids per product the two transforms and the pointwise w J^ (5 per
    point), per solve two products with their subtraction and three FP64
    corrections x += z (the FP32 factor and triangular solves not counted)."""
    n = N + 1
    nQ = n ** 3
    if t == 0:
        return 7 * nQ + 5 * nQ
    nM = n_modes(t, N)
    fwd, bwd = transform_macs(t, N)
    prod = 2 * 5 * (fwd + bwd) + 5 * nQ
    base = 8 * nQ
    if weight:
        return base + prod
    return base + 2 * (prod + 5 * nM) + 3 * 5 * nM


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


with open(os.path.join(ROOT, "alg_counts.json")) as _f:
    ALG = json.load(_f)["per_point_flops"]
# w S times the Riemann flux per face point, as the face kernel evaluates it
# (derived by counting in tests/test_alg_counts.py)
FACE_POINT_FLOPS = {"lf": ALG["kernel_lf_per_face_point"], "roe": ALG["kernel_roe_per_face_point"]}


def five_pass_element_flops(t, N, flux):
    """The per-element, per-stage flop model written before the kernels
    existed: modal <-> quadrature transforms counted as five C_V passes per
    variable (the forward transform, the projection and three volume-integral
    derivative passes), trace and lift (nM + 2 n^3) MACs per face side each,
    f_F per volume point, the Riemann flux f_R per face point once per face
    (half per element side), and 20 nM for the LSERK update, with f_F and f_R
    counted from the oracle's formulas (alg_counts.json)."""
    n = N + 1
    nM = n_modes(t, N)
    T = n * (n + 1) // 2
    cv = (3 * n ** 4, n ** 4 + 2 * n * n * T, 2 * n ** 4 + n * nM, n ** 4 + n * n * T + n * nM)[t]
    nf = (6, 5, 5, 4)[t]
    fR = ALG["oracle_lf_per_face_point" if flux == "lf" else "oracle_roe_per_face_point"]
    return (2 * 5 * (5 * cv + nf * 2 * (nM + 2 * n ** 3)) + n ** 3 * ALG["f_F_per_point"]
            + n * n * nf / 2 * fR + 20 * nM)


def split_hex_flops(N):
    """Algorithmic flops of one hexahedron for one stage in the entropy-stable
    split form (alg_counts.json, model split_hex): the weak-form element
    without its collocation derivative and contravariant flux, plus every
    unordered node pair of every coordinate line once, every (face state,
    node) pair once, the nodal two-point states and entropy variables, and
    the extrapolated and converted face states."""
    n = N + 1
    f2 = ALG["split_two_point_flux"]
    base = element_flops(0, N) - 2 * 5 * 3 * n ** 4 - n ** 3 * (61 + 9)
    pairs = 3 * n * n * (n * (n - 1) // 2) * (f2 + 2 * 2 * 5)
    face_pairs = 3 * n * n * 2 * n * (f2 + 2 * 2 * 5)
    nodes = n ** 3 * (ALG["split_two_point_state"] + ALG["split_entropy_variables"])
    face_states = 6 * n * n * (2 * 5 * n + ALG["split_from_entropy_variables"])
    return base + pairs + face_pairs + nodes + face_states


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
# (backward + LSERK + forward) of this workload, from the committed ncu
# capture of the element kernel on the 16^3 N = 4 mesh; set to None whenever
# the element kernel changes until it is captured again.
NCU_TRAFFIC_FUSED_LAUNCH = (154.316032 + 144.723456) * 1e6
# the same capture's executed FP64 rate: (2 DFMA + DMUL + DADD thread
# instructions per cycle, all SMs) x the SM clock of the launch, and the FP64
# pipe's busy fraction (the same rule: None once the kernel changes)
NCU_FP64_FUSED_LAUNCH = {"executed_tflops": (2 * 215.843480 + 31.503288 + 1.640137) * 2.073804e9 / 1e12,
                         "fp64_pipe_busy": 0.92798396}
# dram__bytes_read.sum + dram__bytes_write.sum of one stage solve of the
# moving leg (its launches for hexahedra, prisms and pyramids), from the
# committed ncu capture of the mass kernel on the 16^3 N = 4 mesh in motion;
# None whenever the mass kernel changes until it is captured again.
NCU_TRAFFIC_MASS_SOLVE = (10.084608 + (210.038528 + 16.756480) + (233.019648 + 95.310336)) * 1e6


def fp64_probes():
    """Measured FP64 rates of this device from the benchmark's probe library
    (libfp64probe.so, built beside libdg.so): DFMA loop, mma.sync f64 loop,
    and both at once, TFLOP/s."""
    import ctypes

    from paper_2511_08020_gb300.build import PROBE_LIB, build_probe
    if not os.path.exists(PROBE_LIB):
        build_probe()
    lib = ctypes.CDLL(PROBE_LIB)
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    for rc in (lib.fp64_probe_peak(ctypes.byref(a), ctypes.byref(b)), lib.fp64_probe_mixed(ctypes.byref(c))):
        if rc != 0:
            raise RuntimeError(f"FP64 probe failed with CUDA error {rc}")
    return a.value, b.value, c.value


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
    """nvidia-smi clocks and throttle reasons sampled every 50 ms for the whole
    run; every timed region marks its host-time window (after the
    synchronisation that opens it, before the one that closes it is left),
    and the summary keeps the samples that fall inside the windows."""
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.windows = []
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
            self.rows.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def mark(self, name, t0, t1):
        self.windows.append((name, t0, t1))

    def summary(self, names=None):
        """Median SM clock, maximum clock, throttle reasons seen and sample
        counts over the windows (all, or those whose name is in `names`)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        wins = [(a, b) for n, a, b in self.windows if names is None or n in names]
        sm, mx, reasons = [], [], set()
        for t, r in list(self.rows):
            if not any(a <= t <= b for a, b in wins):
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(self.REASONS, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "timed_seconds": round(sum(b - a for a, b in wins), 3)}

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)


# the run's sampler (started by run_ours; the legs mark their timed windows)
CLOCKS = ClockSampler()


class timed_window:
    """Marks a timed region's host-time window in CLOCKS."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *exc):
        CLOCKS.mark(self.name, self.t0, time.monotonic())
        return False


def interleaved_repeats(arms, timed_fn, reps):
    """Scheduler comparison with a spread: `reps` rounds, in each of which
    every arm (name, set-up callable) is set up and timed once by
    timed_fn() -> ms per step; the order rotates every round.  Returns per
    name the repeats' ms per step with their median and quartiles."""
    times = {name: [] for name, _ in arms}
    for r in range(reps):
        k = r % len(arms)
        for name, setup in arms[k:] + arms[:k]:
            setup()
            times[name].append(timed_fn())
    out = {}
    for name, v in times.items():
        q1, med, q3 = np.percentile(v, [25, 50, 75])
        out[name] = {"median_ms_per_step": float(med), "q1_ms_per_step": float(q1), "q3_ms_per_step": float(q3),
                     "repeats": len(v), "ms_per_step": [round(x, 4) for x in v]}
    return out


def compare_to(stats, a, b):
    """Median ratio time(b)/time(a) (> 1: a is faster) and whether the two
    interquartile ranges are disjoint."""
    sa, sb = stats[a], stats[b]
    return {"speedup_median": sb["median_ms_per_step"] / sa["median_ms_per_step"],
            "iqr_disjoint": bool(sa["q3_ms_per_step"] < sb["q1_ms_per_step"]
                                 or sb["q3_ms_per_step"] < sa["q1_ms_per_step"])}


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
def _oracle_worker(conn, flux, elems):
    """A spawned process that owns a fixed part of the element list (so its
    oracle's face tables stay warm): receives states, returns the residual
    blocks of its elements, until it receives None."""
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    o = Oracle(from_box(build_workload(), N_DEG), flux=flux)
    off = o.mesh.dof_off
    conn.send("ready")
    while True:
        Q = conn.recv()
        if Q is None:
            break
        R = o.rhs(Q, elems=elems)
        conn.send(np.concatenate([R[off[e]:off[e + 1]] for e in elems]))
    conn.close()


class OracleRun:
    """The CPU oracle on the benchmark workload, timed in full LSERK steps:
    the residual of `elems` (every element, or a seeded sample whose
    neighbours stay frozen) is evaluated by `cores` spawned worker processes,
    each with its own oracle and one BLAS thread and always the same equal
    part of the element list; the stage updates run in this process.  Initial
    state: the TGV projected with the oracle (Algorithm 1)."""

    def __init__(self, flux, cores, n_sample=None):
        import multiprocessing as mp

        from oracle.dg import LSERK_A, LSERK_B, Oracle
        from oracle.mesh import from_box
        self.A, self.B = LSERK_A, LSERK_B
        box = build_workload()
        self.box = box
        self.o = o = Oracle(from_box(box, N_DEG), flux=flux)
        E = box.n_elems
        self.dof_total = int(o.mesh.nM.sum())
        if n_sample is None or n_sample >= E:
            self.elems = np.arange(E)
            touched = self.elems
        else:
            self.elems = np.sort(np.random.default_rng(0).choice(E, size=n_sample, replace=False))
            t = set(self.elems.tolist())
            for e in self.elems:
                for f, _ in o.mesh.elem_faces[e]:
                    t.update((o.mesh.faces[f][0], o.mesh.faces[f][2]))
            touched = sorted(t)
        self.Q = np.zeros(o.mesh.n_dof())
        xyz = []
        for e in touched:
            op = o.ops[o.mesh.etype[e]]
            x = o.quad_points(e)
            xyz.append(x)
            r = o.mesh.J[e] * (di.tgv_state(x) * op.w) @ op.V
            self.Q[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = o.apply_minv(e, r).ravel()
        self.dt = tgv_dt(box, np.concatenate(xyz), N_DEG)
        self.dof = int(sum(o.mesh.nM[e] for e in self.elems))
        self.parts = [p for p in np.array_split(self.elems, cores) if len(p)]
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for part in self.parts:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, flux, part), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            assert c.recv() == "ready"

    def rhs(self, Q):
        R = np.zeros_like(Q)
        off = self.o.mesh.dof_off
        for c in self.conns:
            c.send(Q)
        for c, part in zip(self.conns, self.parts):
            blocks = c.recv()
            k = 0
            for e in part:
                n = off[e + 1] - off[e]
                R[off[e]:off[e + 1]] = blocks[k:k + n]
                k += n
        return R

    def step(self):
        K = np.zeros_like(self.Q)
        for s in range(5):
            K = self.A[s] * K + self.dt * self.rhs(self.Q)
            self.Q = self.Q + self.B[s] * K

    def describe(self):
        what = "all" if len(self.elems) == self.box.n_elems else f"a seeded sample of {len(self.elems)} of the"
        return (f"{what} {self.box.n_elems} elements, full LSERK steps (5 residual evaluations and stage "
                f"updates), {len(self.parts)} worker process(es), one BLAS thread each")

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=30)


def run_reference(args):
    """The CPU oracle timed on this host's cores: full LSERK steps of the
    workload on every core (a seeded sample of 1024 elements per core when
    the host has too few cores for whole steps within a few minutes)."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    run = OracleRun(args.flux, cores, n_sample=1024 * cores)
    run.rhs(run.Q)                      # warm-up: builds the workers' face tables
    for _ in range(args.warmup):
        run.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step()
    dt = time.perf_counter() - t0
    run.close()
    value = run.dof * 5 * args.steps / dt
    sample_txt = run.describe()
    cfg = workload_config(run.box, len(run.o.mesh.faces), run.dof_total, run.dt, args.flux, ws)
    cfg["sample"] = sample_txt
    line = {"metric": METRIC, "value": value, "unit": "DOF-updates/s",
            "impl": "reference", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": len(run.parts), "kind": "oracle",
                             "sample": sample_txt},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(flux, one_core_sample=256, min_seconds=10.0):
    """The oracle timed on this host, after one warm-up residual evaluation
    (which builds the oracle's face tables): full LSERK steps of the whole
    benchmark mesh on every core (os.cpu_count() worker processes), and on
    one core full LSERK steps of a seeded sample of elements (a whole-mesh
    step on one core needs minutes of face-table set-up alone); in each case
    steps until min_seconds have passed (at least one)."""
    out = {"unit": "DOF-updates/s", "kind": "oracle", "nproc": os.cpu_count()}
    for label, cores, sample in (("all_cores", os.cpu_count() or 1, None), ("one_core", 1, one_core_sample)):
        run = OracleRun(flux, cores, n_sample=sample)
        run.rhs(run.Q)
        steps, t0 = 0, time.perf_counter()
        while True:
            run.step()
            steps += 1
            el = time.perf_counter() - t0
            if el >= min_seconds:
                break
        out[label] = {"value": run.dof * 5 * steps / el, "cores": len(run.parts), "steps": steps,
                      "seconds": round(el, 2), "sample": run.describe()}
        run.close()
    for k in ("value", "cores", "sample"):
        out[k] = out["all_cores"][k]
    return out


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
    CLOCKS.index = local
    CLOCKS.start()
    try:
        run_ours_legs(args, dg, torch, ws, rank, local, box, dev, stream, barrier, max_over_ranks)
    finally:
        CLOCKS.stop()


def run_ours_legs(args, dg, torch, ws, rank, local, box, dev, stream, barrier, max_over_ranks):
    if args.split_only:
        sp = split_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, None)
        if rank == 0:
            print(json.dumps({"metric": "FP64 RHS DOF-updates/s per RK stage (split form on hexahedra)",
                              "value": sp["value"], "unit": "DOF-updates/s", "split_form": sp,
                              "split_only": True}), flush=True)
        return
    if args.moving_only:
        mv = moving_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, None)
        if rank == 0:
            print(json.dumps({"metric": "FP64 RHS DOF-updates/s per RK stage (moving mesh)", "value": mv["value"],
                              "unit": "DOF-updates/s", "moving": mv, "moving_only": True}), flush=True)
        return
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


    def timed_steps(m, Q, K, steps, warmup, profile=False, window="main legs"):
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
        with timed_window(window):
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
    ms, _ = timed_steps(mesh, Q, K, args.steps, args.warmup, window="main")
    clk = CLOCKS.summary(["main"])
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
    five_pass_flops_stage = sum(five_pass_element_flops(int(t), N_DEG, args.flux) for t in box.etype)
    five_pass_tflops = five_pass_flops_stage * 5 * args.steps / (ms * 1e-3) / 1e12 / ws

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

    dfma, dmma, fp64_mixed = fp64_probes()
    # ALU roofline: FP64 peak from unit counts and clocks -- every SM retires
    # 2 DFMA per clock (the sm__inst_executed_pipe_fp64 peak ncu reports for
    # this part), 2 flops each, at the maximum SM clock seen during the run
    props = torch.cuda.get_device_properties(dev)
    sm_max_ghz = (clk.get("sm_max_mhz") or 2070.0) / 1e3
    peak_derived = props.multi_processor_count * 2 * 2 * sm_max_ghz / 1e3

    # scheduler comparison on the same workload and state: one timed run per
    # scheduler (its final state for the bitwise comparison), then
    # interleaved repeats for the spread
    def use(sched):
        def setup():
            mesh.set_scheduler(sched)
            if sched == "balanced" and not args.warps:
                for t, N, w in shapes_main:      # the autotuned per-table tile shapes of the main leg
                    mesh.set_table_warps(t, N, w)
            else:
                mesh.set_element_warps(tuned["static" if sched == "weighted" else sched][0])
        return setup

    use("naive")()
    Qn = Q0.clone()
    ms_naive, _ = timed_steps(mesh, Qn, K, args.steps, args.warmup)
    use("static")()
    Qst = Q0.clone()
    ms_static, _ = timed_steps(mesh, Qst, K, args.steps, args.warmup)
    # the paper's balanced partition: equal-weight Hilbert segments with the
    # per-type weights the in-kernel timers measured (dg_rebalance reads them)
    _, imb_static = mesh.cost_table()
    mesh.rebalance(force=True)
    use("weighted")()
    Qwt = Q0.clone()
    ms_weighted, _ = timed_steps(mesh, Qwt, K, args.steps, args.warmup)
    _, imb_weighted = mesh.cost_table()
    use("balanced")()
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
    rep_steps = max(5, args.steps // 4)
    Qr, Kr = Q0.clone(), torch.empty_like(Q0)

    def timed_rep():
        Qr.copy_(Q0)
        ms_r, _ = timed_steps(mesh, Qr, Kr, rep_steps, 1, window="scheduler repeats")
        return ms_r / rep_steps

    sched_stats = interleaved_repeats([(sd, use(sd)) for sd in ("naive", "static", "weighted", "balanced")],
                                      timed_rep, args.sched_repeats)
    use("balanced")()
    sched_cmp = {"steps_per_repeat": rep_steps, "stats": sched_stats,
                 "balanced_vs_naive": compare_to(sched_stats, "balanced", "naive"),
                 "balanced_vs_static": compare_to(sched_stats, "balanced", "static"),
                 "weighted_vs_static": compare_to(sched_stats, "weighted", "static")}

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

    # per step (one dg_rk_step call): the parameter node of the replayed
    # graphs, a forward prime and 5 element phases per launch group (tables
    # sharing N and tile shape), and 5 face phases
    n_groups = len({(N, w) for _, N, w in shapes_main})
    gpu_launches = args.steps * (1 + 6 * n_groups + 5)

    # the batch and Navier-Stokes legs time every rank's replica (barriers and
    # the max over ranks inside), so every rank runs them
    batch = batch_leg(dg, dev, stream, args, barrier, max_over_ranks, ws) if args.batch_steps > 0 else None
    nsl = ns_leg(dg, dev, stream, args, barrier, max_over_ranks, ws) if args.ns_steps > 0 else None
    cvl = curved_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, value) if args.curved_steps > 0 else None
    mvl = (moving_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, cvl["balanced"]["value"] if cvl else None)
           if args.moving_steps > 0 else None)
    spl = split_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, value) if args.split_steps > 0 else None
    prt = (partitioned_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, rank)
           if args.partition_steps > 0 else None)
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
        "scheduler_repeats": sched_cmp,
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
                     "ncu_fp64": NCU_FP64_FUSED_LAUNCH,
                     "traffic_source": "ncu dram read+write of one fused element launch (16^3 mixed, N = 4)",
                     "algorithmic_bytes_per_stage": el_bytes_stage, "algorithmic_flops_per_stage": el_flops_stage,
                     "element_ms_per_step": elem_ms / steps_p, "face_ms_per_step": face_ms / steps_p,
                     "face_kernel_tflops": face_tflops, "whole_step_tflops": total_tflops,
                     "flop_models": {
                         "schedule": {"flops_per_stage": el_flops_stage + face_flops_stage,
                                      "whole_step_tflops": total_tflops, "frac": total_tflops / peak_derived,
                                      "what": "the sum-factorised schedule the kernels run (element + face kernel)"},
                         "five_pass": {"flops_per_stage": five_pass_flops_stage, "whole_step_tflops": five_pass_tflops,
                                    "frac": five_pass_tflops / peak_derived,
                                    "what": "five C_V passes per variable, trace/lift per face side, f_F and f_R "
                                            "from the oracle's formulas (alg_counts.json); above 1 where the "
                                            "schedule removes work the model counts (hexahedral transforms)"}},
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
    if mvl is not None:
        line["moving"] = mvl
    if spl is not None:
        line["split_form"] = spl
    if prt is not None:
        prt["over_whole_mesh"] = prt["value"] / value if prt["value"] and ws == 1 else None
        line["partitioned"] = prt
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.flux, args.cpu_one_core_sample)
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

    def timed(Q, K, profile=False, nsteps=steps, warmup=args.warmup):
        mesh.set_profiling(profile)
        for _ in range(warmup):
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
        # the adjoint of the whole trajectory may keep stage data in most of
        # the free memory (fewer segments recomputed); freed after the leg
        mesh.set_adjoint_memory(args.ke_adjoint_memory)
        grad = torch.empty_like(seed)
        mesh.rk_vjp(Q0, dt, steps, 5, seed, grad)     # allocates the stage store (untimed)
        torch.cuda.synchronize()
        e0.record(stream)
        mesh.rk_vjp(Q0, dt, steps, 5, seed, grad)
        e1.record(stream)
        torch.cuda.synchronize()
        adj_full = e0.elapsed_time(e1)
        mesh.set_adjoint_storage(False)
        mesh.set_adjoint_storage(True)
        mesh.set_adjoint_memory(0.5)
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
                             "stage_store_share_of_free_memory": args.ke_adjoint_memory,
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


MOVING_WORKLOAD = ("the curved 16^3 mixed box (every vertex moved by up to 0.1 h, seed 11) in motion: vertex v "
                   "at x_v + t u_v with u = 0.5 (sin y sin z, sin z sin x, sin x sin y) "
                   "(dg_inputs.vertex_velocities); per stage the geometry at the stage time from its polynomial "
                   "coefficients, the moving-frame residual, and the mass solve with the LSERK stage value of J "
                   "(Cholesky per prism and pyramid, pointwise for hexahedra); N=4, Euler TGV (and Navier-Stokes "
                   "Re 1600 in the navier_stokes key), LF, FP64")


def moving_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, curved_value):
    """Moving mesh (time-varying geometry): LSERK steps of the mass-weighted
    state with the geometry and the projection of Algorithm 1 evaluated
    afresh at every stage; its cost against the static curved mesh, and the
    share of the per-stage geometry and mass-solve kernels."""
    import torch
    box = di.perturb_vertices(di.box_mesh(MESH_M, "mixed", seed=MESH_SEED), 0.1, seed=11)
    vel = di.vertex_velocities(box.xyz, 0.5)
    mesh = dg.MovingMesh(box, N_DEG, vel, scheduler="balanced")
    warps = args.warps or 4
    mesh.set_element_warps(warps)
    n = N_DEG + 1
    xyz = mesh.quad_points()
    vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Q0 = mesh.project(torch.from_numpy(vals).to(dev))
    dt = 0.8 * tgv_dt(box, xyz, N_DEG)
    dof = int(sum(n_modes(int(t), N_DEG) for t in box.etype))
    steps = args.moving_steps
    out = {"workload": MOVING_WORKLOAD, "elements": box.n_elems, "dof_per_var": dof, "steps": steps, "dt": dt,
           "unit": "DOF-updates/s", "warps": warps,
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), mesh.type_counts))}

    def timed(Q, K, profile=False):
        mesh.set_profiling(profile)
        for _ in range(args.warmup):
            mesh.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ph = np.zeros(6)
        with timed_window("moving"):
            e0.record(stream)
            mesh.rk_step(Q, K, dt, steps)
            e1.record(stream)
            torch.cuda.synchronize()
        if profile:
            a, b_, _, _ = mesh.phase_times()
            g, m, _, nm = mesh.moving_phase_times()
            ph += (a, b_, g, m, nm, 1)
        barrier()
        mesh.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1)), ph

    Q = Q0.clone()
    K = torch.empty_like(Q)
    ms, _ = timed(Q, K)
    mesh.sync()
    out["value"] = ws * dof * 5 * steps / (ms * 1e-3)
    out["ms_per_step"] = ms / steps
    out["mesh_time_end"] = mesh.time
    out["finite"] = bool(torch.isfinite(Q).all())
    Qp = Q0.clone()
    msp, (el, fa, geo, mass, n_mass, _) = timed(Qp, K, profile=True)
    out["element_ms_per_step"] = el / steps
    out["face_ms_per_step"] = fa / steps
    out["geometry_ms_per_step"] = geo / steps
    out["mass_ms_per_step"] = mass / steps
    out["mass_share"] = mass / msp
    out["over_static_curved"] = out["value"] / curved_value if curved_value else None
    # the stage mass kernels: per step five solves (stages 2-5 and the step's
    # end) and the products M Q that ran (the first step of a call; later
    # steps carry M Q over while the stage values stay exact), counted from
    # the mass calls the profiled run made; FP64 flops as the kernels
    # evaluate them (the FP32 Cholesky preconditioner not counted)
    products = max(0.0, n_mass / steps - 5.0)
    fl_step = sum(products * mass_flops(int(t), N_DEG, 1) + 5 * mass_flops(int(t), N_DEG, 0) for t in box.etype)
    achieved = fl_step / (mass / steps * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    clk = CLOCKS.summary(["moving"])
    peak = props.multi_processor_count * 2 * 2 * (clk.get("sm_max_mhz") or 2070.0) / 1e6
    out["clocks"] = clk
    # Navier-Stokes on the same moving mesh (Re 1600 by the TGV scales):
    # the lifting's three extra stage solves for prisms and pyramids
    nsm = dg.MovingMesh(box, N_DEG, vel, scheduler="balanced")
    nsm.set_element_warps(warps)
    nsm.set_physics("navier_stokes", 1.0 / 1600.0, 0.72)
    Qn = nsm.project(torch.from_numpy(vals).to(dev))
    Kn = torch.empty_like(Qn)
    for _ in range(args.warmup):
        nsm.rk_step(Qn, Kn, dt, 1)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with timed_window("moving"):
        e0.record(stream)
        nsm.rk_step(Qn, Kn, dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ns_ms = max_over_ranks(e0.elapsed_time(e1))
    nsm.sync()
    out["navier_stokes"] = {"value": ws * dof * 5 * steps / (ns_ms * 1e-3), "ms_per_step": ns_ms / steps,
                            "mu": 1.0 / 1600.0, "Pr": 0.72, "finite": bool(torch.isfinite(Qn).all()),
                            "over_euler_moving": (ns_ms / steps) and out["ms_per_step"] / (ns_ms / steps)}
    del nsm, Qn, Kn
    out["roofline"] = {"bound": "alu", "kernel": "stage mass kernels (FP64 products, FP32-preconditioned solves)",
                       "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                       "flops_per_step": fl_step, "mass_calls_per_step": n_mass / steps,
                       "products_per_step": products, "traffic_per_solve": NCU_TRAFFIC_MASS_SOLVE,
                       "traffic_source": "ncu dram read+write of one stage solve (three launches, one per "
                                         "element type; 16^3 N = 4 mesh in motion)",
                       "peak_kind": "derived FP64: SMs x 2 DFMA/clk x 2 flop x max SM clock"}
    return out


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

    def timed(Q, K, profile=False, nsteps=steps, warmup=args.warmup):
        mesh.set_profiling(profile)
        for _ in range(warmup):
            mesh.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = fa = 0.0
        with timed_window("curved"):
            e0.record(stream)
            for _ in range(nsteps):
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

    res, wsched = {}, {}
    for sched in ("naive", "static", "weighted", "balanced"):
        if sched == "weighted":
            mesh.rebalance(force=True)          # per-type weights measured by the in-kernel timers
        mesh.set_scheduler(sched)
        if args.warps:
            mesh.set_element_warps(args.warps)
            warps = args.warps
        else:
            warps, _ = mesh.autotune(Q0, dt)
        wsched[sched] = warps
        Q = Q0.clone()
        ms, _, _ = timed(Q, torch.empty_like(Q))
        res[sched] = Q
        out[sched] = {"value": ws * dof * 5 * steps / (ms * 1e-3), "ms_per_step": ms / steps, "warps": warps}

    shapes_cv = mesh.tile_shapes()      # balanced was tuned last: its per-table shapes

    def use(sched):
        def setup():
            mesh.set_scheduler(sched)
            if sched == "balanced" and not args.warps:
                for t, N, w in shapes_cv:
                    mesh.set_table_warps(t, N, w)
            else:
                mesh.set_element_warps(wsched[sched])
        return setup
    rep_steps = max(5, steps // 4)
    Qr, Kr = Q0.clone(), torch.empty_like(Q0)

    def timed_rep():
        Qr.copy_(Q0)
        return timed(Qr, Kr, nsteps=rep_steps, warmup=1)[0] / rep_steps
    stats = interleaved_repeats([(sd, use(sd)) for sd in ("naive", "static", "weighted", "balanced")], timed_rep,
                                args.sched_repeats)
    use("balanced")()
    out["scheduler_repeats"] = {"steps_per_repeat": rep_steps, "stats": stats,
                                "balanced_vs_naive": compare_to(stats, "balanced", "naive"),
                                "balanced_vs_static": compare_to(stats, "balanced", "static"),
                                "weighted_vs_static": compare_to(stats, "weighted", "static")}
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


def partitioned_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, rank):
    """The benchmark mesh partitioned along the Hilbert curve (Sec. 3,
    dg_partition_plan, equal element weights): one part per rank under
    torchrun, the halo traces exchanged every stage by NCCL send/recv; on one
    rank, args.parts parts in this process on this GPU with the exchange by
    device copies.  Steps through dg_rk_prime / dg_rk_stage."""
    import torch
    box = build_workload()
    N = N_DEG
    nparts = ws if ws > 1 else args.parts
    plan = dg.partition_plan(box, N, nparts)[0]
    mine = [rank] if ws > 1 else list(range(nparts))
    parts = [dg.Part(box, N, plan, nparts, p, flux=args.flux) for p in mine]
    n = N + 1
    Qs, Ks = [], []
    for P in parts:
        xyz = P.quad_points()
        vals = di.tgv_state(xyz).reshape(5, P.n_elems, n ** 3).transpose(1, 0, 2).copy()
        Qs.append(P.project(torch.from_numpy(vals).to(dev)))
        Ks.append(torch.empty_like(Qs[-1]))
    dt = tgv_dt(box, dg.check_mesh(box, N)[1], N)
    per = parts[0].doubles_per_face
    bufs = [P.halo_buffers() for P in parts]

    def seg(counts, k):
        a = int(counts[:k].sum()) * per
        return slice(a, a + int(counts[k]) * per)

    if ws > 1:
        import torch.distributed as dist
        P, (send, recv) = parts[0], bufs[0]

        def exchange():
            P.halo_pack(send)
            ops = []
            for q in range(nparts):
                if P.send_faces[q]:
                    ops.append(dist.P2POp(dist.isend, send[seg(P.send_faces, q)], q))
                if P.recv_faces[q]:
                    ops.append(dist.P2POp(dist.irecv, recv[seg(P.recv_faces, q)], q))
            if ops:
                for r in dist.batch_isend_irecv(ops):
                    r.wait()
            P.halo_unpack(recv)
    else:
        def exchange():
            for Pp, (snd, _) in zip(parts, bufs):
                Pp.halo_pack(snd)
            for p in range(nparts):
                for q in range(nparts):
                    if parts[p].send_faces[q]:
                        bufs[q][1][seg(parts[q].recv_faces, p)].copy_(bufs[p][0][seg(parts[p].send_faces, q)])
            for Pp, (_, rcv) in zip(parts, bufs):
                Pp.halo_unpack(rcv)

    owned = [int((P.is_ghost == 0).sum()) for P in parts]
    dof_owned = sum(int(sum(n_modes(int(box.etype[g]), N) for g, gh in zip(P.global_of_local, P.is_ghost) if not gh))
                    for P in parts)
    steps = args.partition_steps
    dg.step_parts(parts, Qs, Ks, dt, args.warmup, exchange)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with timed_window("partitioned"):
        e0.record(stream)
        dg.step_parts(parts, Qs, Ks, dt, steps, exchange)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    total_dof = dof_owned * (ws if ws > 1 else 1)    # each rank owns a different part: the job's DOF
    out = {"parts": nparts, "ranks": ws, "parts_per_gpu": len(parts), "steps": steps, "ms_per_step": ms / steps,
           "value": total_dof * 5 * steps / (ms * 1e-3) if ws == 1 else None, "unit": "DOF-updates/s",
           "owned_elements": owned, "halo_faces_sent": [int(P.send_faces.sum()) for P in parts],
           "exchange": "NCCL send/recv per stage" if ws > 1 else "device copies between parts on one GPU",
           "finite": all(bool(torch.isfinite(Q).all()) for Q in Qs)}
    if ws > 1:
        # every rank owns a disjoint part: the job's rate is the sum of the parts' DOF over the slowest rank's time
        t = torch.tensor([float(dof_owned)], device=dev)
        import torch.distributed as dist
        dist.all_reduce(t)
        out["value"] = float(t.item()) * 5 * steps / (ms * 1e-3)
        out["scaling"] = "strong"
    for P in parts:
        P.sync()
        P.close()
    return out


SPLIT_WORKLOAD = ("16^3-cube periodic box, mixed hex/prism/pyramid (seed 2), N=4, Euler TGV (Ma 0.1), LF, CFL 0.5, "
                  "FP64; hexahedra in the entropy-stable split form (Chandrashekar two-point flux, hybridised Gauss "
                  "SBP lines, entropy-projected traces), prisms and pyramids in the weak form")


def split_leg(dg, dev, stream, args, barrier, max_over_ranks, ws, weak_value):
    """The benchmark mesh with the hexahedra in the entropy-stable split form
    (dg_set_volume_form): balanced and naive, the element kernel's rate
    against the split-form flop model, and the cost per element type."""
    import torch
    box = build_workload()
    mesh = dg.Mesh(box, N_DEG, flux=args.flux, scheduler="balanced")
    mesh.set_volume_form("split")
    n = N_DEG + 1
    xyz = mesh.quad_points()
    vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Q0 = mesh.project(torch.from_numpy(vals).to(dev))
    dt = tgv_dt(box, xyz, N_DEG)
    del vals, xyz
    dof = int(sum(n_modes(int(t), N_DEG) for t in box.etype))
    steps = args.split_steps
    out = {"workload": SPLIT_WORKLOAD, "steps": steps, "dt": dt, "unit": "DOF-updates/s",
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), mesh.type_counts))}

    def timed(Q, K, profile=False, nsteps=steps, warmup=args.warmup):
        mesh.set_profiling(profile)
        for _ in range(warmup):
            mesh.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = fa = 0.0
        with timed_window("split form"):
            e0.record(stream)
            for _ in range(nsteps):
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
    for sched in ("naive", "balanced"):
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
    out["tile_shapes"] = {f"{('hex', 'prism', 'pyramid', 'tet')[t]}/N{N}": w for t, N, w in mesh.tile_shapes()}
    Qp = Q0.clone()
    _, el_ms, fa_ms = timed(Qp, torch.empty_like(Qp), profile=True)
    el_flops = sum(split_hex_flops(N_DEG) if int(t) == 0 else element_flops(int(t), N_DEG) for t in box.etype)
    el_bytes = sum(element_bytes(int(t), N_DEG) for t in box.etype)
    props = torch.cuda.get_device_properties(dev)
    clk = CLOCKS.summary(["split form"])
    peak = props.multi_processor_count * 2 * 2 * (clk.get("sm_max_mhz") or 2070.0) / 1e6
    tflops = el_flops * 5 * steps / (el_ms * 1e-3) / 1e12
    out["value"] = out["balanced"]["value"]
    out["balanced_over_naive"] = out["balanced"]["value"] / out["naive"]["value"]
    out["split_over_weak"] = out["balanced"]["value"] / weak_value if weak_value else None
    out["schedulers_bitwise_equal"] = bool(torch.equal(res["naive"], res["balanced"]))
    out["finite"] = bool(torch.isfinite(res["balanced"]).all())
    out["element_ms_per_step"] = el_ms / steps
    out["face_ms_per_step"] = fa_ms / steps
    out["roofline"] = {"bound": "alu", "kernel": "element kernel (balanced, fused), hexahedra in the split form",
                       "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                       "algorithmic_flops_per_stage": el_flops, "algorithmic_bytes_per_stage": el_bytes,
                       "hex_flops_split": split_hex_flops(N_DEG), "hex_flops_weak": element_flops(0, N_DEG),
                       "model": "alg_counts.json split_hex (every unordered node pair and every (face state, "
                                "node) pair of a line once, as the kernel evaluates them)"}
    ns, imb = mesh.cost_table()
    out["cost_table_ns_per_elem"] = dict(zip(("hex", "prism", "pyramid", "tet"), [round(x, 1) for x in ns]))
    out["sm_load_imbalance"] = imb
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

    def timed(Q, K, profile=False, nsteps=steps, warmup=args.warmup):
        b.set_profiling(profile)
        for _ in range(warmup):
            b.rk_step(Q, K, dt, 1)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        el = 0.0
        nl = 0
        with timed_window("batch"):
            e0.record(stream)
            for _ in range(nsteps):
                b.rk_step(Q, K, dt, 1)
                if profile:
                    pt = b.phase_times()
                    el += pt[0]
                    nl = pt[2]
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        b.set_profiling(False)
        return max_over_ranks(e0.elapsed_time(e1)), el, nl

    out = {"workload": BATCH_WORKLOAD, "instances": len(work), "elements": b.n_elems, "faces": b.n_faces,
           "dof_per_var": dof, "degrees": {str(k): Ns.count(k) for k in sorted(set(Ns))},
           "type_counts": dict(zip(("hex", "prism", "pyramid", "tet"), b.type_counts)), "steps": steps, "dt": dt}
    res = {}
    for sched in ("naive", "balanced"):
        b.set_scheduler(sched)
        warps, tms = b.autotune(Q0, dt)
        Q = Q0.clone()
        K = torch.empty_like(Q)
        ms, _, _ = timed(Q, K)
        res[sched] = Q
        out[sched] = {"value": ws * dof * 5 * steps / (ms * 1e-3), "ms_per_step": ms / steps, "warps": warps,
                      "autotune_ms_per_step": [round(x, 3) for x in tms.tolist()]}
        if sched == "balanced":
            names = ("hex", "prism", "pyramid", "tet")
            out[sched]["tile_shapes"] = {f"{names[t]}/N{N}": w for t, N, w in b.tile_shapes()}
    shapes = b.tile_shapes()

    def use(sched):
        def setup():
            b.set_scheduler(sched)
            if sched == "naive":
                b.set_element_warps(out["naive"]["warps"])
            else:
                for t, N, w in shapes:
                    b.set_table_warps(t, N, w)
        return setup
    rep_steps = max(2, steps // 2)
    Qr, Kr = Q0.clone(), torch.empty_like(Q0)

    def timed_rep():
        Qr.copy_(Q0)
        return timed(Qr, Kr, nsteps=rep_steps, warmup=1)[0] / rep_steps
    stats = interleaved_repeats([(sd, use(sd)) for sd in ("naive", "balanced")], timed_rep, args.sched_repeats)
    use("balanced")()
    out["scheduler_repeats"] = {"steps_per_repeat": rep_steps, "stats": stats,
                                "balanced_vs_naive": compare_to(stats, "balanced", "naive")}
    Qp = Q0.clone()
    _, el_ms, nl = timed(Qp, torch.empty_like(Qp), profile=True)
    # every element phase of the balanced scheduler is one launch per launch
    # group (tables sharing N and tile shape); a step has nl element phases
    # (the forward prime and one per stage) and 5 face launches
    out["launch_groups"] = len({(N, w) for _, N, w in shapes})
    out["element_launches_per_stage"] = out["launch_groups"]
    out["element_phases_per_step"] = nl
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
    ap.add_argument("--sched-repeats", type=int, default=10,
                    help="interleaved repeats per scheduler in the scheduler comparisons")
    ap.add_argument("--cpu-one-core-sample", type=int, default=256,
                    help="seeded sample of elements whose full LSERK steps the one-core oracle timing runs")
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
    ap.add_argument("--ke-adjoint-memory", type=float, default=0.95,
                    help="share of the free device memory the kinetic-energy adjoint may keep stage data in")
    ap.add_argument("--moving-steps", type=int, default=20,
                    help="LSERK steps of the moving-mesh leg (0: skip)")
    ap.add_argument("--moving-only", action="store_true",
                    help="profiling aid: the moving-mesh leg alone")
    ap.add_argument("--curved-steps", type=int, default=100,
                    help="steps of the curved-geometry leg (0 skips it)")
    ap.add_argument("--partition-steps", type=int, default=20,
                    help="steps of the partitioned leg (0 skips it)")
    ap.add_argument("--parts", type=int, default=2,
                    help="parts of the partitioned leg when one rank runs them all on its GPU")
    ap.add_argument("--split-steps", type=int, default=50,
                    help="steps of the split-form leg (0 skips it)")
    ap.add_argument("--split-only", action="store_true",
                    help="profiling aid: run the split-form leg only")
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
