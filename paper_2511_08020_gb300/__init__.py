"""GB300 modal DG hot path: thin Python binding of libdg.so (include/dg.h).

Every function here only marshals arguments to the C ABI; all compute runs in
the library's CUDA kernels.  Importing the package loads the in-tree
libdg.so; if it is missing or cannot be loaded the import raises (there is
no CPU path).  Device buffers are torch tensors (float64, CUDA); torch is used
for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB, build as _build

__all__ = ["lib", "DGError", "Mesh", "Batch", "Part", "step_parts", "halo_plan", "check_mesh", "partition_plan", "FLUX", "SCHED",
           "PHYSICS", "GEOMETRY", "load"]

FLUX = {"lf": 0, "roe": 1, "ec": 2}
VOLUME = {"weak": 0, "split": 1}
SCHED = {"balanced": 0, "naive": 1, "static": 2, "weighted": 3}
PHYSICS = {"euler": 0, "navier_stokes": 1}
GEOMETRY = {"affine": 0, "vertex": 1}
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_MESH", -3: "DG_ERR_CUDA", -4: "DG_ERR_OOM",
          -5: "DG_ERR_TIMEOUT", -6: "DG_ERR_NONFINITE", -7: "DG_ERR_UNSUPPORTED"}


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("xyz", ctypes.c_void_p),
                ("n_elems", ctypes.c_int64), ("type", ctypes.c_void_p),
                ("elem_vert_off", ctypes.c_void_p), ("elem_verts", ctypes.c_void_p),
                ("period", ctypes.c_void_p), ("N", ctypes.c_int), ("flux", ctypes.c_int),
                ("gamma", ctypes.c_double), ("scheduler", ctypes.c_int),
                ("imbalance_threshold", ctypes.c_double), ("geometry", ctypes.c_int)]


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "dg_mesh_create": [ctypes.POINTER(MeshDesc), _P, ctypes.POINTER(_P)],
    "dg_batch_create": [ctypes.POINTER(MeshDesc), ctypes.c_int, _P, ctypes.POINTER(_P)],
    "dg_batch_layout": [_P, _P, _P],
    "dg_mesh_geometry": [_P, _P, _P, _P],
    "dg_mesh_destroy": [_P],
    "dg_mesh_check": [ctypes.POINTER(MeshDesc), _P, _P, _P],
    "dg_partition_plan": [ctypes.POINTER(MeshDesc), ctypes.c_int, _P, _P, _P, _P],
    "dg_mesh_layout": [_P, _P, _P, _P],
    "dg_set_state": [_P, _P, ctypes.c_int, _P, _P],
    "dg_get_state": [_P, _P, _P, ctypes.c_int, _P],
    "dg_quad_points": [_P, _P],
    "dg_project": [_P, _P, _P, _P],
    "dg_eval_nodal": [_P, _P, _P, _P],
    "dg_load_vector": [_P, _P, _P, _P],
    "dg_rhs": [_P, _P, _P, _P],
    "dg_rk_step": [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P],
    "dg_rhs_vjp": [_P, _P, _P, _P, _P],
    "dg_rk_vjp": [_P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P],
    "dg_rk_step_checkpointed": [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P],
    "dg_rk_vjp_checkpointed": [_P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P],
    "dg_set_scheduler": [_P, ctypes.c_int],
    "dg_set_physics": [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double],
    "dg_set_volume_form": [_P, ctypes.c_int],
    "dg_mesh_create_part": [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P],
    "dg_halo_plan": [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P],
    "dg_part_elements": [_P, _P, _P, _P],
    "dg_halo_counts": [_P, _P, _P, _P],
    "dg_halo_pack": [_P, _P, _P],
    "dg_halo_unpack": [_P, _P, _P],
    "dg_rk_prime": [_P, _P, _P],
    "dg_rk_stage": [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P],
    "dg_set_adjoint_memory": [_P, ctypes.c_double],
    "dg_set_table_warps": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "dg_tile_shapes": [_P, ctypes.c_int, _P, _P, _P, _P],
    "dg_set_adjoint_storage": [_P, ctypes.c_int],
    "dg_cost_table": [_P, _P, _P, _P],
    "dg_rebalance": [_P, ctypes.c_int, _P, _P],
    "dg_set_rebalance_interval": [_P, ctypes.c_int],
    "dg_rebalance_stats": [_P, _P, _P],
    "dg_graph_captures": [_P, _P],
    "dg_sync": [_P, _P],
    "dg_set_profiling": [_P, ctypes.c_int],
    "dg_set_stage_fusion": [_P, ctypes.c_int],
    "dg_set_element_warps": [_P, ctypes.c_int],
    "dg_autotune": [_P, _P, ctypes.c_double, _P, _P, _P],
    "dg_phase_times": [_P, _P, _P],
    "dg_mesh_create_moving": [ctypes.POINTER(MeshDesc), _P, _P, ctypes.POINTER(_P)],
    "dg_mesh_time": [_P, _P],
    "dg_set_mesh_time": [_P, ctypes.c_double],
    "dg_geometry_at": [ctypes.POINTER(MeshDesc), _P, ctypes.c_double, _P, _P, _P, _P],
    "dg_moving_phase_times": [_P, _P, _P],
    "dg_halo_pack_gradients": [_P, _P, _P],
    "dg_halo_unpack_gradients": [_P, _P, _P],
    "dg_rk_stage_lift": [_P, _P],
}

_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the in-tree libdg.so (building it first when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        if not build_if_missing:
            raise OSError(f"{LIB} is missing; run paper_2511_08020_gb300.build.build()")
        _build()
    lib = ctypes.CDLL(LIB)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.dg_last_error.argtypes = []
    lib.dg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def lib() -> ctypes.CDLL:
    return load()


def _check(status):
    if status != 0:
        raise DGError(status, load().dg_last_error().decode())


def _ptr(a):
    """Address of a numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _desc(box_or_arrays, N, flux="lf", gamma=1.4, scheduler="balanced", imbalance_threshold=0.1, geometry="affine"):
    import numpy as np
    b = box_or_arrays
    keep = dict(xyz=np.ascontiguousarray(b.xyz, dtype=np.float64),
                etype=np.ascontiguousarray(b.etype, dtype=np.int8),
                off=np.ascontiguousarray(b.elem_vert_off, dtype=np.int64),
                verts=np.ascontiguousarray(b.elem_verts, dtype=np.int64),
                period=np.ascontiguousarray(b.period, dtype=np.float64))
    d = MeshDesc(keep["xyz"].shape[0], keep["xyz"].ctypes.data, keep["etype"].shape[0], keep["etype"].ctypes.data,
                 keep["off"].ctypes.data, keep["verts"].ctypes.data, keep["period"].ctypes.data, int(N),
                 FLUX[flux] if isinstance(flux, str) else int(flux), float(gamma),
                 SCHED[scheduler] if isinstance(scheduler, str) else int(scheduler), float(imbalance_threshold),
                 GEOMETRY[geometry] if isinstance(geometry, str) else int(geometry))
    return d, keep


def check_mesh(box, N, geometry="affine"):
    """dg_mesh_check: host-only set-up; returns (counts[8], quad points [E*n^3, 3], slot_of_elem)."""
    import numpy as np
    d, keep = _desc(box, N, geometry=geometry)
    n = N + 1
    counts = np.zeros(8, dtype=np.int64)
    qp = np.zeros((len(keep["etype"]) * n ** 3, 3))
    slots = np.zeros(len(keep["etype"]), dtype=np.int64)
    _check(load().dg_mesh_check(ctypes.byref(d), _ptr(counts), _ptr(qp), _ptr(slots)))
    return counts, qp, slots


def halo_plan(box, N, part_of_elem, nparts, part, geometry="affine"):
    """dg_halo_plan (host-only): (send_faces [nparts], recv_faces [nparts],
    send_keys, recv_keys) of one part."""
    import numpy as np
    d, keep = _desc(box, N, geometry=geometry)
    poe = np.ascontiguousarray(part_of_elem, dtype=np.int64)
    sf, rf = np.zeros(nparts, dtype=np.int64), np.zeros(nparts, dtype=np.int64)
    _check(load().dg_halo_plan(ctypes.byref(d), _ptr(poe), int(nparts), int(part), _ptr(sf), _ptr(rf), None, None))
    sk, rk = np.zeros(max(1, int(sf.sum())), dtype=np.int64), np.zeros(max(1, int(rf.sum())), dtype=np.int64)
    _check(load().dg_halo_plan(ctypes.byref(d), _ptr(poe), int(nparts), int(part), _ptr(sf), _ptr(rf), _ptr(sk),
                               _ptr(rk)))
    return sf, rf, sk[:int(sf.sum())], rk[:int(rf.sum())]


def partition_plan(box, N, nparts, type_weight=None, geometry="affine"):
    """dg_partition_plan (host-only): (part_of_elem [E], halo_off [nparts+1], halo_elems)."""
    import numpy as np
    d, keep = _desc(box, N, geometry=geometry)
    E = len(keep["etype"])
    part = np.zeros(E, dtype=np.int64)
    off = np.zeros(nparts + 1, dtype=np.int64)
    tw = None if type_weight is None else np.ascontiguousarray(type_weight, dtype=np.float64)
    twp = ctypes.c_void_p(0) if tw is None else _ptr(tw)
    _check(load().dg_partition_plan(ctypes.byref(d), int(nparts), twp, _ptr(part), _ptr(off), ctypes.c_void_p(0)))
    halo = np.zeros(max(1, int(off[-1])), dtype=np.int64)
    _check(load().dg_partition_plan(ctypes.byref(d), int(nparts), twp, _ptr(part), _ptr(off), _ptr(halo)))
    return part, off, halo[:int(off[-1])]


class Mesh:
    """Owns a dg_mesh handle.  State tensors are float64 CUDA tensors of n_dof
    entries in the storage layout (see dg_set_state / dg_get_state)."""

    def __init__(self, box, N, flux="lf", gamma=1.4, scheduler="balanced", imbalance_threshold=0.1, stream=None,
                 geometry="affine"):
        """geometry: "affine" (every element an affine image of its reference
        element) or "vertex" (non-affine elements are curved, with
        vertex-interpolated maps; see dg_geometry in include/dg.h)."""
        import numpy as np
        self.N = int(N)
        self.flux = flux
        d, keep = _desc(box, N, flux, gamma, scheduler, imbalance_threshold, geometry)
        h = ctypes.c_void_p()
        _check(load().dg_mesh_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._adopt(h, keep["etype"].copy())
        self.points_per_elem = np.full(self.n_elems, (self.N + 1) ** 3, dtype=np.int64)

    def _adopt(self, h, etype):
        import numpy as np
        self.handle = h
        n_dof = ctypes.c_int64()
        self.slot_of_elem = np.zeros(len(etype), dtype=np.int64)
        counts = np.zeros(6, dtype=np.int64)
        _check(load().dg_mesh_layout(h, ctypes.byref(n_dof), _ptr(self.slot_of_elem), _ptr(counts)))
        self.n_dof = n_dof.value
        self.n_elems, self.n_faces = int(counts[0]), int(counts[1])
        self.type_counts = counts[2:].tolist()
        self.etype = etype
        nc, nf, gd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().dg_mesh_geometry(h, ctypes.byref(nc), ctypes.byref(nf), ctypes.byref(gd)))
        self.n_curved, self.n_curved_faces, self.geometry_doubles = nc.value, nf.value, gd.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(load().dg_mesh_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    def empty(self):
        import torch
        return torch.empty(self.n_dof, dtype=torch.float64, device="cuda")

    def set_state(self, Q_ext, Q_store=None, stream=None):
        """Q_ext: CUDA tensor or host (numpy / CPU tensor) in caller layout."""
        import numpy as np
        import torch
        if Q_store is None:
            Q_store = self.empty()
        if isinstance(Q_ext, torch.Tensor) and Q_ext.is_cuda:
            _check(load().dg_set_state(self.handle, _ptr(Q_ext), 1, _ptr(Q_store), _stream(stream)))
        else:
            a = Q_ext.numpy() if isinstance(Q_ext, torch.Tensor) else np.ascontiguousarray(Q_ext, dtype=np.float64)
            _check(load().dg_set_state(self.handle, _ptr(a), 0, _ptr(Q_store), _stream(stream)))
        return Q_store

    def get_state(self, Q_store, out=None, stream=None):
        """Caller-layout copy: into `out` (CUDA tensor or numpy array) or a new numpy array."""
        import numpy as np
        import torch
        if out is None:
            out = np.empty(self.n_dof)
        if isinstance(out, torch.Tensor) and out.is_cuda:
            _check(load().dg_get_state(self.handle, _ptr(Q_store), _ptr(out), 1, _stream(stream)))
        else:
            a = out.numpy() if isinstance(out, torch.Tensor) else out
            _check(load().dg_get_state(self.handle, _ptr(Q_store), _ptr(a), 0, _stream(stream)))
        return out

    def quad_points(self):
        import numpy as np
        xyz = np.zeros((int(self.points_per_elem.sum()), 3))
        _check(load().dg_quad_points(self.handle, _ptr(xyz)))
        return xyz

    def project(self, q_points, Q_store=None, stream=None):
        """Algorithm 1 projection of point values (CUDA tensor): per caller
        element its [5, n^3] block, elements concatenated ([n_elems, 5, n^3]
        for a single mesh)."""
        if Q_store is None:
            Q_store = self.empty()
        _check(load().dg_project(self.handle, _ptr(q_points), _ptr(Q_store), _stream(stream)))
        return Q_store

    def load_vector(self, q_points, b_store=None, stream=None):
        """dg_load_vector: b = V^T W J q (storage layout) for point values q (CUDA tensor)."""
        if b_store is None:
            b_store = self.empty()
        _check(load().dg_load_vector(self.handle, _ptr(q_points), _ptr(b_store), _stream(stream)))
        return b_store

    def eval_nodal(self, Q_store, out=None, stream=None):
        """dg_eval_nodal: U = V Q at the volume points, per caller element [5, n^3] (CUDA tensor)."""
        import torch
        if out is None:
            out = torch.empty(int(self.points_per_elem.sum()) * 5, dtype=torch.float64, device=Q_store.device)
        _check(load().dg_eval_nodal(self.handle, _ptr(Q_store), _ptr(out), _stream(stream)))
        return out

    # ---------------------------------------------------------------- hot path
    def rhs(self, Q_store, R_store=None, stream=None):
        if R_store is None:
            R_store = self.empty()
        _check(load().dg_rhs(self.handle, _ptr(Q_store), _ptr(R_store), _stream(stream)))
        return R_store

    def rk_step(self, Q_store, K_store, dt, nsteps=1, stream=None):
        _check(load().dg_rk_step(self.handle, _ptr(Q_store), _ptr(K_store), float(dt), int(nsteps), _stream(stream)))
        return Q_store

    def rhs_vjp(self, Q_store, Rbar, Qbar=None, stream=None):
        if Qbar is None:
            Qbar = self.empty()
        _check(load().dg_rhs_vjp(self.handle, _ptr(Q_store), _ptr(Rbar), _ptr(Qbar), _stream(stream)))
        return Qbar

    def rk_vjp(self, Q0_store, dt, nsteps, ckpt_every, QKbar, Q0bar=None, stream=None):
        if Q0bar is None:
            Q0bar = self.empty()
        _check(load().dg_rk_vjp(self.handle, _ptr(Q0_store), float(dt), int(nsteps), int(ckpt_every),
                                _ptr(QKbar), _ptr(Q0bar), _stream(stream)))
        return Q0bar

    def set_adjoint_storage(self, keep_stages=True):
        """dg_rk_vjp keeps per-stage forward data (True) or recomputes it (False)."""
        _check(load().dg_set_adjoint_storage(self.handle, int(bool(keep_stages))))

    # ---------------------------------------------------------------- physics
    def set_adjoint_memory(self, fraction=0.5):
        """Share of the free device memory dg_rk_vjp may keep stage data in."""
        _check(load().dg_set_adjoint_memory(self.handle, float(fraction)))

    def set_volume_form(self, form="weak"):
        """'weak' (Eq. 1) or 'split' (the entropy-stable split form on the hexahedra)."""
        _check(load().dg_set_volume_form(self.handle, VOLUME[form] if isinstance(form, str) else int(form)))

    def set_physics(self, physics="euler", mu=0.0, Pr=0.72):
        """'euler' or 'navier_stokes' (BR1 lifting, constant mu, Prandtl number Pr)."""
        _check(load().dg_set_physics(self.handle, PHYSICS[physics] if isinstance(physics, str) else int(physics),
                                     float(mu), float(Pr)))

    def rk_step_checkpointed(self, Q_store, K_store, dt, nsteps, ckpt_every, ckpt=None, stream=None):
        """dg_rk_step that also writes the segment-start checkpoints; returns them
        ([ceil(nsteps / ckpt_every), n_dof] CUDA tensor)."""
        import torch
        nseg = max(1, -(-int(nsteps) // max(1, min(int(ckpt_every), max(1, int(nsteps))))))
        if ckpt is None:
            ckpt = torch.empty((nseg, self.n_dof), dtype=torch.float64, device=Q_store.device)
        _check(load().dg_rk_step_checkpointed(self.handle, _ptr(Q_store), _ptr(K_store), float(dt), int(nsteps),
                                              int(ckpt_every), _ptr(ckpt), _stream(stream)))
        return ckpt

    def rk_vjp_checkpointed(self, ckpt, dt, nsteps, ckpt_every, QKbar, Q0bar=None, stream=None):
        if Q0bar is None:
            Q0bar = self.empty()
        _check(load().dg_rk_vjp_checkpointed(self.handle, _ptr(ckpt), float(dt), int(nsteps), int(ckpt_every),
                                             _ptr(QKbar), _ptr(Q0bar), _stream(stream)))
        return Q0bar

    # ---------------------------------------------------------------- scheduler
    def set_scheduler(self, kind):
        _check(load().dg_set_scheduler(self.handle, SCHED[kind] if isinstance(kind, str) else int(kind)))

    def cost_table(self, stream=None):
        import numpy as np
        ns = np.zeros(4)
        imb = ctypes.c_double()
        _check(load().dg_cost_table(self.handle, _ptr(ns), ctypes.byref(imb), _stream(stream)))
        return ns, imb.value

    def rebalance(self, force=False, stream=None):
        r = ctypes.c_int()
        _check(load().dg_rebalance(self.handle, int(bool(force)), ctypes.byref(r), _stream(stream)))
        return bool(r.value)

    def set_rebalance_interval(self, nsteps):
        """dg_set_rebalance_interval: check the imbalance every nsteps steps of rk_step (0: off)."""
        _check(load().dg_set_rebalance_interval(self.handle, int(nsteps)))

    def rebalance_stats(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(load().dg_rebalance_stats(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def graph_captures(self):
        """How many times dg_rk_step captured its graphs on this mesh."""
        n = ctypes.c_int64()
        _check(load().dg_graph_captures(self.handle, ctypes.byref(n)))
        return n.value

    def set_element_warps(self, warps):
        _check(load().dg_set_element_warps(self.handle, int(warps)))

    def autotune(self, Q_store, dt, stream=None):
        """Pick the fastest tile shapes; returns (uniform warps, ms per step [5]: the four
        uniform shapes and the per-table shapes, 0 when not tried)."""
        import numpy as np
        best = ctypes.c_int()
        ms = np.zeros(5)
        _check(load().dg_autotune(self.handle, _ptr(Q_store), float(dt), ctypes.byref(best), _ptr(ms), _stream(stream)))
        return best.value, ms

    def set_table_warps(self, etype, N, warps):
        _check(load().dg_set_table_warps(self.handle, int(etype), int(N), int(warps)))

    def tile_shapes(self):
        """[(type, N, warps)] of the tables present."""
        import numpy as np
        k = ctypes.c_int()
        _check(load().dg_tile_shapes(self.handle, 0, ctypes.byref(k), None, None, None))
        t, n, w = (np.zeros(max(1, k.value), dtype=np.int32) for _ in range(3))
        _check(load().dg_tile_shapes(self.handle, k.value, ctypes.byref(k), _ptr(t), _ptr(n), _ptr(w)))
        return [(int(a), int(b), int(c)) for a, b, c in zip(t[:k.value], n[:k.value], w[:k.value])]

    def set_stage_fusion(self, fused=True):
        _check(load().dg_set_stage_fusion(self.handle, int(bool(fused))))

    def set_profiling(self, on=True):
        _check(load().dg_set_profiling(self.handle, int(bool(on))))

    def phase_times(self, stream=None):
        """(element ms, face ms, element phases, face phases) of the last call."""
        import numpy as np
        out = np.zeros(4)
        _check(load().dg_phase_times(self.handle, _ptr(out), _stream(stream)))
        return float(out[0]), float(out[1]), int(out[2]), int(out[3])

    def sync(self, stream=None):
        _check(load().dg_sync(self.handle, _stream(stream)))


def geometry_at(box, N, velocity=None, t=0.0):
    """dg_geometry_at (host only): (element geometry, face geometry) of the box
    with every non-tetrahedral element on the curved path, static (velocity
    None) or of the moving mesh at time t."""
    import numpy as np
    d, keep = _desc(box, N, "lf", 1.4, "balanced", 0.1, "vertex")
    vel = None if velocity is None else np.ascontiguousarray(velocity, dtype=np.float64)
    ne, nf = ctypes.c_int64(), ctypes.c_int64()
    vp = None if vel is None else _ptr(vel)
    _check(load().dg_geometry_at(ctypes.byref(d), vp, float(t), ctypes.byref(ne), ctypes.byref(nf), None, None))
    eg, fg = np.zeros(ne.value), np.zeros(nf.value)
    _check(load().dg_geometry_at(ctypes.byref(d), vp, float(t), ctypes.byref(ne), ctypes.byref(nf), _ptr(eg), _ptr(fg)))
    return eg, fg


class MovingMesh(Mesh):
    """A mesh whose vertices move at constant velocities (dg_mesh_create_moving):
    vertex v sits at xyz[v] + t * velocity[v] at mesh time t (0 at creation).
    rhs evaluates at the mesh time; rk_step advances the state and the mesh
    time; project projects at the mesh time.  The Euler or (set_physics) the
    Navier-Stokes equations with the LF flux on hexahedra, prisms and
    pyramids."""

    def __init__(self, box, N, velocity, gamma=1.4, scheduler="balanced", imbalance_threshold=0.1, stream=None):
        import numpy as np
        self.N = int(N)
        self.flux = "lf"
        d, keep = _desc(box, N, "lf", gamma, scheduler, imbalance_threshold, "vertex")
        vel = np.ascontiguousarray(velocity, dtype=np.float64)
        if vel.shape != keep["xyz"].shape:
            raise ValueError("velocity must have the shape of the vertex coordinates")
        h = ctypes.c_void_p()
        _check(load().dg_mesh_create_moving(ctypes.byref(d), _ptr(vel), _stream(stream), ctypes.byref(h)))
        self._adopt(h, keep["etype"].copy())
        self.points_per_elem = np.full(self.n_elems, (self.N + 1) ** 3, dtype=np.int64)

    @property
    def time(self):
        t = ctypes.c_double()
        _check(load().dg_mesh_time(self.handle, ctypes.byref(t)))
        return t.value

    def set_time(self, t):
        _check(load().dg_set_mesh_time(self.handle, float(t)))

    def moving_phase_times(self, stream=None):
        """(geometry ms, mass-matrix ms, geometry launches, mass launches) of
        the last call (profiling on)."""
        import numpy as np
        out = np.zeros(4)
        _check(load().dg_moving_phase_times(self.handle, _ptr(out), _stream(stream)))
        return float(out[0]), float(out[1]), int(out[2]), int(out[3])


class Part(Mesh):
    """One part of a partitioned mesh (dg_mesh_create_part): the elements of
    `part` under part_of_elem plus their ghosts, in ascending global caller
    index (global_of_local); steps with rk_prime / rk_stage and the halo
    exchange (halo_pack / halo_unpack)."""

    def __init__(self, box, N, part_of_elem, nparts, part, flux="lf", gamma=1.4, scheduler="balanced",
                 stream=None, geometry="affine"):
        import numpy as np
        self.N = int(N)
        self.flux = flux
        self.nparts, self.part = int(nparts), int(part)
        d, keep = _desc(box, N, flux, gamma, scheduler, 0.1, geometry)
        poe = np.ascontiguousarray(part_of_elem, dtype=np.int64)
        h = ctypes.c_void_p()
        _check(load().dg_mesh_create_part(ctypes.byref(d), _ptr(poe), self.nparts, self.part, _stream(stream),
                                          ctypes.byref(h)))
        n = ctypes.c_int64()
        _check(load().dg_part_elements(h, ctypes.byref(n), None, None))
        self.global_of_local = np.zeros(n.value, dtype=np.int64)
        self.is_ghost = np.zeros(n.value, dtype=np.int8)
        _check(load().dg_part_elements(h, ctypes.byref(n), _ptr(self.global_of_local), _ptr(self.is_ghost)))
        self._adopt(h, keep["etype"][self.global_of_local].copy())
        self.points_per_elem = np.full(self.n_elems, (self.N + 1) ** 3, dtype=np.int64)
        self.send_faces = np.zeros(self.nparts, dtype=np.int64)
        self.recv_faces = np.zeros(self.nparts, dtype=np.int64)
        per = ctypes.c_int64()
        _check(load().dg_halo_counts(h, _ptr(self.send_faces), _ptr(self.recv_faces), ctypes.byref(per)))
        self.doubles_per_face = per.value

    def halo_buffers(self):
        """Device send and receive buffers of the halo exchange."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        return (torch.empty(max(1, int(self.send_faces.sum())) * self.doubles_per_face, dtype=torch.float64, device=dev),
                torch.empty(max(1, int(self.recv_faces.sum())) * self.doubles_per_face, dtype=torch.float64, device=dev))

    def halo_pack(self, send, stream=None):
        _check(load().dg_halo_pack(self.handle, _ptr(send), _stream(stream)))

    def halo_unpack(self, recv, stream=None):
        _check(load().dg_halo_unpack(self.handle, _ptr(recv), _stream(stream)))

    def halo_gradient_buffers(self):
        """Send and receive buffers of the Navier-Stokes gradient-trace
        exchange (three times the trace blocks)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        per = 3 * self.doubles_per_face
        return (torch.empty(max(1, int(self.send_faces.sum())) * per, dtype=torch.float64, device=dev),
                torch.empty(max(1, int(self.recv_faces.sum())) * per, dtype=torch.float64, device=dev))

    def halo_pack_gradients(self, send, stream=None):
        _check(load().dg_halo_pack_gradients(self.handle, _ptr(send), _stream(stream)))

    def halo_unpack_gradients(self, recv, stream=None):
        _check(load().dg_halo_unpack_gradients(self.handle, _ptr(recv), _stream(stream)))

    def rk_stage_lift(self, stream=None):
        _check(load().dg_rk_stage_lift(self.handle, _stream(stream)))

    def rk_prime(self, Q_store, stream=None):
        _check(load().dg_rk_prime(self.handle, _ptr(Q_store), _stream(stream)))

    def rk_stage(self, Q_store, K_store, dt, stage, last, stream=None):
        _check(load().dg_rk_stage(self.handle, _ptr(Q_store), _ptr(K_store), float(dt), int(stage), int(bool(last)),
                                  _stream(stream)))


def step_parts(parts, Qs, Ks, dt, nsteps, exchange, exchange_gradients=None):
    """nsteps LSERK steps of a partitioned mesh: parts[i] advances Qs[i]
    (storage layout) with register Ks[i]; exchange() moves every part's packed
    halo blocks into its peers' receive buffers between the forward phase and
    the face phase of every stage.  Navier-Stokes parts need the second
    exchange, exchange_gradients(), of the gradient traces between the
    lifting half of the stage (rk_stage_lift) and the flux half (rk_stage)."""
    for step in range(nsteps):
        if step == 0:
            for P, Q in zip(parts, Qs):
                P.rk_prime(Q)
        for s in range(5):
            exchange()
            if exchange_gradients is not None:
                for P in parts:
                    P.rk_stage_lift()
                exchange_gradients()
            for P, Q, K in zip(parts, Qs, Ks):
                P.rk_stage(Q, K, dt, s, last=(s == 4 and step == nsteps - 1))


class Batch(Mesh):
    """Several independent periodic meshes, each with its own degree N,
    advanced as one (dg_batch_create).  States, residuals and point values are
    the instances' own layouts concatenated in instance order:
    instance i owns caller elements elem_off[i]:elem_off[i+1] and state
    entries dof_off[i]:dof_off[i+1] (in both the caller and the storage
    layout).  All instances share flux and gamma."""

    def __init__(self, boxes, Ns, flux="lf", gamma=1.4, scheduler="balanced", imbalance_threshold=0.1, stream=None,
                 geometry="affine"):
        import numpy as np
        if len(boxes) != len(Ns) or not boxes:
            raise ValueError("one N per mesh, at least one mesh")
        k = len(boxes)
        descs = (MeshDesc * k)()
        self._keep = []
        for i, (b, N) in enumerate(zip(boxes, Ns)):
            d, keep = _desc(b, N, flux, gamma, scheduler, imbalance_threshold, geometry)
            descs[i] = d
            self._keep.append(keep)
        self.Ns = [int(N) for N in Ns]
        self.N = max(self.Ns)
        self.flux = flux
        h = ctypes.c_void_p()
        _check(load().dg_batch_create(descs, k, _stream(stream), ctypes.byref(h)))
        self._adopt(h, np.concatenate([kp["etype"] for kp in self._keep]))
        self.elem_off = np.zeros(k + 1, dtype=np.int64)
        self.dof_off = np.zeros(k + 1, dtype=np.int64)
        _check(load().dg_batch_layout(h, _ptr(self.elem_off), _ptr(self.dof_off)))
        self.points_per_elem = np.concatenate(
            [np.full(len(kp["etype"]), (N + 1) ** 3, dtype=np.int64) for kp, N in zip(self._keep, self.Ns)])
        self._keep = None

    @property
    def n_instances(self):
        return len(self.Ns)

    def instance(self, x, i):
        """Entries of instance i in a batch state (caller or storage layout)."""
        return x[int(self.dof_off[i]):int(self.dof_off[i + 1])]
