"""CPU-only checks of the C-ABI library: it builds, loads, exports every entry
point include/dg.h declares, and its host-side set-up (reference tables, mesh
geometry, face matching, Hilbert ordering) agrees with the oracle's
independent set-up.  No compute call is made without a GPU."""
import os
import re

import numpy as np
import pytest

import dg_inputs as di

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:dg_status|const char\s*\*)\s*(dg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def dg():
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def test_library_exports_every_declared_symbol(dg):
    syms = declared_symbols()
    assert len(syms) >= 18
    lib = dg.load()
    for s in syms:
        assert hasattr(lib, s), s


@pytest.mark.parametrize("kind,m,N,reorder", [("mixed", 4, 3, False), ("kuhn", 2, 3, True),
                                              ("mixed", 3, 2, True), ("hex", 2, 5, True),
                                              ("pyramid", 2, 1, False), ("prism", 3, 4, True),
                                              ("four", 4, 3, True)])
def test_host_setup_matches_oracle(dg, kind, m, N, reorder):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = di.box_mesh(m, kind, seed=1)
    if reorder:
        box = di.reorder_vertices(box, seed=9)
    counts, qp, slots = dg.check_mesh(box, N)
    o = Oracle(from_box(box, N))
    assert counts[0] == box.n_elems
    assert counts[1] == len(o.mesh.faces)
    assert counts[2:6].tolist() == [int((box.etype == t).sum()) for t in range(4)]
    oq = np.concatenate([o.quad_points(e) for e in range(box.n_elems)])
    assert np.abs(qp - oq).max() < 1e-13
    assert sorted(slots.tolist()) == list(range(box.n_elems))


def test_four_type_mesh_recipe():
    """The 'four' recipe holds all four element types in one conforming mesh."""
    box = di.box_mesh(5, "four", seed=3)
    counts = box.type_counts()
    assert all(counts[t] > 0 for t in ("hex", "prism", "pyramid", "tet")), counts


def test_hilbert_order_is_local(dg):
    """Consecutive Hilbert slots are spatial neighbours far more often than in
    caller order (the locality the chunked scheduler relies on)."""
    box = di.box_mesh(8, "hex", seed=1)
    _, qp, slots = dg.check_mesh(box, 1)
    cent = qp.reshape(box.n_elems, 8, 3).mean(1)
    order = np.argsort(slots)
    d = np.linalg.norm(np.diff(cent[order], axis=0), axis=1)
    h = 2 * np.pi / 8
    assert np.mean(d < 1.01 * h) > 0.99


@pytest.mark.parametrize("bad", ["nonaffine", "unmatched", "type", "degree", "degree0", "empty", "vertex", "onecube"])
def test_bad_mesh_rejected(dg, bad):
    box = di.box_mesh(3, "hex", seed=1)
    N = 2
    if bad == "nonaffine":
        xyz = box.xyz.copy()
        xyz[box.verts_of(0)[7]] += 0.1
        box = di.BoxMesh(xyz, box.etype, box.elem_vert_off, box.elem_verts, box.period, 3, "hex", 1)
        status = -2
    elif bad == "unmatched":
        box = di.BoxMesh(box.xyz, box.etype[:-1], box.elem_vert_off[:-1], box.elem_verts[:box.elem_vert_off[-2]],
                         box.period, 3, "hex", 1)
        status = -2
    elif bad == "type":
        et = box.etype.copy()
        et[0] = 7
        box = di.BoxMesh(box.xyz, et, box.elem_vert_off, box.elem_verts, box.period, 3, "hex", 1)
        status = -1
    elif bad == "degree":
        N = 9
        status = -1
    elif bad == "degree0":
        N = 0
        status = -1
    elif bad == "empty":
        box = di.BoxMesh(box.xyz, box.etype[:0], box.elem_vert_off[:1], box.elem_verts[:0], box.period, 3, "hex", 1)
        status = -1
    elif bad == "onecube":
        # one cube per period: every face would be its own periodic image,
        # the owner rule has no neighbour to pick
        box = di.box_mesh(1, "hex", seed=1)
        status = -2
    else:
        ev = box.elem_verts.copy()
        ev[3] = len(box.xyz) + 5                     # vertex index out of range
        box = di.BoxMesh(box.xyz, box.etype, box.elem_vert_off, ev, box.period, 3, "hex", 1)
        status = -1
    with pytest.raises(dg.DGError) as ei:
        dg.check_mesh(box, N)
    assert ei.value.status == status


def test_no_cpu_fallback_without_gpu(dg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dg.DGError) as ei:
        dg.Mesh(di.box_mesh(2, "hex", seed=1), 2, stream=0)
    assert ei.value.status == -3


def test_batch_argument_checks_without_gpu(dg):
    """dg_batch_create validates its descriptions before touching a device:
    mixed flux is DG_ERR_ARG, an empty batch is DG_ERR_ARG, and a valid batch
    without a GPU is DG_ERR_CUDA (no CPU path)."""
    import ctypes
    torch = pytest.importorskip("torch")
    b0, b1 = di.box_mesh(2, "hex", seed=1), di.box_mesh(2, "kuhn", seed=2)
    d0, k0 = dg._desc(b0, 2, flux="lf")
    d1, k1 = dg._desc(b1, 3, flux="roe")
    h = ctypes.c_void_p()
    assert dg.load().dg_batch_create((dg.MeshDesc * 2)(d0, d1), 2, None, ctypes.byref(h)) == -1
    assert dg.load().dg_batch_create((dg.MeshDesc * 1)(d0), 0, None, ctypes.byref(h)) == -1
    if torch.cuda.is_available():
        return
    d1, k1 = dg._desc(b1, 3, flux="lf")
    with pytest.raises(dg.DGError) as ei:
        dg.Batch([b0, b1], [2, 3], stream=0)
    assert ei.value.status == -3


def test_moving_and_partition_argument_checks_without_gpu(dg):
    """The moving-mesh and stage-wise entry points validate their arguments
    before touching a device: a null or non-finite velocity field and null
    handles are DG_ERR_ARG, a moving mesh with the Roe flux is
    DG_ERR_UNSUPPORTED, and a valid moving mesh without a GPU is DG_ERR_CUDA
    (no CPU path)."""
    import ctypes
    import numpy as np
    torch = pytest.importorskip("torch")
    lib = dg.load()
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    d, keep = dg._desc(box, 2, flux="lf", geometry="vertex")
    h = ctypes.c_void_p()
    assert lib.dg_mesh_create_moving(ctypes.byref(d), None, None, ctypes.byref(h)) == -1
    bad = np.full_like(box.xyz, np.nan)
    assert lib.dg_mesh_create_moving(ctypes.byref(d), dg._ptr(bad), None, ctypes.byref(h)) == -1
    vel = np.ascontiguousarray(di.vertex_velocities(box.xyz, 0.1))
    droe, _ = dg._desc(box, 2, flux="roe", geometry="vertex")
    assert lib.dg_mesh_create_moving(ctypes.byref(droe), dg._ptr(vel), None, ctypes.byref(h)) == -7
    t = ctypes.c_double()
    assert lib.dg_mesh_time(None, ctypes.byref(t)) == -1
    assert lib.dg_set_mesh_time(None, 0.1) == -1
    assert lib.dg_rk_stage_lift(None, None) == -1
    assert lib.dg_halo_pack_gradients(None, None, None) == -1
    assert lib.dg_halo_unpack_gradients(None, None, None) == -1
    assert lib.dg_moving_phase_times(None, None, None) == -1
    ne, nf = ctypes.c_int64(), ctypes.c_int64()
    assert lib.dg_geometry_at(None, None, 0.0, ctypes.byref(ne), ctypes.byref(nf), None, None) == -1
    assert lib.dg_geometry_at(ctypes.byref(d), None, float("nan"), ctypes.byref(ne), ctypes.byref(nf), None, None) == -1
    if not torch.cuda.is_available():
        assert lib.dg_mesh_create_moving(ctypes.byref(d), dg._ptr(vel), None, ctypes.byref(h)) == -3


@pytest.mark.parametrize("kind,m,N,reorder", [("mixed", 3, 3, False), ("four", 4, 2, True), ("hex", 2, 4, True),
                                              ("pyramid", 2, 2, True), ("prism", 2, 3, False)])
def test_curved_host_setup_matches_oracle(dg, kind, m, N, reorder):
    """Curved (vertex-interpolated) element maps: the host's quadrature points
    equal the curved oracle's, and a perturbed mesh is rejected unless the
    curved geometry is requested."""
    from oracle.curved import CurvedOracle, curved_from_box
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=1), 0.1)
    if reorder:
        box = di.reorder_vertices(box, seed=9)
    with pytest.raises(dg.DGError) as ei:
        dg.check_mesh(box, N)
    assert ei.value.status == -2
    counts, qp, slots = dg.check_mesh(box, N, geometry="vertex")
    o = CurvedOracle(curved_from_box(box, N))
    assert counts[1] == len(o.mesh.faces)
    oq = np.concatenate([o.quad_points(e) for e in range(box.n_elems)])
    assert np.abs(qp - oq).max() < 1e-13
    assert sorted(slots.tolist()) == list(range(box.n_elems))


def test_curved_inverted_element_rejected(dg):
    """A vertex moved through the opposite face makes the trilinear map change
    orientation inside the element: DG_ERR_MESH."""
    box = di.box_mesh(3, "hex", seed=1)
    xyz = box.xyz.copy()
    v = box.verts_of(4)
    xyz[v[7]] = xyz[v[0]] - 0.3 * (xyz[v[7]] - xyz[v[0]])
    bad = di.BoxMesh(xyz, box.etype, box.elem_vert_off, box.elem_verts, box.period, 3, "hex", 1)
    with pytest.raises(dg.DGError) as ei:
        dg.check_mesh(bad, 2, geometry="vertex")
    assert ei.value.status == -2


def test_affine_mesh_is_unchanged_by_the_curved_flag(dg):
    box = di.box_mesh(3, "mixed", seed=2)
    c0, q0, s0 = dg.check_mesh(box, 3)
    c1, q1, s1 = dg.check_mesh(box, 3, geometry="vertex")
    assert np.array_equal(c0, c1) and np.array_equal(q0, q1) and np.array_equal(s0, s1)
