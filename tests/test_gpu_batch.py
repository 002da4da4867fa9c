"""GPU tests of multi-instance batching (dg_batch_create): several independent
periodic meshes with different element mixes and degrees N, advanced as one
handle.  No face couples two instances, so every instance's slice of a batch
result must equal, bit for bit, the same call on that instance alone (the
element and face arithmetic per element does not depend on which other
elements share the launch), and each slice must match the oracle on that
instance (relative L-infinity per variable <= 1e-11)."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import TOL, make_box, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (kind, m, N, vertex reordering seed)
INSTANCES = [("mixed", 3, 2, None), ("kuhn", 2, 3, 7), ("hex", 2, 4, None), ("mixed", 2, 1, 5),
             ("pyramid", 2, 3, None), ("prism", 2, 5, 3), ("mixed", 2, 6, 9)]


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def parts():
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    out = []
    for i, (kind, m, N, reorder) in enumerate(INSTANCES):
        box = make_box(kind, m, seed=1 + i, reorder=reorder)
        o = Oracle(from_box(box, N), flux="lf")
        Q = o.project(lambda x, s=10 + i: di.perturbed_tgv_state(x, seed=s, amp=0.05))
        out.append((box, N, o, Q))
    return out


def make_batch(dg, parts, flux="lf", scheduler="balanced"):
    return dg.Batch([p[0] for p in parts], [p[1] for p in parts], flux=flux, scheduler=scheduler)


def test_batch_layout(dg, parts):
    b = make_batch(dg, parts)
    assert b.n_instances == len(parts)
    singles = [dg.Mesh(p[0], p[1]) for p in parts]
    assert b.n_elems == sum(s.n_elems for s in singles)
    assert b.n_faces == sum(s.n_faces for s in singles)
    assert b.n_dof == sum(s.n_dof for s in singles)
    assert list(np.diff(b.elem_off)) == [s.n_elems for s in singles]
    assert list(np.diff(b.dof_off)) == [s.n_dof for s in singles]
    xyz = b.quad_points()
    off = 0
    for s in singles:
        q = s.quad_points()
        np.testing.assert_array_equal(xyz[off:off + len(q)], q)
        off += len(q)
    assert off == len(xyz)


@pytest.mark.parametrize("flux", ["lf", "roe"])
@pytest.mark.parametrize("scheduler", ["balanced", "naive", "static", "weighted"])
def test_batch_rhs_equals_instances(dg, parts, flux, scheduler):
    b = make_batch(dg, parts, flux=flux, scheduler=scheduler)
    Q = np.concatenate([p[3] for p in parts])
    R = b.get_state(b.rhs(b.set_state(torch.from_numpy(Q).cuda())))
    for i, p in enumerate(parts):
        s = dg.Mesh(p[0], p[1], flux=flux)
        Ri = s.get_state(s.rhs(s.set_state(torch.from_numpy(p[3]).cuda())))
        np.testing.assert_array_equal(b.instance(R, i), Ri)
    b.sync()


@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_batch_rhs_parity(dg, parts, flux):
    from oracle.dg import Oracle
    b = make_batch(dg, parts, flux=flux)
    Q = np.concatenate([p[3] for p in parts])
    R = b.get_state(b.rhs(b.set_state(torch.from_numpy(Q).cuda())))
    for i, (box, N, o, Qi) in enumerate(parts):
        oi = o if flux == "lf" else Oracle(o.mesh, flux=flux)
        err = rel_err(b.instance(R, i), oi.rhs(Qi), var_index(o.mesh.nM))
        assert err < TOL, (i, err)


def test_batch_rk_step(dg, parts):
    b = make_batch(dg, parts)
    Q = np.concatenate([p[3] for p in parts])
    dt, nsteps = 1e-3, 2
    Qs = b.set_state(torch.from_numpy(Q).cuda())
    K = b.empty()
    b.rk_step(Qs, K, dt, nsteps)
    Qb = b.get_state(Qs)
    for i, (box, N, o, Qi) in enumerate(parts):
        s = dg.Mesh(box, N)
        Qsi = s.set_state(torch.from_numpy(Qi).cuda())
        s.rk_step(Qsi, s.empty(), dt, nsteps)
        np.testing.assert_array_equal(b.instance(Qb, i), s.get_state(Qsi))
        if i < 3:
            Qref = o.run(Qi, dt, nsteps)
            assert rel_err(b.instance(Qb, i) - Qi, Qref - Qi, var_index(o.mesh.nM)) < 1e-10
    b.sync()


def test_batch_project(dg, parts):
    b = make_batch(dg, parts)
    xyz = b.quad_points()
    chunks, off = [], 0
    for i, (box, N, o, Qi) in enumerate(parts):
        P = box.n_elems * (N + 1) ** 3
        v = di.tgv_state(xyz[off:off + P]).reshape(5, box.n_elems, (N + 1) ** 3).transpose(1, 0, 2)
        chunks.append(v.reshape(-1))
        off += P
    Qb = b.get_state(b.project(torch.from_numpy(np.concatenate(chunks)).cuda()))
    for i, (box, N, o, Qi) in enumerate(parts):
        Qref = o.project(di.tgv_state)
        assert rel_err(b.instance(Qb, i), Qref, var_index(o.mesh.nM)) < TOL


def test_batch_rhs_vjp_equals_instances(dg, parts):
    b = make_batch(dg, parts)
    Q = np.concatenate([p[3] for p in parts])
    Rbar = di.random_vector(b.n_dof, seed=21)
    Qs = b.set_state(torch.from_numpy(Q).cuda())
    G = b.get_state(b.rhs_vjp(Qs, b.set_state(torch.from_numpy(Rbar).cuda())))
    for i, (box, N, o, Qi) in enumerate(parts):
        s = dg.Mesh(box, N)
        Gi = s.get_state(s.rhs_vjp(s.set_state(torch.from_numpy(Qi).cuda()),
                                   s.set_state(torch.from_numpy(b.instance(Rbar, i).copy()).cuda())))
        np.testing.assert_array_equal(b.instance(G, i), Gi)


def test_batch_rebalance_keeps_results(dg, parts):
    b = make_batch(dg, parts)
    Q = np.concatenate([p[3] for p in parts])
    Qs = b.set_state(torch.from_numpy(Q).cuda())
    R0 = b.get_state(b.rhs(Qs))
    b.set_profiling(True)
    b.rk_step(b.set_state(torch.from_numpy(Q).cuda()), b.empty(), 1e-4, 2)
    ns, imb = b.cost_table()
    assert all(ns[t] > 0 for t in range(4))      # every type appears in the batch
    assert b.rebalance(force=True)
    b.set_profiling(False)
    R1 = b.get_state(b.rhs(Qs))
    np.testing.assert_array_equal(R0, R1)


def test_batch_rejects_mixed_flux(dg, parts):
    import ctypes
    d0, k0 = dg._desc(parts[0][0], parts[0][1], flux="lf")
    d1, k1 = dg._desc(parts[1][0], parts[1][1], flux="roe")
    descs = (dg.MeshDesc * 2)(d0, d1)
    h = ctypes.c_void_p()
    assert dg.load().dg_batch_create(descs, 2, None, ctypes.byref(h)) == -1


def test_batch_per_table_tile_shapes(dg, parts):
    """Per-(type, N) tile shapes: tables sharing (N, warps) form one launch
    group each; results are bitwise independent of the shapes, and the
    autotuner's choice (per table or uniform) keeps them."""
    b = make_batch(dg, parts)
    Q = np.concatenate([p[3] for p in parts])
    Qs = b.set_state(torch.from_numpy(Q).cuda())
    R0 = b.get_state(b.rhs(Qs))
    shapes = b.tile_shapes()
    assert sorted((t, N) for t, N, _ in shapes) == sorted({(int(t), p[1]) for p in parts for t in set(p[0].etype)})
    for t, N, _ in shapes:
        b.set_table_warps(t, N, 1 if N <= 2 else (2 if N <= 4 else 4))
    assert {(t, N): w for t, N, w in b.tile_shapes()}[(shapes[0][0], shapes[0][1])] in (1, 2, 4)
    R1 = b.empty().fill_(float("nan"))                  # every element written by some group
    b.rhs(Qs, R1)
    assert bool(torch.isfinite(R1).all())
    np.testing.assert_array_equal(b.get_state(R1), R0)
    Q2a = Qs.clone()
    b.rk_step(Q2a, b.empty(), 1e-4, 1)
    warps, ms = b.autotune(Qs, 1e-4)
    assert 1 <= warps <= 4 and len(ms) == 5
    np.testing.assert_array_equal(b.get_state(b.rhs(Qs)), R0)
    Q2b = Qs.clone()
    b.rk_step(Q2b, b.empty(), 1e-4, 1)
    assert torch.equal(Q2a, Q2b)
    with pytest.raises(dg.DGError):
        b.set_table_warps(3, 6, 2)                  # no tet at N = 6 in this batch
