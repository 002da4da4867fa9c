"""GPU parity of the moving-mesh path (dg_mesh_create_moving) against the
moving-mesh oracle (oracle/moving.py): the moving-frame residual at several
mesh times on every element type at N = 1..5, LSERK steps with the discrete
geometric conservation law (the stage solves of Algorithm 1's projection
with the stage values of J), the free stream kept through steps on a mesh in
motion, conservation of int J q, zero velocity against the static curved
path, projection at the mesh time, an element turned inside out reported by
dg_sync, and the calls a moving mesh rejects.  N = 5 prisms (126 modes)
take the stage solve's widest configuration (four rows per lane)."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import FULL_SIZE_AMP, TOL, assert_sampled_parity, make_box, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONST = np.array([1.2, 0.3, -0.2, 0.1, 3.0])


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def setup(dg, kind, m, N, amp=0.3, seed=1, scheduler="balanced"):
    from oracle.moving import MovingOracle
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=seed), 0.1)
    vel = di.vertex_velocities(box.xyz, amp)
    mo = MovingOracle(box, N, vel)
    mesh = dg.MovingMesh(box, N, vel, scheduler=scheduler)
    return box, vel, mo, mesh


def tgv(mo):
    return mo.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1), 0.0)


CASES = [("hex", 2, 2), ("prism", 2, 3), ("pyramid", 2, 2), ("mixed", 2, 3), ("mixed", 3, 4), ("mixed", 2, 1),
         ("hex", 3, 4), ("prism", 2, 5), ("pyramid", 2, 5)]


@pytest.mark.parametrize("kind,m,N", CASES)
def test_moving_rhs_parity(dg, kind, m, N):
    box, vel, mo, mesh = setup(dg, kind, m, N)
    Q = tgv(mo)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    vidx = var_index(mo.mesh.nM)
    for t in (0.0, 0.05, -0.2):
        mesh.set_time(t)
        assert mesh.time == t
        R = mesh.get_state(mesh.rhs(Qs))
        err = rel_err(R, mo.rhs(Q, t), vidx)
        assert err < TOL, (t, err)
    mesh.sync()


@pytest.mark.parametrize("kind,m,N,sched", [("mixed", 2, 3, "balanced"), ("pyramid", 2, 2, "naive"),
                                            ("hex", 2, 2, "static"), ("prism", 2, 3, "balanced"),
                                            ("prism", 2, 5, "balanced")])
def test_moving_rk_step_parity(dg, kind, m, N, sched):
    box, vel, mo, mesh = setup(dg, kind, m, N, scheduler=sched)
    Q = tgv(mo)
    dt = 1e-3
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    mesh.rk_step(Qs, mesh.empty(), dt, 2)
    assert abs(mesh.time - 2 * dt) < 1e-15
    Qg = mesh.get_state(Qs)
    ref = mo.run(Q, 0.0, dt, 2)
    vidx = var_index(mo.mesh.nM)
    assert rel_err(Qg - Q, ref - Q, vidx) < 1e-10
    assert rel_err(Qg, ref, vidx) < TOL
    mesh.sync()


def test_moving_free_stream_and_conservation(dg):
    """A constant state stays constant to rounding through LSERK steps on a
    mesh in motion (the stage values of J in the stage solves); int J q is
    conserved."""
    box, vel, mo, mesh = setup(dg, "mixed", 3, 3, amp=0.5)
    Qc = mo.project(lambda x: np.repeat(CONST[:, None], len(x), axis=1), 0.0)
    Qs = mesh.set_state(torch.from_numpy(Qc).cuda())
    mesh.rk_step(Qs, mesh.empty(), 0.02, 3)
    Qg = mesh.get_state(Qs)
    assert np.abs(Qg - Qc).max() < 1e-12 * np.abs(Qc).max()
    mesh2 = dg.MovingMesh(box, 3, vel)
    Q = tgv(mo)
    Qs = mesh2.set_state(torch.from_numpy(Q).cuda())
    mesh2.rk_step(Qs, mesh2.empty(), 0.01, 3)
    before, after = mo.integral(Q, 0.0), mo.integral(mesh2.get_state(Qs), 0.03)
    assert np.abs(after - before).max() < 1e-13 * np.abs(before).max()
    mesh.sync()
    mesh2.sync()


def test_zero_velocity_equals_static_curved_path(dg):
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    N = 3
    static = dg.Mesh(box, N, geometry="vertex")
    moving = dg.MovingMesh(box, N, np.zeros_like(box.xyz))
    from oracle.curved import CurvedOracle, curved_from_box
    co = CurvedOracle(curved_from_box(box, N))
    Q = co.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    a = static.get_state(static.rhs(static.set_state(torch.from_numpy(Q).cuda())))
    b = moving.get_state(moving.rhs(moving.set_state(torch.from_numpy(Q).cuda())))
    vidx = var_index(co.mesh.nM)
    assert rel_err(b, a, vidx) < 1e-13
    Qa = static.set_state(torch.from_numpy(Q).cuda())
    Qb = moving.set_state(torch.from_numpy(Q).cuda())
    static.rk_step(Qa, static.empty(), 1e-3, 2)
    moving.rk_step(Qb, moving.empty(), 1e-3, 2)
    assert rel_err(moving.get_state(Qb), static.get_state(Qa), vidx) < 1e-13


def test_moving_projection_at_mesh_time(dg):
    """dg_project on a moving mesh solves with M(t) on the geometry of the
    mesh time: at t the projection of point values at the moved quadrature
    points equals the oracle's projection at t."""
    box, vel, mo, mesh = setup(dg, "mixed", 2, 3)
    t = 0.1
    mesh.set_time(t)
    n = mesh.N + 1
    o = mo.at(t)
    # the quadrature points of the mesh at time t, caller element order
    xyz = mesh.quad_points().reshape(box.n_elems, n ** 3, 3)
    from oracle.curved import shape_functions
    pts = np.empty_like(xyz)
    for e in range(box.n_elems):
        ref = mo.at(0.0).ops[o.mesh.etype[e]].pts
        Nv = shape_functions(o.mesh.etype[e], ref)
        np.testing.assert_allclose(Nv @ box.xyz[o.mesh.verts[e]], xyz[e], rtol=0, atol=1e-13)
        pts[e] = Nv @ (box.xyz[o.mesh.verts[e]] + t * vel[o.mesh.verts[e]])
    vals = np.stack([di.perturbed_tgv_state(pts[e], seed=3, amp=0.1) for e in range(box.n_elems)])
    Qs = mesh.project(torch.from_numpy(vals.copy()).cuda())
    got = mesh.get_state(Qs)
    ref = mo.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1), t)
    assert rel_err(got, ref, var_index(o.mesh.nM)) < 1e-12


def test_moving_benchmark_mesh_sampled(dg):
    """The bench's moving workload -- the curved 16^3 mixed box (vertices moved
    by up to 0.1 h, seed 11) with velocities 0.5 (sin y sin z, ...), N = 4,
    balanced scheduler, 4 warps per element -- at mesh time 0.02: the
    residual on 24 sampled elements (hexahedra among them) against the
    oracle with the plain per-variable metric, and the free stream through
    two LSERK steps of the whole mesh (the stage solves at full size)."""
    from oracle.moving import MovingOracle
    box = di.perturb_vertices(di.box_mesh(16, "mixed", seed=2), 0.1, seed=11)
    vel = di.vertex_velocities(box.xyz, 0.5)
    N, n = 4, 5
    mesh = dg.MovingMesh(box, N, vel)
    mesh.set_element_warps(4)
    vals = di.perturbed_tgv_state(mesh.quad_points(), seed=3, amp=FULL_SIZE_AMP)
    Qs = mesh.project(torch.from_numpy(vals.reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()).cuda())
    Q = mesh.get_state(Qs)
    mesh.set_time(0.02)
    R = mesh.get_state(mesh.rhs(Qs))
    mesh.sync()
    mo = MovingOracle(box, N, vel)
    rng = np.random.default_rng(21)
    hexes = np.where(box.etype == 0)[0]
    elems = np.unique(np.concatenate([rng.choice(hexes, 6, replace=False), rng.choice(box.n_elems, 18, replace=False)]))
    mask = np.zeros(len(Q), dtype=bool)
    for e in elems:
        mask[mo.mesh.dof_off[e]:mo.mesh.dof_off[e + 1]] = True
    assert_sampled_parity(R, mo.rhs(Q, 0.02, elems), var_index(mo.mesh.nM), mask, label="moving 16^3")
    # free stream at full size: a constant state through two steps in motion
    mesh.set_time(0.0)
    const = np.tile(CONST[None, :, None], (box.n_elems, 1, n ** 3))
    Qc = mesh.project(torch.from_numpy(const).cuda())
    Q0 = Qc.clone()
    mesh.rk_step(Qc, mesh.empty(), 0.01, 2)
    mesh.sync()
    assert float((Qc - Q0).abs().max()) < 1e-12 * float(Q0.abs().max())


NS_CASES = [("mixed", 2, 3), ("prism", 2, 3), ("pyramid", 2, 2), ("hex", 2, 3), ("mixed", 2, 1)]


@pytest.mark.parametrize("kind,m,N", NS_CASES)
def test_moving_navier_stokes_rhs_parity(dg, kind, m, N):
    """Navier-Stokes on a moving mesh (reading m7): the lifting on the geometry
    of the mesh time (prisms and pyramids solve M(t) for the lifted gradient
    between the two halves of the volume phase), the convective flux in the
    moving frame."""
    from oracle.moving import MovingOracle
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 0.3)
    mu = 0.05
    mo = MovingOracle(box, N, vel, mu=mu)
    mesh = dg.MovingMesh(box, N, vel)
    mesh.set_physics("navier_stokes", mu, 0.72)
    Q = tgv(mo)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    vidx = var_index(mo.mesh.nM)
    for t in (0.0, 0.05):
        mesh.set_time(t)
        err = rel_err(mesh.get_state(mesh.rhs(Qs)), mo.rhs(Q, t), vidx)
        assert err < TOL, (t, err)
    mesh.sync()


def test_moving_navier_stokes_steps_and_free_stream(dg):
    from oracle.moving import MovingOracle
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 0.3)
    N, mu, dt = 3, 0.05, 1e-3
    mo = MovingOracle(box, N, vel, mu=mu)
    mesh = dg.MovingMesh(box, N, vel)
    mesh.set_physics("navier_stokes", mu, 0.72)
    Q = tgv(mo)
    vidx = var_index(mo.mesh.nM)
    # dt = 1e-3: the lifting solves use the stage solves' factors and M Q is
    # carried between the steps; dt = 1e-2: the stage values miss the powers
    # of the stage times by more than the library allows, so every lifting
    # forms its own factor and every step its own M Q
    for dt in (dt, 1e-2):
        mesh.set_time(0.0)
        Qs = mesh.set_state(torch.from_numpy(Q).cuda())
        mesh.rk_step(Qs, mesh.empty(), dt, 2)
        Qg = mesh.get_state(Qs)
        ref = mo.run(Q, 0.0, dt, 2)
        assert rel_err(Qg - Q, ref - Q, vidx) < 1e-10
        assert rel_err(Qg, ref, vidx) < TOL
    mesh.set_time(0.0)
    Qc = mo.project(lambda x: np.repeat(CONST[:, None], len(x), axis=1), 0.0)
    Qcs = mesh.set_state(torch.from_numpy(Qc).cuda())
    mesh.rk_step(Qcs, mesh.empty(), 0.02, 2)
    assert np.abs(mesh.get_state(Qcs) - Qc).max() < 1e-12 * np.abs(Qc).max()
    mesh.sync()


def test_moving_navier_stokes_zero_velocity_equals_static_curved(dg):
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    N, mu = 3, 0.05
    static = dg.Mesh(box, N, geometry="vertex")
    static.set_physics("navier_stokes", mu, 0.72)
    moving = dg.MovingMesh(box, N, np.zeros_like(box.xyz))
    moving.set_physics("navier_stokes", mu, 0.72)
    from oracle.curved import CurvedOracle, curved_from_box
    co = CurvedOracle(curved_from_box(box, N))
    Q = co.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    a = static.get_state(static.rhs(static.set_state(torch.from_numpy(Q).cuda())))
    b = moving.get_state(moving.rhs(moving.set_state(torch.from_numpy(Q).cuda())))
    assert rel_err(b, a, var_index(co.mesh.nM)) < 1e-13


def test_inside_out_element_is_reported(dg):
    box = di.perturb_vertices(di.box_mesh(3, "hex", seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 1.0)
    mesh = dg.MovingMesh(box, 2, vel)
    Q = mesh.empty().fill_(0.0)
    mesh.set_time(2.0)
    mesh.rhs(Q)
    with pytest.raises(dg.DGError, match="inside out"):
        mesh.sync()
    mesh.set_time(0.0)
    mesh.sync()


def test_moving_mesh_rejections(dg):
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 0.2)
    mesh = dg.MovingMesh(box, 2, vel)
    Q = mesh.empty().fill_(1.0)
    for call in (lambda: mesh.rhs_vjp(Q, Q),
                 lambda: mesh.set_volume_form("split"), lambda: mesh.autotune(Q, 1e-3),
                 lambda: mesh.rk_vjp(Q, 1e-3, 1, 1, Q),
                 lambda: mesh.rk_step_checkpointed(Q, mesh.empty(), 1e-3, 2, 1)):
        with pytest.raises(dg.DGError):
            call()
    four = make_box("four", 4, seed=1)
    with pytest.raises(dg.DGError):
        dg.MovingMesh(four, 2, di.vertex_velocities(four.xyz, 0.1))
    with pytest.raises(dg.DGError):      # prisms of N = 6 have 196 modes: beyond the stage solve's 128
        dg.MovingMesh(box, 6, vel)
    with pytest.raises(dg.DGError):
        dg.MovingMesh(box, 2, vel * np.nan)
    static = dg.Mesh(box, 2, geometry="vertex")
    with pytest.raises(dg.DGError):
        dg._check(dg.load().dg_set_mesh_time(static.handle, 0.1))
    # the stage-by-stage entry points of partitioned solves: a moving mesh
    # steps through dg_rk_step only
    lib, K = dg.load(), mesh.empty()
    for call in (lambda: lib.dg_rk_prime(mesh.handle, dg._ptr(Q), dg._stream(None)),
                 lambda: lib.dg_rk_stage(mesh.handle, dg._ptr(Q), dg._ptr(K), 1e-3, 0, 0, dg._stream(None)),
                 lambda: lib.dg_rk_stage_lift(mesh.handle, dg._stream(None))):
        assert call() == -7      # DG_ERR_UNSUPPORTED
