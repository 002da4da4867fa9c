"""GPU parity on curved meshes (vertex-interpolated element maps, pointwise J
in Eq. 1 and in the Algorithm 1 projection) against the curved oracle,
through the C ABI: dg_rhs, dg_rk_step, dg_project, dg_eval_nodal, the
quadrature points, free-stream preservation, scheduler and batch
equivalence, the affine limit, dg_rhs_vjp and dg_rk_vjp (oracle parity and
central differences), the Navier-Stokes residual, steps and adjoint (BR1 with
pointwise metric and normals, a 12^3 Re 1600 sampled check), and a
sampled check of the 16^3 mixed N = 4 perturbed mesh in the launch
configuration the benchmark times.  Tolerance: relative L-infinity per
variable <= 1e-11."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import FULL_SIZE_AMP, TOL, assert_sampled_parity, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def curved_box(kind, m, seed=1, reorder=None, amp=0.1):
    box = di.perturb_vertices(di.box_mesh(m, kind, seed=seed), amp)
    if reorder is not None:
        box = di.reorder_vertices(box, seed=reorder)
    return box


def check_sampled(o, Q, R, elems, volume_term, label):
    """Plain per-variable parity on the sampled elements (the failure message
    also gives the error against the volume-term magnitude)."""
    mask = np.zeros(len(Q), dtype=bool)
    for e in elems:
        mask[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = True

    def volume():
        vol = np.zeros(len(Q))
        for e in elems:
            vol[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = o.apply_minv(e, volume_term(e)).ravel()
        return vol
    assert_sampled_parity(R, o.rhs(Q, elems), var_index(o.mesh.nM), mask, volume=volume, label=label)


def setup(dg, kind, m, N, flux="lf", reorder=None, scheduler="balanced"):
    from oracle.curved import CurvedOracle, curved_from_box
    box = curved_box(kind, m, reorder=reorder)
    o = CurvedOracle(curved_from_box(box, N), flux=flux)
    mesh = dg.Mesh(box, N, flux=flux, scheduler=scheduler, geometry="vertex")
    return box, o, mesh


def state(o, seed=3, amp=0.05):
    return o.project(lambda x: di.perturbed_tgv_state(x, seed=seed, amp=amp))


CASES = [("mixed", 3, 3, "lf", None), ("mixed", 3, 3, "roe", 5), ("hex", 2, 4, "lf", 3),
         ("prism", 2, 5, "roe", 3), ("pyramid", 2, 2, "lf", 7), ("pyramid", 2, 1, "roe", None),
         ("mixed", 2, 6, "lf", 3), ("four", 4, 2, "lf", 5), ("kuhn", 2, 3, "roe", 7),
         ("mixed", 2, 1, "lf", None), ("prism", 2, 6, "lf", None)]


@pytest.mark.parametrize("kind,m,N,flux,reorder", CASES)
def test_curved_rhs_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    if kind != "kuhn":
        assert mesh.n_curved > 0
    Q = state(o)
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    err = rel_err(R, o.rhs(Q), var_index(o.mesh.nM))
    assert err < TOL, err


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("four", 4, 2), ("prism", 2, 4)])
def test_curved_project_eval_and_points(dg, kind, m, N):
    box, o, mesh = setup(dg, kind, m, N)
    n = N + 1
    xyz = mesh.quad_points()
    oq = np.concatenate([o.quad_points(e) for e in range(box.n_elems)])
    assert np.abs(xyz - oq).max() < 1e-13
    vals = di.tgv_state(xyz).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).reshape(-1)
    Q = mesh.get_state(mesh.project(torch.from_numpy(vals).cuda()))
    Qref = o.project(di.tgv_state)
    assert rel_err(Q, Qref, var_index(o.mesh.nM)) < TOL
    U = mesh.eval_nodal(mesh.set_state(torch.from_numpy(Qref).cuda())).cpu().numpy()
    Uref = np.concatenate([(o.mesh.block(Qref, e) @ o.ops[o.mesh.etype[e]].V.T).ravel()
                           for e in range(box.n_elems)])
    assert np.abs(U - Uref).max() < 1e-12 * np.abs(Uref).max()


def test_curved_load_vector(dg):
    box, o, mesh = setup(dg, "four", 4, 3)
    n = 4
    vals = di.tgv_state(mesh.quad_points()).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2)
    b = mesh.get_state(mesh.load_vector(torch.from_numpy(vals.reshape(-1).copy()).cuda()))
    ref = np.concatenate([((vals[e] * (o.ops[o.mesh.etype[e]].w * o.Jq[e])) @ o.ops[o.mesh.etype[e]].V).ravel()
                          for e in range(box.n_elems)])
    assert rel_err(b, ref, var_index(o.mesh.nM)) < TOL


@pytest.mark.parametrize("kind,m,N,flux,nsteps", [("mixed", 3, 3, "lf", 2), ("four", 4, 2, "roe", 1)])
def test_curved_rk_step_parity(dg, kind, m, N, flux, nsteps):
    box, o, mesh = setup(dg, kind, m, N, flux)
    Q = state(o)
    dt = 1e-3
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    mesh.rk_step(Qs, mesh.empty(), dt, nsteps)
    Qg = mesh.get_state(Qs)
    Qref = o.run(Q, dt, nsteps)
    assert rel_err(Qg - Q, Qref - Q, var_index(o.mesh.nM)) < 1e-10
    assert rel_err(Qg, Qref, var_index(o.mesh.nM)) < TOL
    mesh.sync()


@pytest.mark.parametrize("kind,m,N", [("mixed", 3, 3), ("four", 4, 2), ("pyramid", 2, 1)])
def test_curved_free_stream(dg, kind, m, N):
    box, o, mesh = setup(dg, kind, m, N)
    U0 = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    n = N + 1
    vals = np.tile(U0[None, :, None], (box.n_elems, 1, n ** 3)).reshape(-1)
    Qs = mesh.project(torch.from_numpy(vals).cuda())
    R = mesh.get_state(mesh.rhs(Qs))
    # flux scale: |F| ~ p + rho u^2 ~ 1; R = M^{-1}(vol - surf) ~ |F| / h
    assert np.abs(R).max() < 1e-12


@pytest.mark.parametrize("scheduler", ["naive", "static", "weighted"])
def test_curved_schedulers_agree(dg, scheduler):
    box, o, mesh = setup(dg, "mixed", 3, 3)
    other = dg.Mesh(box, 3, scheduler=scheduler, geometry="vertex")
    Q = torch.from_numpy(state(o)).cuda()
    R0 = mesh.get_state(mesh.rhs(mesh.set_state(Q)))
    R1 = other.get_state(other.rhs(other.set_state(Q)))
    np.testing.assert_array_equal(R0, R1)


def test_affine_mesh_same_with_curved_flag(dg):
    box = di.box_mesh(3, "mixed", seed=2)
    a = dg.Mesh(box, 3)
    b = dg.Mesh(box, 3, geometry="vertex")
    assert b.n_curved == 0 and b.geometry_doubles == 0
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    Q = torch.from_numpy(state(Oracle(from_box(box, 3)))).cuda()
    np.testing.assert_array_equal(a.get_state(a.rhs(a.set_state(Q))), b.get_state(b.rhs(b.set_state(Q))))


def test_curved_batch_equals_instances(dg):
    from oracle.curved import CurvedOracle, curved_from_box
    parts = [(curved_box("mixed", 3, seed=1), 3), (curved_box("four", 4, seed=2, reorder=4), 2),
             (di.box_mesh(2, "hex", seed=3), 4), (curved_box("prism", 2, seed=4), 5)]
    b = dg.Batch([p[0] for p in parts], [p[1] for p in parts], geometry="vertex")
    Qs, singles = [], []
    for i, (box, N) in enumerate(parts):
        o = CurvedOracle(curved_from_box(box, N))
        Qs.append(state(o, seed=10 + i))
        singles.append((dg.Mesh(box, N, geometry="vertex"), o))
    R = b.get_state(b.rhs(b.set_state(torch.from_numpy(np.concatenate(Qs)).cuda())))
    for i, (s, o) in enumerate(singles):
        Ri = s.get_state(s.rhs(s.set_state(torch.from_numpy(Qs[i]).cuda())))
        np.testing.assert_array_equal(b.instance(R, i), Ri)
        assert rel_err(Ri, o.rhs(Qs[i]), var_index(o.mesh.nM)) < TOL


@pytest.mark.parametrize("kind,m,N,flux,reorder", [("mixed", 2, 2, "lf", None), ("four", 4, 1, "lf", 5),
                                                    ("pyramid", 2, 3, "roe", 7), ("prism", 2, 4, "lf", 3),
                                                    ("hex", 2, 3, "roe", None)])
def test_curved_rhs_vjp_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q = state(o)
    w = di.random_vector(Q.size, seed=31)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    G = mesh.get_state(mesh.rhs_vjp(Qs, mesh.set_state(torch.from_numpy(w).cuda())))
    err = rel_err(G, o.rhs_vjp(Q, w), var_index(o.mesh.nM))
    assert err < TOL, err


def test_curved_rk_vjp_parity(dg):
    from oracle.adjoint import rk_vjp
    box, o, mesh = setup(dg, "mixed", 2, 2)
    Q = state(o)
    w = di.random_vector(Q.size, seed=32)
    dt, K = 1e-3, 3
    Q0 = mesh.set_state(torch.from_numpy(Q).cuda())
    for ckpt in (1, 2, 0):
        G = mesh.get_state(mesh.rk_vjp(Q0, dt, K, ckpt, mesh.set_state(torch.from_numpy(w).cuda())))
        err = rel_err(G, rk_vjp(o, Q, dt, K, w), var_index(o.mesh.nM))
        assert err < TOL, (ckpt, err)


def test_curved_rk_vjp_central_differences(dg):
    """<Q_K(Q0 + h v) - Q_K(Q0 - h v), w>/(2h) against <v, dg_rk_vjp(w)>
    through K = 10 steps on the curved 6^3 mixed mesh at N = 3."""
    box = curved_box("mixed", 6, seed=2)
    N = 3
    mesh = dg.Mesh(box, N, geometry="vertex")
    n = N + 1
    vals = di.perturbed_tgv_state(mesh.quad_points(), seed=3, amp=FULL_SIZE_AMP).reshape(5, box.n_elems, n ** 3)
    Q0 = mesh.project(torch.from_numpy(vals.transpose(1, 0, 2).reshape(-1)).cuda())
    Qh = mesh.get_state(Q0)
    nM = np.array([{0: 64, 1: 40, 2: 30}[int(t)] for t in box.etype])
    scale = np.zeros(Qh.size)
    for idx in var_index(nM):
        scale[idx] = np.abs(Qh[idx]).max()        # per-variable size of the state
    v = di.random_vector(Qh.size, seed=41) * scale
    w = di.random_vector(Qh.size, seed=42)
    dt, K, h = 5e-4, 10, 1e-7

    def run(Q):
        Qs = mesh.set_state(Q)
        mesh.rk_step(Qs, mesh.empty(), dt, K)
        return mesh.get_state(Qs)

    fd = w @ (run(Qh + h * v) - run(Qh - h * v)) / (2 * h)
    ad = v @ mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w)))
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


# ---------------------------------------------------------------- Navier-Stokes (BR1) on curved meshes
NS_CASES = [("mixed", 2, 2, "lf", None), ("four", 4, 2, "roe", 5), ("prism", 2, 3, "lf", 3),
            ("hex", 2, 4, "roe", None), ("pyramid", 2, 3, "lf", 7), ("mixed", 3, 3, "lf", None)]


def setup_ns(dg, kind, m, N, flux="lf", reorder=None, mu=0.05, Pr=0.72):
    from oracle.curved import CurvedNSOracle, curved_from_box
    box = curved_box(kind, m, reorder=reorder)
    o = CurvedNSOracle(curved_from_box(box, N), flux=flux, mu=mu, Pr=Pr)
    mesh = dg.Mesh(box, N, flux=flux, geometry="vertex")
    mesh.set_physics("navier_stokes", mu, Pr)
    return box, o, mesh


@pytest.mark.parametrize("kind,m,N,flux,reorder", NS_CASES)
def test_curved_ns_rhs_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup_ns(dg, kind, m, N, flux, reorder)
    Q = state(o)
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    err = rel_err(R, o.rhs(Q), var_index(o.mesh.nM))
    assert err < TOL, err


def test_curved_ns_rk_step_and_free_stream(dg):
    box, o, mesh = setup_ns(dg, "mixed", 2, 3)
    Q = state(o)
    dt = 1e-3
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    mesh.rk_step(Qs, mesh.empty(), dt, 2)
    Qg = mesh.get_state(Qs)
    Qref = o.run(Q, dt, 2)
    assert rel_err(Qg - Q, Qref - Q, var_index(o.mesh.nM)) < 1e-10
    n = 4
    U0 = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    vals = np.tile(U0[None, :, None], (box.n_elems, 1, n ** 3)).reshape(-1)
    R = mesh.get_state(mesh.rhs(mesh.project(torch.from_numpy(vals).cuda())))
    assert np.abs(R).max() < 1e-12
    mesh.sync()


@pytest.mark.parametrize("kind,m,N,flux,reorder", [("mixed", 2, 2, "lf", None), ("four", 4, 1, "roe", 5),
                                                    ("pyramid", 2, 2, "lf", 7), ("hex", 2, 3, "lf", 3)])
def test_curved_ns_rhs_vjp_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup_ns(dg, kind, m, N, flux, reorder)
    Q = state(o)
    w = di.random_vector(Q.size, seed=33)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    G = mesh.get_state(mesh.rhs_vjp(Qs, mesh.set_state(torch.from_numpy(w).cuda())))
    err = rel_err(G, o.rhs_vjp(Q, w), var_index(o.mesh.nM))
    assert err < TOL, err


def test_curved_ns_rk_vjp_parity(dg):
    from oracle.adjoint import rk_vjp
    box, o, mesh = setup_ns(dg, "mixed", 2, 2)
    Q = state(o)
    w = di.random_vector(Q.size, seed=34)
    dt, K = 1e-3, 2
    Q0 = mesh.set_state(torch.from_numpy(Q).cuda())
    for ckpt in (1, 2):
        G = mesh.get_state(mesh.rk_vjp(Q0, dt, K, ckpt, mesh.set_state(torch.from_numpy(w).cuda())))
        err = rel_err(G, rk_vjp(o, Q, dt, K, w), var_index(o.mesh.nM))
        assert err < TOL, (ckpt, err)


def test_curved_ns_12cube_N4_sampled(dg):
    """Viscous TGV at Re 1600 on the 12^3 mixed box with moved vertices, N = 4,
    autotuned balanced launches, TGV perturbed at amplitude 0.1: sampled
    elements against the oracle, plain per-variable metric at 1e-11."""
    from oracle.curved import CurvedNSOracle, curved_from_box
    box = di.perturb_vertices(di.box_mesh(12, "mixed", seed=4, p_prism=0.25, p_pyr=1.0 / 9.0), 0.1)
    N, mu, Pr = 4, 1.0 / 1600, 0.72
    mesh = dg.Mesh(box, N, geometry="vertex")
    mesh.set_physics("navier_stokes", mu, Pr)
    n = N + 1
    vals = di.perturbed_tgv_state(mesh.quad_points(), seed=8, amp=FULL_SIZE_AMP).reshape(5, box.n_elems, n ** 3)
    Qs = mesh.project(torch.from_numpy(vals.transpose(1, 0, 2).reshape(-1)).cuda())
    mesh.autotune(Qs, 1e-4)
    R = mesh.get_state(mesh.rhs(Qs))
    Q = mesh.get_state(Qs)
    o = CurvedNSOracle(curved_from_box(box, N), flux="lf", mu=mu, Pr=Pr)
    elems = np.sort(np.random.default_rng(9).choice(box.n_elems, 16, replace=False))
    G = o.lifted_gradient(Q, elems)
    check_sampled(o, Q, R, elems, lambda e: o.ns_volume_term(Q, e, G), "curved NS 12^3")


def test_curved_autograd(dg):
    """torch.autograd through the curved residual and K steps: gradients of a
    scalar loss equal dg_rhs_vjp / dg_rk_vjp of its seed."""
    from paper_2511_08020_gb300 import autograd as dga
    box, o, mesh = setup(dg, "mixed", 2, 3)
    Q0 = mesh.set_state(torch.from_numpy(state(o)).cuda())
    w = mesh.set_state(torch.from_numpy(di.random_vector(mesh.n_dof, seed=35)).cuda())
    Q = Q0.clone().requires_grad_(True)
    (dga.rhs(Q, mesh) * w).sum().backward()
    assert torch.equal(Q.grad, mesh.rhs_vjp(Q0, w))
    Q = Q0.clone().requires_grad_(True)
    (dga.rk(Q, mesh, 1e-3, 4, 2) * w).sum().backward()
    ref = mesh.rk_vjp(Q0, 1e-3, 4, 2, w)
    assert rel_err(Q.grad.cpu().numpy(), ref.cpu().numpy(), var_index(o.mesh.nM)) < TOL


def test_curved_ns_batch_equals_instances(dg):
    parts = [(curved_box("mixed", 2, seed=1), 2), (curved_box("four", 4, seed=2), 2), (curved_box("prism", 2, seed=3), 3)]
    b = dg.Batch([p[0] for p in parts], [p[1] for p in parts], geometry="vertex")
    b.set_physics("navier_stokes", 0.05, 0.72)
    from oracle.curved import CurvedOracle, curved_from_box
    Qs, singles = [], []
    for i, (box, N) in enumerate(parts):
        Qs.append(state(CurvedOracle(curved_from_box(box, N)), seed=20 + i))
        s = dg.Mesh(box, N, geometry="vertex")
        s.set_physics("navier_stokes", 0.05, 0.72)
        singles.append(s)
    R = b.get_state(b.rhs(b.set_state(torch.from_numpy(np.concatenate(Qs)).cuda())))
    for i, s in enumerate(singles):
        Ri = s.get_state(s.rhs(s.set_state(torch.from_numpy(Qs[i]).cuda())))
        np.testing.assert_array_equal(b.instance(R, i), Ri)


def test_curved_16cube_N4_sampled(dg):
    """The benchmark's curved workload (16^3 mixed, vertices moved by up to
    0.1 h per coordinate, N = 4) after autotuning: sampled elements against
    the oracle evaluated on those elements only, TGV perturbed at amplitude
    0.1, plain per-variable metric at 1e-11."""
    from oracle.curved import CurvedOracle, curved_from_box
    box = di.perturb_vertices(di.box_mesh(16, "mixed", seed=2), 0.1)
    N = 4
    mesh = dg.Mesh(box, N, geometry="vertex")
    n = N + 1
    vals = di.perturbed_tgv_state(mesh.quad_points(), seed=3, amp=FULL_SIZE_AMP).reshape(5, box.n_elems, n ** 3)
    Qs = mesh.project(torch.from_numpy(vals.transpose(1, 0, 2).reshape(-1)).cuda())
    mesh.autotune(Qs, 1e-4)
    R = mesh.get_state(mesh.rhs(Qs))
    Q = mesh.get_state(Qs)
    elems = np.sort(np.random.default_rng(7).choice(box.n_elems, 24, replace=False))
    o = CurvedOracle(curved_from_box(box, N))
    check_sampled(o, Q, R, elems, lambda e: o.volume_term(Q, e), "curved 16^3")
