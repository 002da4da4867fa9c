"""GPU parity of the Navier-Stokes path (BR1 lifting, central viscous flux)
against the oracle's NSOracle, through the C ABI (dg_set_physics, dg_rhs,
dg_rk_step).  Tolerance: relative L-infinity per variable <= 1e-11.  The
viscosity of the parity cases (mu = 0.05 on boxes of 2-4 cubes) makes the
viscous terms a sizeable part of the residual; one case uses the Re = 1600
TGV value."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import FULL_SIZE_AMP, TOL, assert_sampled_parity, make_box, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU, PR = 0.05, 0.72


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def setup(dg, kind, m, N, flux="lf", reorder=None, seed=1, mu=MU, scheduler="balanced"):
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    box = make_box(kind, m, seed=seed, reorder=reorder)
    o = NSOracle(from_box(box, N), flux=flux, mu=mu, Pr=PR)
    mesh = dg.Mesh(box, N, flux=flux, scheduler=scheduler)
    mesh.set_physics("navier_stokes", mu, PR)
    return box, o, mesh


def state(o, seed=3, amp=0.05):
    return o.project(lambda x: di.perturbed_tgv_state(x, seed=seed, amp=amp))


CASES = [("mixed", 3, 3, "lf", None, MU), ("kuhn", 2, 3, "roe", 7, MU), ("mixed", 2, 4, "lf", 5, MU),
         ("hex", 2, 2, "roe", 3, MU), ("pyramid", 2, 3, "lf", None, MU), ("prism", 2, 5, "lf", 3, MU),
         ("kuhn", 2, 2, "lf", 11, MU), ("mixed", 3, 1, "roe", 2, MU), ("mixed", 3, 4, "lf", None, 1.0 / 1600),
         ("mixed", 2, 6, "lf", 4, MU),                                        # N = 6 = DG_MAX_N
         ("four", 4, 2, "roe", 3, MU)]                                        # all four types


@pytest.mark.parametrize("kind,m,N,flux,reorder,mu", CASES)
def test_ns_rhs_parity(dg, kind, m, N, flux, reorder, mu):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder, mu=mu)
    Q = state(o)
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    err = rel_err(R, o.rhs(Q), var_index(o.mesh.nM))
    assert err < TOL, err


def test_ns_viscous_part_parity(dg):
    """The viscous contribution alone (NS residual minus Euler residual) also
    matches: the 1e-11 bar is not met by the inviscid part only."""
    from oracle.dg import Oracle
    box, o, mesh = setup(dg, "mixed", 3, 3, "lf", None)
    Q = state(o)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    Rns = mesh.get_state(mesh.rhs(Qs))
    mesh.set_physics("euler")
    Reu = mesh.get_state(mesh.rhs(Qs))
    ref = o.rhs(Q) - Oracle(o.mesh, flux="lf").rhs(Q)
    err = rel_err(Rns - Reu, ref, var_index(o.mesh.nM))
    assert err < 1e-9, err                   # a difference of two residuals: cancellation
    vidx = var_index(o.mesh.nM)
    assert np.abs(ref[vidx[4]]).max() > 1e-3 * np.abs(o.rhs(Q)[vidx[4]]).max()


def test_ns_mu_zero_equals_euler(dg):
    box, o, mesh = setup(dg, "mixed", 3, 3, "roe", 5, mu=0.0)
    Q = state(o)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    Rns = mesh.get_state(mesh.rhs(Qs))
    mesh.set_physics("euler")
    Reu = mesh.get_state(mesh.rhs(Qs))
    # same arithmetic up to the compiler's choice of fused multiply-adds
    assert rel_err(Rns, Reu, var_index(o.mesh.nM)) < 1e-14


@pytest.mark.parametrize("kind,m,N,flux,reorder", [("mixed", 3, 3, "lf", None), ("kuhn", 2, 3, "roe", 7)])
def test_ns_rk_step_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q = state(o)
    dt, nsteps = 1e-3, 2
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    mesh.rk_step(Qs, mesh.empty(), dt, nsteps)
    Qg = mesh.get_state(Qs)
    Qref = o.run(Q, dt, nsteps)
    vidx = var_index(o.mesh.nM)
    assert rel_err(Qg - Q, Qref - Q, vidx) < 1e-10
    assert rel_err(Qg, Qref, vidx) < TOL
    mesh.sync()


def test_ns_schedulers_bitwise_equal(dg):
    box, o, mesh = setup(dg, "mixed", 4, 3, "lf", None)
    Q = state(o)
    out = {}
    for sched in ("balanced", "naive", "static", "weighted"):
        mesh.set_scheduler(sched)
        Qs = mesh.set_state(torch.from_numpy(Q).cuda())
        mesh.rk_step(Qs, mesh.empty(), 1e-3, 2)
        out[sched] = mesh.get_state(Qs)
    np.testing.assert_array_equal(out["balanced"], out["naive"])
    np.testing.assert_array_equal(out["balanced"], out["static"])
    np.testing.assert_array_equal(out["balanced"], out["weighted"])


def test_ns_free_stream(dg):
    box, o, mesh = setup(dg, "mixed", 3, 4, "roe", 5)
    U0 = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    Q = o.project(lambda x: np.tile(U0[:, None], (1, x.shape[0])))
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    assert np.abs(R).max() < 1e-12


def test_ns_batch_equals_instances(dg):
    parts = [("mixed", 3, 2, None), ("kuhn", 2, 3, 7), ("hex", 2, 4, None)]
    boxes, Qs = [], []
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    for i, (kind, m, N, reorder) in enumerate(parts):
        box = make_box(kind, m, seed=1 + i, reorder=reorder)
        boxes.append(box)
        Qs.append(Oracle(from_box(box, N)).project(lambda x, s=20 + i: di.perturbed_tgv_state(x, seed=s, amp=0.05)))
    b = dg.Batch(boxes, [p[2] for p in parts])
    b.set_physics("navier_stokes", MU, PR)
    R = b.get_state(b.rhs(b.set_state(torch.from_numpy(np.concatenate(Qs)).cuda())))
    for i, (box, p) in enumerate(zip(boxes, parts)):
        s = dg.Mesh(box, p[2])
        s.set_physics("navier_stokes", MU, PR)
        Ri = s.get_state(s.rhs(s.set_state(torch.from_numpy(Qs[i]).cuda())))
        np.testing.assert_array_equal(b.instance(R, i), Ri)


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("kind,m,N,flux,reorder", [("mixed", 2, 2, "lf", None), ("kuhn", 2, 2, "roe", 7),
                                                    ("mixed", 2, 3, "lf", 5), ("hex", 2, 1, "roe", 3),
                                                    ("prism", 2, 3, "lf", None), ("hex", 2, 6, "roe", 5),
                                                    ("four", 4, 1, "lf", 7)])
def test_ns_rhs_vjp_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q = state(o)
    w = di.random_vector(Q.size, seed=11)
    Qb = mesh.get_state(mesh.rhs_vjp(mesh.set_state(Q), mesh.set_state(w)))
    ref = o.rhs_vjp(Q, w)
    assert rel_err(Qb, ref, var_index(o.mesh.nM)) < TOL


def test_ns_rhs_vjp_dot_product(dg):
    """<J v, w> (oracle complex-step JVP through the NS residual) = <v, J^T w> (GPU)."""
    box, o, mesh = setup(dg, "mixed", 3, 3, "roe", 4)
    Q = state(o)
    Qs = mesh.set_state(Q)
    for k in range(3):
        v = di.random_vector(Q.size, seed=20 + k)
        w = di.random_vector(Q.size, seed=30 + k)
        jv = o.rhs(Q + 1e-30j * v).imag / 1e-30
        a = w @ jv
        b = v @ mesh.get_state(mesh.rhs_vjp(Qs, mesh.set_state(w)))
        assert abs(a - b) < 1e-11 * np.abs(w).sum() * np.abs(jv).max()


@pytest.mark.parametrize("kind,m,N,flux,reorder,nsteps,ckpt", [("mixed", 2, 2, "lf", 5, 2, 1),
                                                                ("kuhn", 2, 2, "roe", 7, 3, 2)])
def test_ns_rk_vjp_parity(dg, kind, m, N, flux, reorder, nsteps, ckpt):
    from oracle.adjoint import rk_vjp
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q0 = state(o)
    w = di.random_vector(Q0.size, seed=13)
    dt = 2e-3
    Q0b = mesh.get_state(mesh.rk_vjp(mesh.set_state(Q0), dt, nsteps, ckpt, mesh.set_state(w)))
    ref = rk_vjp(o, Q0, dt, nsteps, w)
    assert rel_err(Q0b, ref, var_index(o.mesh.nM)) < TOL


def test_ns_rk_vjp_checkpoint_invariance(dg):
    box, o, mesh = setup(dg, "mixed", 3, 2, "lf", 8)
    Q0 = state(o)
    Qs = mesh.set_state(Q0)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=5))
    outs = [mesh.rk_vjp(Qs, 1e-3, 4, c, Ws).clone() for c in (1, 2, 4)]
    for x in outs[1:]:
        assert torch.equal(x, outs[0])


def test_ns_rk_vjp_stored_equals_recomputed(dg):
    box, o, mesh = setup(dg, "mixed", 3, 3, "roe", 6)
    Q0 = state(o)
    Qs = mesh.set_state(Q0)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=7))
    kept = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_storage(False)
    recomputed = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_storage(True)
    # compact store: nodal state and gradient kept, traces and gradient
    # traces rebuilt per reverse stage
    mesh.set_adjoint_memory(1e-9)
    compact = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_memory(0.5)
    assert torch.equal(kept, recomputed)
    assert torch.equal(kept, compact)


def test_ns_rk_checkpointed_split(dg):
    box, o, mesh = setup(dg, "mixed", 2, 3, "lf", 6)
    Q0 = state(o)
    Q0s = mesh.set_state(Q0)
    Qb = Q0s.clone()
    ck = mesh.rk_step_checkpointed(Qb, mesh.empty(), 1e-3, 5, 2)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=8))
    ref = mesh.rk_vjp(Q0s, 1e-3, 5, 2, Ws).clone()
    assert torch.equal(ref, mesh.rk_vjp_checkpointed(ck, 1e-3, 5, 2, Ws))


def test_ns_noalloc_unsupported(dg):
    import ctypes
    box, o, mesh = setup(dg, "hex", 2, 2)
    Q = mesh.empty().fill_(1.0)
    st = dg.load().dg_rhs_vjp_noalloc(mesh.handle, dg._ptr(Q), dg._ptr(Q), dg._ptr(mesh.empty()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -7


def test_ns_kinetic_energy_adjoint_central_differences(dg):
    """Adjoint of the final kinetic energy through K = 20 Navier-Stokes steps
    (checkpoints every 5) on a 6^3 mixed box at N = 3, Re = 1600: the
    directional derivative <dE_k/dQ0, v> by dg_rk_vjp against central
    differences of E_k(Q_K(Q0 +- h v)).  E_k = sum over volume points of
    w J |m|^2 / (2 rho), evaluated from the states on the host."""
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    box = di.box_mesh(6, "mixed", seed=4, p_prism=0.25, p_pyr=1.0 / 9.0)
    N = 3
    o = NSOracle(from_box(box, N), flux="lf", mu=1.0 / 1600, Pr=PR)
    mesh = dg.Mesh(box, N)
    mesh.set_physics("navier_stokes", 1.0 / 1600, PR)
    Q0 = o.project(lambda x: di.perturbed_tgv_state(x, seed=9, amp=1e-2))
    dt, K = 2e-3, 20

    def ek_and_grad(Q):
        """E_k and dE_k/dQ (caller layout) by the oracle's quadrature."""
        val, grad = 0.0, np.zeros_like(Q)
        for e in range(o.mesh.n_elems):
            op = o.ops[o.mesh.etype[e]]
            U = o.mesh.block(Q, e) @ op.V.T
            wq = o.mesh.J[e] * op.w
            m2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
            val += np.sum(wq * 0.5 * m2 / U[0])
            dU = np.stack([-0.5 * m2 / U[0] ** 2, U[1] / U[0], U[2] / U[0], U[3] / U[0], 0 * U[0]]) * wq
            grad[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = (dU @ op.V).ravel()
        return val, grad

    def run(Q):
        Qs = mesh.set_state(Q)
        mesh.rk_step(Qs, mesh.empty(), dt, K)
        return mesh.get_state(Qs)

    _, gK = ek_and_grad(run(Q0))
    g0 = mesh.get_state(mesh.rk_vjp(mesh.set_state(Q0), dt, K, 5, mesh.set_state(gK)))
    # perturbation scaled per variable, small enough not to cross the kinks of max
    v = di.random_vector(Q0.size, seed=41)
    for idx in var_index(o.mesh.nM):
        v[idx] *= np.abs(Q0[idx]).max()
    h = 1e-7
    ep, _ = ek_and_grad(run(Q0 + h * v))
    em, _ = ek_and_grad(run(Q0 - h * v))
    fd = (ep - em) / (2 * h)
    ad = g0 @ v
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


def test_ns_sampled_12cube_N4(dg):
    """12^3 mixed box (the 40/30/30 recipe of the viscous TGV workload), N = 4,
    Re = 1600 viscosity, TGV perturbed at amplitude 0.1: sampled elements
    against the oracle, plain per-variable metric at 1e-11."""
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    box = di.box_mesh(12, "mixed", seed=4, p_prism=0.25, p_pyr=1.0 / 9.0)
    N = 4
    o = NSOracle(from_box(box, N), flux="lf", mu=1.0 / 1600, Pr=PR)
    mesh = dg.Mesh(box, N)
    mesh.set_physics("navier_stokes", 1.0 / 1600, PR)
    xyz = mesh.quad_points()
    n = N + 1
    vals = di.perturbed_tgv_state(xyz, seed=8, amp=FULL_SIZE_AMP)
    vals = vals.reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Qs = mesh.project(torch.from_numpy(vals).cuda())
    Q = mesh.get_state(Qs)
    R = mesh.get_state(mesh.rhs(Qs))
    rng = np.random.default_rng(1)
    elems = np.sort(rng.choice(box.n_elems, 24, replace=False))
    Rref = o.rhs(Q, elems)
    mask = np.zeros(len(Q), dtype=bool)
    for e in elems:
        mask[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = True
    G = o.lifted_gradient(Q, elems)

    def volume():
        vol = np.zeros(mesh.n_dof)
        for e in elems:
            vol[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = o.apply_minv(e, o.ns_volume_term(Q, e, G)).ravel()
        return vol
    assert_sampled_parity(R, Rref, var_index(o.mesh.nM), mask, volume=volume, label="NS 12^3")
