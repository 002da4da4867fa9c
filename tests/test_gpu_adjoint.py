"""GPU parity of the adjoint entry points (no counterpart in the paper):
dg_rhs_vjp against the oracle's transposed residual, dot-product tests with
the oracle's exact (complex-step) JVP, dg_rk_vjp against the oracle's
reverse LSERK, checkpoint-interval invariance, and on the 12^3 Kuhn-tet
mesh (10,368 tets) through K = 20 steps with checkpoints every 5 steps,
central differences of the GPU forward map."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import TOL, make_box, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def setup(dg, kind, m, N, flux, reorder=None, seed=1):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = make_box(kind, m, seed=seed, reorder=reorder)
    return box, Oracle(from_box(box, N), flux=flux), dg.Mesh(box, N, flux=flux)


def state(o, seed=3, amp=0.05):
    return o.project(lambda x: di.perturbed_tgv_state(x, seed=seed, amp=amp))


CASES = [("mixed", 2, 3, "lf", 5), ("mixed", 2, 3, "roe", 5), ("kuhn", 2, 3, "lf", 7), ("kuhn", 2, 2, "roe", 7),
         ("hex", 2, 4, "lf", 3), ("mixed", 3, 2, "lf", None), ("prism", 2, 5, "roe", 2),
         ("mixed", 2, 6, "lf", 4),                                            # N = 6 = DG_MAX_N
         ("four", 4, 2, "roe", 6)]                                            # all four types


@pytest.mark.parametrize("kind,m,N,flux,reorder", CASES)
def test_rhs_vjp_parity(dg, kind, m, N, flux, reorder):
    from oracle.adjoint import rhs_vjp
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q = state(o)
    w = di.random_vector(Q.size, seed=11)
    Qs = mesh.set_state(Q)
    Ws = mesh.set_state(w)
    Qb = mesh.get_state(mesh.rhs_vjp(Qs, Ws))
    ref = rhs_vjp(o, Q, w)
    assert rel_err(Qb, ref, var_index(o.mesh.nM)) < TOL


@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_rhs_vjp_dot_product(dg, flux):
    """<J v, w> (oracle complex-step JVP) = <v, J^T w> (GPU VJP) to 1e-11."""
    from oracle.adjoint import rhs_jvp
    box, o, mesh = setup(dg, "mixed", 2, 3, flux, 4)
    Q = state(o)
    Qs = mesh.set_state(Q)
    for k in range(3):
        v = di.random_vector(Q.size, seed=20 + k)
        w = di.random_vector(Q.size, seed=30 + k)
        a = w @ rhs_jvp(o, Q, v)
        b = v @ mesh.get_state(mesh.rhs_vjp(Qs, mesh.set_state(w)))
        assert abs(a - b) < 1e-11 * abs(a)


@pytest.mark.parametrize("kind,m,N,flux,reorder,nsteps,ckpt", [("mixed", 2, 3, "lf", 5, 2, 1),
                                                                ("kuhn", 2, 2, "roe", 7, 3, 2),
                                                                ("mixed", 2, 2, "lf", None, 3, 5)])
def test_rk_vjp_parity(dg, kind, m, N, flux, reorder, nsteps, ckpt):
    from oracle.adjoint import rk_vjp
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q0 = state(o)
    w = di.random_vector(Q0.size, seed=13)
    dt = 2e-3
    Q0b = mesh.get_state(mesh.rk_vjp(mesh.set_state(Q0), dt, nsteps, ckpt, mesh.set_state(w)))
    ref = rk_vjp(o, Q0, dt, nsteps, w)
    assert rel_err(Q0b, ref, var_index(o.mesh.nM)) < TOL


@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_rk_vjp_stored_equals_recomputed(dg, flux):
    """dg_rk_vjp with the per-stage forward data kept (default), with every
    reverse stage recomputing it from the stage state, and with the compact
    store (a memory share too small for the trajectory: only the nodal state
    kept, the traces rebuilt per reverse stage): bitwise equal."""
    box, o, mesh = setup(dg, "mixed", 3, 3, flux, 6)
    Q0 = state(o)
    Qs = mesh.set_state(Q0)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=7))
    kept = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_storage(False)
    recomputed = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_storage(True)
    mesh.set_adjoint_memory(1e-9)
    compact = mesh.rk_vjp(Qs, 1e-3, 4, 2, Ws).clone()
    mesh.set_adjoint_memory(0.5)
    assert torch.equal(kept, recomputed)
    assert torch.equal(kept, compact)


@pytest.mark.parametrize("nsteps,ckpt", [(4, 2), (5, 2), (3, 5)])
def test_rk_checkpointed_split(dg, nsteps, ckpt):
    """dg_rk_step_checkpointed == dg_rk_step and dg_rk_vjp_checkpointed ==
    dg_rk_vjp, bitwise (including a shorter last segment)."""
    box, o, mesh = setup(dg, "mixed", 2, 3, "roe", 6)
    Q0 = state(o)
    Qa = mesh.set_state(Q0)
    Qb = Qa.clone()
    Q0s = Qa.clone()
    mesh.rk_step(Qa, mesh.empty(), 1e-3, nsteps)
    ck = mesh.rk_step_checkpointed(Qb, mesh.empty(), 1e-3, nsteps, ckpt)
    assert torch.equal(Qa, Qb)
    assert torch.equal(ck[0], Q0s)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=8))
    ref = mesh.rk_vjp(Q0s, 1e-3, nsteps, ckpt, Ws).clone()
    got = mesh.rk_vjp_checkpointed(ck, 1e-3, nsteps, ckpt, Ws)
    assert torch.equal(ref, got)


def test_rk_vjp_zero_steps_is_identity(dg):
    box, o, mesh = setup(dg, "mixed", 2, 2, "lf")
    Q0 = state(o)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=3))
    out = mesh.rk_vjp(mesh.set_state(Q0), 1e-3, 0, 1, Ws)
    assert torch.equal(out, Ws)


def test_rk_vjp_checkpoint_invariance(dg):
    box, o, mesh = setup(dg, "mixed", 3, 2, "lf", 8)
    Q0 = state(o)
    Qs = mesh.set_state(Q0)
    Ws = mesh.set_state(di.random_vector(Q0.size, seed=5))
    outs = [mesh.rk_vjp(Qs, 1e-3, 6, c, Ws).clone() for c in (1, 2, 4, 6, 0)]   # 0: automatic
    for x in outs[1:]:
        assert torch.equal(x, outs[0])


def test_tet_mesh_k20_central_differences(dg):
    """12^3 Kuhn tets, N = 3, perturbed TGV: <Q_K(Q0 + h v) - Q_K(Q0 - h v), w>/(2h)
    against <v, dg_rk_vjp(w)> through K = 20 LSERK steps, checkpoints every 5
    steps; the perturbation is scaled per variable and h is small enough not
    to cross the kinks of max and |.|."""
    box = make_box("kuhn", 12, seed=3)
    N = 3
    mesh = dg.Mesh(box, N, flux="lf")
    n = N + 1
    xyz = mesh.quad_points()
    vals = di.perturbed_tgv_state(xyz, seed=3).reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()
    Q0 = mesh.project(torch.from_numpy(vals).cuda())
    Qh = mesh.get_state(Q0)
    nM = (n * (n + 1) * (n + 2)) // 6
    scale = np.abs(Qh.reshape(-1, 5, nM)).max(axis=(0, 2))
    v = di.random_vector(Qh.size, seed=41).reshape(-1, 5, nM) * scale[None, :, None]
    v = v.ravel()
    w = di.random_vector(Qh.size, seed=42)
    dt, K = 2e-3, 20
    grad = mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w)))
    rhs = v @ grad
    h = 1e-6
    def run(x):
        Qs = mesh.set_state(x)
        mesh.rk_step(Qs, mesh.empty(), dt, K)
        return mesh.get_state(Qs)
    fd = w @ (run(Qh + h * v) - run(Qh - h * v)) / (2 * h)
    assert abs(fd - rhs) < 1e-6 * abs(rhs)
    # dot-product consistency of two cotangents (linearity of the VJP)
    w2 = di.random_vector(Qh.size, seed=43)
    g2 = mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w2)))
    g12 = mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w + w2)))
    assert np.abs(g12 - grad - g2).max() < 1e-11 * np.abs(g12).max()


def test_autograd_wrappers(dg):
    """torch.autograd: backward of DGRHS is dg_rhs_vjp, backward of DGRK is
    dg_rk_vjp; the gradient of a kinetic-energy-like functional agrees with
    central differences of the forward map."""
    from paper_2511_08020_gb300.autograd import rhs, rk
    box, o, mesh = setup(dg, "mixed", 2, 3, "lf", 5)
    Q0 = mesh.set_state(state(o))
    W = mesh.set_state(di.random_vector(mesh.n_dof, seed=3))
    x = Q0.clone().requires_grad_(True)
    (rhs(x, mesh) * W).sum().backward()
    assert torch.equal(x.grad, mesh.rhs_vjp(Q0, W))
    x = Q0.clone().requires_grad_(True)
    QK = rk(x, mesh, 2e-3, 3, 2)
    f = (QK * QK * W).sum()
    f.backward()
    # perturbation relative to each coefficient (no crossing of max / |.| kinks)
    v = torch.from_numpy(di.random_vector(mesh.n_dof, seed=8)).cuda() * Q0.abs()
    h = 1e-6
    def F(q):
        Q = q.clone()
        mesh.rk_step(Q, torch.empty_like(Q), 2e-3, 3)
        return (Q * Q * W).sum()
    fd = (F(Q0 + h * v) - F(Q0 - h * v)) / (2 * h)
    assert abs(float(fd) - float((x.grad * v).sum())) < 1e-6 * abs(float(fd))
