"""Full-size parity of the configurations the benchmark times, on sampled
elements (the oracle evaluates only the sampled elements and what they read):

  * the 24^3 viscous TGV mesh (Navier-Stokes, Re 1600, N = 4);
  * the 64-instance serving batch (N from 2 to 5, sizes 4^3 to 20^3), three
    instances (the smallest, a middle one, the largest) checked;
  * the 12^3 Kuhn tetrahedral mesh at N = 3 and N = 5 (residual, and the
    adjoint of 20 steps with checkpoints every 5 against central differences;
    at N = 3 also the dot test against the oracle's complex-step derivative
    through the same 20 steps).

Each runs in the launch configuration of bench.py: balanced scheduler with
the autotuner's tile shapes.  The state is the TGV with the seeded smooth
perturbation at amplitude 0.1, and each variable's error is the plain
max|gpu - oracle| / max|oracle| over the sampled elements; bar 1e-11."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import FULL_SIZE_AMP, assert_sampled_parity, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def point_values(xyz, n_elems, N, fn):
    n = N + 1
    return fn(xyz).reshape(5, n_elems, n ** 3).transpose(1, 0, 2).reshape(-1)


def check_sample(o, Q, R, elems, volume_term, label=""):
    """Plain per-variable error on the sampled elements (the failure message
    also gives it against the volume-term magnitude)."""
    mask = np.zeros(len(Q), dtype=bool)
    for e in elems:
        mask[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = True

    def volume():
        vol = np.zeros(len(Q))
        for e in elems:
            vol[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = o.apply_minv(e, volume_term(e)).ravel()
        return vol
    assert_sampled_parity(R, o.rhs(Q, elems), var_index(o.mesh.nM), mask, volume=volume, label=label)


def test_ns_24cube_N4_sampled(dg):
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    box = di.box_mesh(24, "mixed", seed=4, p_prism=0.25, p_pyr=1.0 / 9.0)
    N, mu, Pr = 4, 1.0 / 1600, 0.72
    mesh = dg.Mesh(box, N)
    mesh.set_physics("navier_stokes", mu, Pr)
    vals = point_values(mesh.quad_points(), box.n_elems, N,
                        lambda x: di.perturbed_tgv_state(x, seed=8, amp=FULL_SIZE_AMP))
    Qs = mesh.project(torch.from_numpy(vals).cuda())
    mesh.autotune(Qs, 1e-4)
    R = mesh.get_state(mesh.rhs(Qs))
    Q = mesh.get_state(Qs)
    o = NSOracle(from_box(box, N), flux="lf", mu=mu, Pr=Pr)
    elems = np.sort(np.random.default_rng(4).choice(box.n_elems, 24, replace=False))
    G = o.lifted_gradient(Q, elems)
    check_sample(o, Q, R, elems, lambda e: o.ns_volume_term(Q, e, G))


def test_batch_64_instances_sampled(dg):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    work = di.batch_workload(64, seed=5)
    boxes = [di.box_mesh(m, "mixed", seed=sd) for m, N, sd in work]
    Ns = [N for m, N, sd in work]
    b = dg.Batch(boxes, Ns)
    xyz = b.quad_points()
    chunks, off = [], 0
    for box, N in zip(boxes, Ns):
        P = box.n_elems * (N + 1) ** 3
        chunks.append(point_values(xyz[off:off + P], box.n_elems, N,
                                   lambda x: di.perturbed_tgv_state(x, seed=3, amp=FULL_SIZE_AMP)))
        off += P
    Qs = b.project(torch.from_numpy(np.concatenate(chunks)).cuda())
    b.autotune(Qs, 1e-4)
    R = b.get_state(b.rhs(Qs))
    Q = b.get_state(Qs)
    sizes = [m for m, _, _ in work]
    picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    rng = np.random.default_rng(5)
    for i in picks:
        o = Oracle(from_box(boxes[i], Ns[i]), flux="lf")
        Qi, Ri = b.instance(Q, i), b.instance(R, i)
        elems = np.sort(rng.choice(boxes[i].n_elems, 12, replace=False))
        check_sample(o, Qi, Ri, elems, lambda e: o.volume_term(Qi, e))


@pytest.mark.parametrize("N", [3, 5])
def test_kuhn_12cube_sampled(dg, N):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = di.box_mesh(12, "kuhn", seed=3)
    mesh = dg.Mesh(box, N)
    vals = point_values(mesh.quad_points(), box.n_elems, N,
                        lambda x: di.perturbed_tgv_state(x, seed=3, amp=FULL_SIZE_AMP))
    Qs = mesh.project(torch.from_numpy(vals).cuda())
    mesh.autotune(Qs, 1e-4)
    R = mesh.get_state(mesh.rhs(Qs))
    Q = mesh.get_state(Qs)
    o = Oracle(from_box(box, N), flux="lf")
    elems = np.sort(np.random.default_rng(6).choice(box.n_elems, 24, replace=False))
    check_sample(o, Q, R, elems, lambda e: o.volume_term(Q, e))


@pytest.mark.parametrize("N", [3, 5])
def test_kuhn_12cube_adjoint_central_differences(dg, N):
    """<Q_K(Q0 + h v) - Q_K(Q0 - h v), w>/(2h) against <v, dg_rk_vjp(w)>
    through K = 20 steps, checkpoints every 5, at N = 3 and N = 5."""
    box = di.box_mesh(12, "kuhn", seed=3)
    mesh = dg.Mesh(box, N)
    vals = point_values(mesh.quad_points(), box.n_elems, N, lambda x: di.perturbed_tgv_state(x, seed=3))
    Q0 = mesh.project(torch.from_numpy(vals).cuda())
    Qh = mesh.get_state(Q0)
    nM = (N + 1) * (N + 2) * (N + 3) // 6
    scale = np.abs(Qh.reshape(-1, 5, nM)).max(axis=(0, 2))
    v = (di.random_vector(Qh.size, seed=41).reshape(-1, 5, nM) * scale[None, :, None]).reshape(-1)
    w = di.random_vector(Qh.size, seed=42)
    dt, K, h = 2e-4, 20, 1e-7

    def run(Q):
        Qs = mesh.set_state(Q)
        mesh.rk_step(Qs, mesh.empty(), dt, K)
        return mesh.get_state(Qs)

    fd = w @ (run(Qh + h * v) - run(Qh - h * v)) / (2 * h)
    ad = v @ mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w)))
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


def test_kuhn_12cube_dot_test_K20(dg):
    """<J v, w> = <v, J^T w> through K = 20 steps (checkpoints every 5) on the
    12^3 Kuhn tetrahedral mesh at N = 3: J^T w from dg_rk_vjp, J v from the
    oracle's complex-step derivative Im Q_K(Q_0 + i h v)/h (h = 1e-30, exact
    to rounding) through the same 20 steps, the oracle's residual spread over
    the host's cores; bar 1e-11 relative.  (A finite difference cannot reach
    this bar: the LF wave-speed maximum and |u.n| have kinks that a
    perturbation crosses.)"""
    from oracle_pool import PooledOracle
    N = 3
    box = di.box_mesh(12, "kuhn", seed=3)
    mesh = dg.Mesh(box, N)
    vals = point_values(mesh.quad_points(), box.n_elems, N, lambda x: di.perturbed_tgv_state(x, seed=3))
    Q0 = mesh.project(torch.from_numpy(vals).cuda())
    Qh = mesh.get_state(Q0)
    nM = (N + 1) * (N + 2) * (N + 3) // 6
    scale = np.abs(Qh.reshape(-1, 5, nM)).max(axis=(0, 2))
    v = (di.random_vector(Qh.size, seed=43).reshape(-1, 5, nM) * scale[None, :, None]).reshape(-1)
    w = di.random_vector(Qh.size, seed=44)
    dt, K, h = 2e-4, 20, 1e-30
    rhs = v @ mesh.get_state(mesh.rk_vjp(Q0, dt, K, 5, mesh.set_state(w)))
    mesh.sync()
    pool = PooledOracle(box, N, flux="lf")
    try:
        jv = pool.run(Qh + 1j * h * v, dt, K).imag / h
    finally:
        pool.close()
    lhs = w @ jv
    assert abs(lhs - rhs) < 1e-11 * abs(rhs), (lhs, rhs, abs(lhs - rhs) / abs(rhs))
