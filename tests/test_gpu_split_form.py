"""GPU parity of the entropy-stable split form on hexahedra (dg_set_volume_form)
against the split-form oracle (oracle/split_form.py): residuals on small
meshes of every kind at N = 1..5 with the LF, Roe and entropy-conservative
surface fluxes, LSERK steps, entropy conservation of the GPU residual with the
entropy-conservative flux, free stream, scheduler independence, the benchmark
mesh on sampled elements, and the combinations the library rejects."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import FULL_SIZE_AMP, TOL, assert_sampled_parity, make_box, rel_err, var_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def setup(dg, kind, m, N, flux="lf", reorder=None, scheduler="balanced"):
    from oracle.mesh import from_box
    from oracle.split_form import SplitFormOracle
    box = make_box(kind, m, seed=1, reorder=reorder)
    o = SplitFormOracle(from_box(box, N), flux=flux)
    mesh = dg.Mesh(box, N, flux=flux, scheduler=scheduler)
    mesh.set_volume_form("split")
    return box, o, mesh


def state(o, seed=3, amp=0.1):
    from oracle.dg import Oracle
    return Oracle(o.mesh).project(lambda x: di.perturbed_tgv_state(x, seed=seed, amp=amp))


CASES = [("hex", 2, 2, "lf", None), ("hex", 3, 3, "ec", 4), ("hex", 2, 4, "roe", 3), ("hex", 2, 1, "lf", 2),
         ("hex", 2, 5, "ec", None), ("mixed", 3, 3, "lf", None), ("mixed", 2, 4, "roe", 5),
         ("four", 4, 2, "lf", None), ("mixed", 3, 2, "ec", 6)]


@pytest.mark.parametrize("kind,m,N,flux,reorder", CASES)
def test_split_rhs_parity(dg, kind, m, N, flux, reorder):
    box, o, mesh = setup(dg, kind, m, N, flux, reorder)
    Q = state(o)
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    err = rel_err(R, o.rhs(Q), var_index(o.mesh.nM))
    assert err < TOL, err


def test_split_rk_step_parity(dg):
    box, o, mesh = setup(dg, "mixed", 2, 3, "lf", 5)
    Q = state(o)
    Qs = mesh.set_state(torch.from_numpy(Q).cuda())
    mesh.rk_step(Qs, mesh.empty(), 1e-3, 2)
    Qg = mesh.get_state(Qs)
    ref = o.run(Q, 1e-3, 2)
    vidx = var_index(o.mesh.nM)
    assert rel_err(Qg - Q, ref - Q, vidx) < 1e-10
    assert rel_err(Qg, ref, vidx) < TOL
    mesh.sync()


def test_gpu_residual_conserves_entropy_with_the_ec_flux(dg):
    """sum_e sum_q w_q J v(U_q) . R_q of the GPU residual vanishes to rounding
    on a periodic all-hexahedral mesh with the entropy-conservative surface
    flux and is negative with LF."""
    for flux, conserving in (("ec", True), ("lf", False)):
        box, o, mesh = setup(dg, "hex", 3, 3, flux, 2)
        Q = state(o, amp=0.2)
        R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
        rate, scale = o.entropy_rate(Q, R)
        if conserving:
            assert abs(rate) < 1e-12 * scale, (rate, scale)
        else:
            assert rate < -1e-6 * scale, (rate, scale)


def test_split_free_stream_and_conservation(dg):
    box, o, mesh = setup(dg, "four", 4, 3, "lf", None)
    from oracle.dg import Oracle
    const = np.array([1.2, 0.3, -0.2, 0.1, 3.0])
    Qc = Oracle(o.mesh).project(lambda x: np.repeat(const[:, None], len(x), axis=1))
    Rc = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Qc).cuda())))
    assert np.abs(Rc).max() < 1e-12
    Q = state(o)
    R = mesh.get_state(mesh.rhs(mesh.set_state(torch.from_numpy(Q).cuda())))
    total = sum(o.integrate(R, e) for e in range(box.n_elems))
    scale = sum(np.abs(o.integrate(R, e)) for e in range(box.n_elems))
    assert np.abs(total).max() < 1e-13 * scale.max()


def test_split_schedulers_bitwise_equal(dg):
    box, o, mesh = setup(dg, "mixed", 3, 4, "lf", None)
    Q = torch.from_numpy(state(o)).cuda()
    out = {}
    for sched in ("balanced", "naive", "static"):
        mesh.set_scheduler(sched)
        Qs = mesh.set_state(Q)
        mesh.rk_step(Qs, mesh.empty(), 1e-3, 1)
        out[sched] = Qs
    mesh.sync()
    assert torch.equal(out["balanced"], out["naive"]) and torch.equal(out["balanced"], out["static"])


def test_split_benchmark_mesh_sampled(dg):
    """The 16^3 mixed benchmark mesh at N = 4 with the split form, balanced
    scheduler after autotuning: sampled elements (hexahedra among them)
    against the oracle, plain per-variable metric."""
    from oracle.mesh import from_box
    from oracle.split_form import SplitFormOracle
    box = di.box_mesh(16, "mixed", seed=2)
    N = 4
    mesh = dg.Mesh(box, N, flux="lf")
    mesh.set_volume_form("split")
    n = N + 1
    vals = di.perturbed_tgv_state(mesh.quad_points(), seed=3, amp=FULL_SIZE_AMP)
    Qs = mesh.project(torch.from_numpy(vals.reshape(5, box.n_elems, n ** 3).transpose(1, 0, 2).copy()).cuda())
    mesh.autotune(Qs, 1e-4)
    R = mesh.get_state(mesh.rhs(Qs))
    Q = mesh.get_state(Qs)
    o = SplitFormOracle(from_box(box, N), flux="lf")
    rng = np.random.default_rng(12)
    hexes = np.where(box.etype == 0)[0]
    elems = np.sort(np.concatenate([rng.choice(hexes, 6, replace=False),
                                    rng.choice(box.n_elems, 10, replace=False)]))
    mask = np.zeros(len(Q), dtype=bool)
    for e in elems:
        mask[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] = True
    assert_sampled_parity(R, o.rhs(Q, elems), var_index(o.mesh.nM), mask, label="split 16^3")


def test_split_form_rejections(dg):
    import paper_2511_08020_gb300 as pkg
    box = make_box("mixed", 2, seed=1)
    mesh = dg.Mesh(box, 2, flux="lf")
    mesh.set_volume_form("split")
    Q = mesh.empty().fill_(1.0)
    with pytest.raises(pkg.DGError):
        mesh.rhs_vjp(Q, Q)
    with pytest.raises(pkg.DGError):
        mesh.set_physics("navier_stokes", 0.01, 0.72)
    mesh.set_volume_form("weak")
    mesh.set_physics("navier_stokes", 0.01, 0.72)
    with pytest.raises(pkg.DGError):
        mesh.set_volume_form("split")
    curved = dg.Mesh(di.perturb_vertices(make_box("hex", 2, seed=1), 0.1), 2, geometry="vertex")
    with pytest.raises(pkg.DGError):
        curved.set_volume_form("split")
