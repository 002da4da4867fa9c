"""dg_rhs_vjp_noalloc: the allocation-free variant of dg_rhs_vjp for callers
that must not allocate device memory at call time.  Its adjoint face scratch
is a fixed 64 MiB array in the library image instead of a cudaMalloc'd
buffer.  Called through the C ABI; checked against dg_rhs_vjp on two calls
in a row with different cotangents (the second call must not depend on what
the first left in the shared array), and a mesh whose face scratch exceeds
the fixed size must be rejected with DG_ERR_ARG; free device memory must not
change across a call on a mesh that never ran dg_rhs_vjp.  This file is
collected last so that a run stopping at the first failure has run everything
else."""
import ctypes

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
    lib = pkg.load()
    lib.dg_rhs_vjp_noalloc.argtypes = [ctypes.c_void_p] * 5
    lib.dg_rhs_vjp_noalloc.restype = ctypes.c_int
    return pkg


def noalloc(dg, mesh, Q, W, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return dg.load().dg_rhs_vjp_noalloc(mesh.handle, ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("flux", ["lf", "roe"])
def test_noalloc_matches_rhs_vjp_twice(dg, flux):
    from oracle.elements import n_modes
    box = make_box("mixed", 3, seed=1, reorder=6)
    N = 3
    mesh = dg.Mesh(box, N, flux=flux)
    nM = [n_modes(int(t), N) for t in box.etype]
    vidx = var_index(nM)
    Q = mesh.set_state(di.random_modal_state(nM, seed=2, amp=1e-2))
    for seed in (31, 32):
        W = mesh.set_state(di.random_vector(mesh.n_dof, seed=seed))
        ref = mesh.get_state(mesh.rhs_vjp(Q, W))
        out = torch.full_like(Q, float("nan"))
        assert noalloc(dg, mesh, Q, W, out) == 0, dg.load().dg_last_error().decode()
        got = mesh.get_state(out)
        assert np.isfinite(got).all()
        assert rel_err(got, ref, vidx) < TOL
    mesh.sync()


def test_noalloc_on_a_curved_mesh(dg):
    from oracle.elements import n_modes
    box = di.perturb_vertices(make_box("four", 4, seed=1), 0.1)
    N = 2
    mesh = dg.Mesh(box, N, geometry="vertex")
    assert mesh.n_curved > 0
    nM = [n_modes(int(t), N) for t in box.etype]
    Q = mesh.set_state(di.random_modal_state(nM, seed=2, amp=1e-2))
    W = mesh.set_state(di.random_vector(mesh.n_dof, seed=33))
    ref = mesh.get_state(mesh.rhs_vjp(Q, W))
    out = torch.full_like(Q, float("nan"))
    assert noalloc(dg, mesh, Q, W, out) == 0, dg.load().dg_last_error().decode()
    np.testing.assert_array_equal(mesh.get_state(out), ref)
    mesh.sync()


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch(dg):
    box = make_box("mixed", 20, seed=2)   # ~58k faces x 2 x 5 x 25 doubles > 8 Mi doubles
    mesh = dg.Mesh(box, 4)
    Q = mesh.empty().fill_(1.0)
    W = mesh.empty().fill_(0.0)
    out = mesh.empty()
    status = noalloc(dg, mesh, Q, W, out)
    assert status == -1
    assert "64 MiB" in dg.load().dg_last_error().decode()


def test_noalloc_allocates_no_device_memory(dg):
    """Free device memory is the same before and after a call on a fresh mesh
    that has never run dg_rhs_vjp (whose first call cudaMallocs the face
    scratch); the same measurement does see that allocation afterwards."""
    from oracle.elements import n_modes
    N = 4
    # load the entry point's device code and kernels first (a module load
    # allocates device memory once per process)
    warm = dg.Mesh(make_box("mixed", 3, seed=1), N)
    Qw = warm.empty().fill_(0.0)
    assert noalloc(dg, warm, Qw, Qw, warm.empty()) == 0, dg.load().dg_last_error().decode()
    torch.cuda.synchronize()
    box = make_box("mixed", 10, seed=3)   # ~1.9 Mi doubles of face scratch (15 MB)
    mesh = dg.Mesh(box, N)
    nM = [n_modes(int(t), N) for t in box.etype]
    Q = mesh.set_state(di.random_modal_state(nM, seed=2, amp=1e-2))
    W = mesh.set_state(di.random_vector(mesh.n_dof, seed=34))
    out = torch.full_like(Q, float("nan"))
    ref = mesh.empty()
    mesh.rhs(Q)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert noalloc(dg, mesh, Q, W, out) == 0, dg.load().dg_last_error().decode()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    mesh.rhs_vjp(Q, W, ref)   # allocates the mesh's own face scratch
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free0 - free2 >= 8 << 20, (free0, free2)
    assert rel_err(mesh.get_state(out), mesh.get_state(ref), var_index(nM)) < TOL
    mesh.sync()
