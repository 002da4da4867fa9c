"""Partitioned solve on one GPU (Sec. 3: each part owns a contiguous
space-filling-curve segment, the traces on shared faces are exchanged every
stage, and after a rebalance the states of the elements that change owner
move to their new part, the in-memory redistribution of Listing 2).

Two and three parts of one mesh live in one process on one GPU; the halo
exchange moves the packed trace blocks between the parts' device buffers.
The owned elements' states after LSERK steps must equal, bit for bit, those
of the whole mesh advanced by dg_rk_step -- for both fluxes, both schedulers,
four-type meshes with reordered vertices, the split form, Navier-Stokes
(with the second exchange of the gradient traces), and across a
redistribution to a new plan."""
import numpy as np
import pytest

import dg_inputs as di
from gpu_util import make_box

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


def caller_offsets(box, N):
    from oracle.elements import n_modes
    off = np.zeros(box.n_elems + 1, dtype=np.int64)
    off[1:] = np.cumsum([5 * n_modes(int(t), N) for t in box.etype])
    return off


def local_state(Q, off, part):
    """The part's caller-layout state: the blocks of its local elements."""
    return np.concatenate([Q[off[g]:off[g + 1]] for g in part.global_of_local])


def make_exchange(parts, bufs):
    nparts = len(parts)
    per = parts[0].doubles_per_face
    for p in range(nparts):
        for q in range(nparts):
            assert parts[p].send_faces[q] == parts[q].recv_faces[p]

    def seg(counts, k):
        a = int(counts[:k].sum()) * per
        return slice(a, a + int(counts[k]) * per)

    def exchange():
        for P, (send, _) in zip(parts, bufs):
            P.halo_pack(send)
        for p in range(nparts):
            for q in range(nparts):
                if parts[p].send_faces[q]:
                    bufs[q][1][seg(parts[q].recv_faces, p)].copy_(bufs[p][0][seg(parts[p].send_faces, q)])
        for P, (_, recv) in zip(parts, bufs):
            P.halo_unpack(recv)
    return exchange


def make_gradient_exchange(parts, bufs):
    """The Navier-Stokes second exchange: the gradient traces, same peers and
    order as the trace exchange, three times the block size."""
    per = 3 * parts[0].doubles_per_face

    def seg(counts, k):
        a = int(counts[:k].sum()) * per
        return slice(a, a + int(counts[k]) * per)

    def exchange():
        for P, (send, _) in zip(parts, bufs):
            P.halo_pack_gradients(send)
        for p in range(len(parts)):
            for q in range(len(parts)):
                if parts[p].send_faces[q]:
                    bufs[q][1][seg(parts[q].recv_faces, p)].copy_(bufs[p][0][seg(parts[p].send_faces, q)])
        for P, (_, recv) in zip(parts, bufs):
            P.halo_unpack_gradients(recv)
    return exchange


def owned_blocks(box, off, parts, Qs):
    """The whole caller-layout state assembled from every part's owned blocks."""
    out = np.full(int(off[-1]), np.nan)
    for P, Q in zip(parts, Qs):
        Ql = P.get_state(Q)
        loff = np.zeros(len(P.global_of_local) + 1, dtype=np.int64)
        loff[1:] = np.cumsum([off[g + 1] - off[g] for g in P.global_of_local])
        for i, g in enumerate(P.global_of_local):
            if not P.is_ghost[i]:
                out[off[g]:off[g + 1]] = Ql[loff[i]:loff[i + 1]]
    return out


CASES = [("mixed", 4, 3, "lf", None, 2, "balanced", "weak"), ("four", 4, 2, "roe", 5, 3, "naive", "weak"),
         ("mixed", 3, 4, "lf", 3, 2, "balanced", "split"), ("kuhn", 2, 3, "lf", 7, 3, "balanced", "weak")]


@pytest.mark.parametrize("kind,m,N,flux,reorder,nparts,sched,form", CASES)
def test_partitioned_steps_equal_whole_mesh(dg, kind, m, N, flux, reorder, nparts, sched, form):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = make_box(kind, m, seed=1, reorder=reorder)
    Q = Oracle(from_box(box, N)).project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    whole = dg.Mesh(box, N, flux=flux, scheduler=sched)
    whole.set_volume_form(form)
    Qw = whole.set_state(torch.from_numpy(Q).cuda())
    dt, nsteps = 1e-3, 3
    whole.rk_step(Qw, whole.empty(), dt, nsteps)
    ref = whole.get_state(Qw)
    part_of_elem, _, _ = dg.partition_plan(box, N, nparts)
    parts = [dg.Part(box, N, part_of_elem, nparts, p, flux=flux, scheduler=sched) for p in range(nparts)]
    off = caller_offsets(box, N)
    Qs, Ks = [], []
    for P in parts:
        P.set_volume_form(form)
        assert P.is_ghost.sum() > 0 and (P.is_ghost == 0).sum() == (part_of_elem == P.part).sum()
        Qs.append(P.set_state(torch.from_numpy(local_state(Q, off, P)).cuda()))
        Ks.append(P.empty())
    exchange = make_exchange(parts, [P.halo_buffers() for P in parts])
    dg.step_parts(parts, Qs, Ks, dt, nsteps, exchange)
    torch.cuda.synchronize()
    got = owned_blocks(box, off, parts, Qs)
    np.testing.assert_array_equal(got, ref)


NS_CASES = [("mixed", 4, 3, "lf", None, 2, "balanced"), ("four", 4, 2, "roe", 5, 3, "naive"),
            ("kuhn", 2, 3, "lf", 7, 2, "balanced")]


@pytest.mark.parametrize("kind,m,N,flux,reorder,nparts,sched", NS_CASES)
def test_partitioned_navier_stokes_equals_whole_mesh(dg, kind, m, N, flux, reorder, nparts, sched):
    """Navier-Stokes (BR1) parts: two exchanges per stage -- the traces before
    the lifting, the lifted gradient's traces before the flux -- and the
    owned elements equal the whole mesh's steps bit for bit."""
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = make_box(kind, m, seed=1, reorder=reorder)
    Q = Oracle(from_box(box, N)).project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    mu, Pr = 0.05, 0.72
    whole = dg.Mesh(box, N, flux=flux, scheduler=sched)
    whole.set_physics("navier_stokes", mu, Pr)
    Qw = whole.set_state(torch.from_numpy(Q).cuda())
    dt, nsteps = 1e-3, 2
    whole.rk_step(Qw, whole.empty(), dt, nsteps)
    ref = whole.get_state(Qw)
    part_of_elem, _, _ = dg.partition_plan(box, N, nparts)
    parts = [dg.Part(box, N, part_of_elem, nparts, p, flux=flux, scheduler=sched) for p in range(nparts)]
    off = caller_offsets(box, N)
    Qs, Ks = [], []
    for P in parts:
        P.set_physics("navier_stokes", mu, Pr)
        Qs.append(P.set_state(torch.from_numpy(local_state(Q, off, P)).cuda()))
        Ks.append(P.empty())
    exchange = make_exchange(parts, [P.halo_buffers() for P in parts])
    exchange_g = make_gradient_exchange(parts, [P.halo_gradient_buffers() for P in parts])
    dg.step_parts(parts, Qs, Ks, dt, nsteps, exchange, exchange_g)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(owned_blocks(box, off, parts, Qs), ref)
    # the flux half of a stage needs its lifting half first
    import paper_2511_08020_gb300 as pkg
    with pytest.raises(pkg.DGError):
        parts[0].rk_stage(Qs[0], Ks[0], dt, 0, last=False)


def storage_offsets(P, N):
    """Offsets of every local element's block in the part's storage layout
    (blocks in slot order)."""
    from oracle.elements import n_modes
    sizes = np.array([5 * n_modes(int(t), N) for t in P.etype])
    order = np.argsort(P.slot_of_elem)              # local elements by slot
    off = np.zeros(len(sizes), dtype=np.int64)
    off[order] = np.concatenate([[0], np.cumsum(sizes[order])[:-1]])
    return off, sizes


def test_redistribution_after_a_new_plan(dg):
    """Steps on an equal-count plan, then a weighted plan (the imbalance
    trigger's response): the stored blocks of the owned elements move to the
    part that owns them under the new plan (device copies addressed by
    global element), and stepping continues; the result equals the whole
    mesh's steps bit for bit (the blocks move in the storage layout, so the
    hexahedra's nodal values are not converted on the way)."""
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    box = make_box("mixed", 4, seed=2)
    N, dt, nparts = 3, 1e-3, 2
    Q = Oracle(from_box(box, N)).project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.1))
    whole = dg.Mesh(box, N)
    Qw = whole.set_state(torch.from_numpy(Q).cuda())
    whole.rk_step(Qw, whole.empty(), dt, 4)
    ref = whole.get_state(Qw)
    off = caller_offsets(box, N)
    plans = [dg.partition_plan(box, N, nparts)[0], dg.partition_plan(box, N, nparts, type_weight=[1.0, 3.0, 1.5, 1.0])[0]]
    assert (plans[0] != plans[1]).any()
    held = None              # global element -> its stored block (device), after the first plan
    for k, plan in enumerate(plans):
        parts = [dg.Part(box, N, plan, nparts, p) for p in range(nparts)]
        if k == 0:
            Qs = [P.set_state(torch.from_numpy(local_state(Q, off, P)).cuda()) for P in parts]
        else:
            Qs = []
            for P in parts:        # the in-memory redistribution: every owned block from its old part
                so, sz = storage_offsets(P, N)
                Qp = P.empty().fill_(float("nan"))
                for i, g in enumerate(P.global_of_local):
                    if not P.is_ghost[i]:
                        Qp[so[i]:so[i] + sz[i]].copy_(held[int(g)])
                Qs.append(Qp)
        Ks = [P.empty() for P in parts]
        dg.step_parts(parts, Qs, Ks, dt, 2, make_exchange(parts, [P.halo_buffers() for P in parts]))
        torch.cuda.synchronize()
        held = {}
        for P, Qp in zip(parts, Qs):
            so, sz = storage_offsets(P, N)
            for i, g in enumerate(P.global_of_local):
                if not P.is_ghost[i]:
                    held[int(g)] = Qp[so[i]:so[i] + sz[i]].clone()
        moved = sum(1 for g in range(box.n_elems) if plans[0][g] != plans[-1][g])
        assert k == 0 or moved > 0
        final = owned_blocks(box, off, parts, Qs)
        assert np.isfinite(final).all()
    np.testing.assert_array_equal(final, ref)


def test_partition_mesh_rejects_whole_mesh_calls(dg):
    import paper_2511_08020_gb300 as pkg
    box = make_box("mixed", 3, seed=1)
    plan, _, _ = dg.partition_plan(box, 2, 2)
    P = dg.Part(box, 2, plan, 2, 0)
    Q = P.empty().fill_(1.0)
    for call in (lambda: P.rhs(Q), lambda: P.rk_step(Q, P.empty(), 1e-3, 1), lambda: P.set_scheduler("static"),
                 lambda: P.rhs_vjp(Q, Q), lambda: P.halo_pack_gradients(Q), lambda: P.rk_stage_lift()):
        with pytest.raises(pkg.DGError):
            call()
    with pytest.raises(pkg.DGError):
        dg.Part(box, 2, plan, 2, 2)
