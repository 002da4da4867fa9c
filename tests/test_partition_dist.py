"""Multi-rank bookkeeping of the space-filling-curve partition of Sec. 3 on
the CPU with gloo ranks (the library runs one GPU per mesh; this is the plan a
partitioned run would follow, checked without a GPU):

  * dg_partition_plan splits the mesh into contiguous Hilbert runs of equal
    weight and lists each part's halo;
  * every rank holds only its own elements' states, receives its halo from
    the owners (send / recv), and evaluates Eq. 1 on its own elements with the
    oracle; gathered, the residual equals the single-domain one bit for bit
    (the halo holds every state a rank's elements need -- any other entry is
    NaN and would poison the result);
  * the trace-exchange plan of the device path (dg_halo_plan): the face keys
    each rank packs for a peer arrive in exactly the order in which the peer
    unpacks them;
  * the in-memory redistribution of Listing 2: new per-type weights, a new
    plan, and every rank sends the states of the elements it no longer owns
    to their new owners (the all-to-all exchange); afterwards each rank holds
    exactly its new elements, with their states unchanged;
  * Navier-Stokes (BR1) needs the two exchanges of the device path per
    stage: the halo states, then -- after each rank has lifted the gradients
    of its own elements -- the halo's lifted gradients; the residual of the
    own elements then equals the single-domain one bit for bit, and a rank
    holds no gradient it neither computed nor received.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _exchange(dist, rank, ws, send, recv_sizes):
    """send[q]: float64 array for rank q (or empty); recv_sizes[q]: doubles to
    receive from q.  Returns the received arrays."""
    reqs, bufs = [], {}
    for q in range(ws):
        if q == rank:
            continue
        if recv_sizes[q]:
            bufs[q] = torch.empty(recv_sizes[q], dtype=torch.float64)
            reqs.append(dist.irecv(bufs[q], src=q))
        if send[q].size:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send[q])), dst=q))
    for r in reqs:
        r.wait()
    return {q: b.numpy() for q, b in bufs.items()}


def _worker(rank, ws, port, outdir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import dg_inputs as di
    import paper_2511_08020_gb300 as dg
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    box = di.box_mesh(4, "four", seed=3)
    N = 2
    o = Oracle(from_box(box, N))
    m = o.mesh
    Qg = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))   # known to all only to cut blocks

    def blocks(Q, elems):
        if len(elems) == 0:
            return np.zeros(0)
        return np.concatenate([Q[m.dof_off[e]:m.dof_off[e + 1]] for e in elems])

    def size(elems):
        return int(sum(m.dof_off[e + 1] - m.dof_off[e] for e in elems))

    part, off, halo = dg.partition_plan(box, N, ws)
    own = np.nonzero(part == rank)[0]
    Ql = np.full_like(Qg, np.nan)
    for e in own:
        Ql[m.dof_off[e]:m.dof_off[e + 1]] = Qg[m.dof_off[e]:m.dof_off[e + 1]]
    # halo exchange: rank q needs halo[q] elements; I send those I own
    need = {q: halo[off[q]:off[q + 1]] for q in range(ws)}
    send = {q: blocks(Ql, [e for e in need[q] if part[e] == rank]) for q in range(ws)}
    recv_from = {q: [e for e in need[rank] if part[e] == q] for q in range(ws)}
    got = _exchange(dist, rank, ws, send, {q: size(recv_from[q]) for q in range(ws)})
    for q, arr in got.items():
        pos = 0
        for e in recv_from[q]:
            k = m.dof_off[e + 1] - m.dof_off[e]
            Ql[m.dof_off[e]:m.dof_off[e + 1]] = arr[pos:pos + k]
            pos += k
    R = o.rhs(Ql, own)
    np.save(os.path.join(outdir, f"R{rank}.npy"), blocks(R, own))
    np.save(os.path.join(outdir, f"own{rank}.npy"), own)

    # the trace-exchange plan of the device path (dg_halo_plan, host-only):
    # the keys of the faces rank q packs for me arrive in my receive order
    sf, rf, sk, rk = dg.halo_plan(box, N, part, ws, rank)
    soff, roff = np.concatenate([[0], np.cumsum(sf)]), np.concatenate([[0], np.cumsum(rf)])
    got = _exchange(dist, rank, ws, {q: sk[soff[q]:soff[q + 1]].astype(np.float64) for q in range(ws)},
                    {q: int(rf[q]) if q != rank else 0 for q in range(ws)})
    keys_ok = int(sf[rank] == 0 and rf[rank] == 0)
    for q in range(ws):
        if q != rank:
            keys_ok &= int(np.array_equal(got.get(q, np.zeros(0)).astype(np.int64), rk[roff[q]:roff[q + 1]]))
    # every received face touches one of my elements and one of q's
    for q in range(ws):
        for key in rk[roff[q]:roff[q + 1]]:
            e0 = int(key) // 8
            keys_ok &= int(part[e0] in (rank, q))
    np.save(os.path.join(outdir, f"keys{rank}.npy"), np.array([keys_ok, int(rf.sum())]))

    # redistribution after a change of weights (Listing 2): send the states of
    # the elements that move to their new owners, receive the incoming ones
    part2, _, _ = dg.partition_plan(box, N, ws, type_weight=[1.0, 2.5, 1.7, 0.8])
    out_to = {q: [e for e in own if part2[e] == q] for q in range(ws)}
    in_from = {q: [e for e in range(m.n_elems) if part[e] == q and part2[e] == rank] for q in range(ws)}
    got = _exchange(dist, rank, ws, {q: blocks(Ql, out_to[q]) if q != rank else np.zeros(0) for q in range(ws)},
                    {q: size(in_from[q]) if q != rank else 0 for q in range(ws)})
    held = {int(e): Ql[m.dof_off[e]:m.dof_off[e + 1]].copy() for e in own if part2[e] == rank}
    for q, arr in got.items():
        pos = 0
        for e in in_from[q]:
            k = m.dof_off[e + 1] - m.dof_off[e]
            held[int(e)] = arr[pos:pos + k]
            pos += k
    ok = sorted(held) == sorted(np.nonzero(part2 == rank)[0].tolist()) and \
        all(np.array_equal(v, Qg[m.dof_off[e]:m.dof_off[e + 1]]) for e, v in held.items())
    moved = int(sum(len(v) for q, v in out_to.items() if q != rank))
    np.save(os.path.join(outdir, f"redist{rank}.npy"), np.array([int(ok), moved]))
    dist.barrier()
    dist.destroy_process_group()


def _ns_worker(rank, ws, port, outdir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import dg_inputs as di
    import paper_2511_08020_gb300 as dg
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    box = di.box_mesh(3, "mixed", seed=3)
    N = 2
    o = NSOracle(from_box(box, N), mu=0.05)
    m = o.mesh
    Qg = o.project(lambda x: di.perturbed_tgv_state(x, seed=4, amp=0.05))
    part, off, halo = dg.partition_plan(box, N, ws)
    own = [int(e) for e in np.nonzero(part == rank)[0]]
    need = {q: [int(e) for e in halo[off[q]:off[q + 1]]] for q in range(ws)}
    # exchange 1: the halo states
    Ql = np.full_like(Qg, np.nan)
    for e in own:
        Ql[m.dof_off[e]:m.dof_off[e + 1]] = Qg[m.dof_off[e]:m.dof_off[e + 1]]
    mine = {q: [e for e in need[q] if part[e] == rank] for q in range(ws)}
    theirs = {q: [e for e in need[rank] if part[e] == q] for q in range(ws)}
    blk = lambda e: m.dof_off[e + 1] - m.dof_off[e]
    got = _exchange(dist, rank, ws,
                    {q: np.concatenate([Ql[m.dof_off[e]:m.dof_off[e + 1]] for e in mine[q]] or [np.zeros(0)])
                     for q in range(ws)},
                    {q: int(sum(blk(e) for e in theirs[q])) for q in range(ws)})
    for q, arr in got.items():
        pos = 0
        for e in theirs[q]:
            Ql[m.dof_off[e]:m.dof_off[e + 1]] = arr[pos:pos + blk(e)]
            pos += blk(e)
    # the own elements' lifted gradients (their faces reach only the halo)
    G = o.lifted_gradient(Ql, own)
    # exchange 2: the halo's lifted gradients, [3, 5, nM] per element
    gsize = lambda e: 3 * blk(e)
    got = _exchange(dist, rank, ws,
                    {q: np.concatenate([G[e].ravel() for e in mine[q]] or [np.zeros(0)]) for q in range(ws)},
                    {q: int(sum(gsize(e) for e in theirs[q])) for q in range(ws)})
    for q, arr in got.items():
        pos = 0
        for e in theirs[q]:
            G[e] = arr[pos:pos + gsize(e)].reshape(3, 5, -1)
            pos += gsize(e)
    # the residual of the own elements from the states and gradients held
    faces = sorted({f for e in own for f, _ in m.elem_faces[e]})
    fluxes = {f: o.ns_face_flux(Ql, f, G) for f in faces}
    R = np.concatenate([o.apply_minv(e, o.ns_volume_term(Ql, e, G) - o.surface_term(Ql, e, fluxes)).ravel()
                        for e in own])
    np.save(os.path.join(outdir, f"nsR{rank}.npy"), R)
    np.save(os.path.join(outdir, f"nsown{rank}.npy"), np.array(own))
    np.save(os.path.join(outdir, f"nsheld{rank}.npy"), np.array(sorted(G)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_partitioned_residual_and_redistribution(tmp_path, ws):
    sys.path.insert(0, ROOT)
    import dg_inputs as di
    import paper_2511_08020_gb300 as dg
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    torch.multiprocessing.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    box = di.box_mesh(4, "four", seed=3)
    N = 2
    o = Oracle(from_box(box, N))
    Qg = o.project(lambda x: di.perturbed_tgv_state(x, seed=3, amp=0.05))
    R = o.rhs(Qg)
    seen = np.zeros(box.n_elems, dtype=int)
    for r in range(ws):
        own = np.load(tmp_path / f"own{r}.npy")
        Rr = np.load(tmp_path / f"R{r}.npy")
        seen[own] += 1
        ref = np.concatenate([R[o.mesh.dof_off[e]:o.mesh.dof_off[e + 1]] for e in own])
        assert np.array_equal(Rr, ref)
        ok, moved = np.load(tmp_path / f"redist{r}.npy")
        assert ok == 1
        keys_ok, received = np.load(tmp_path / f"keys{r}.npy")
        assert keys_ok == 1 and received > 0
    assert np.all(seen == 1)
    part, _, _ = dg.partition_plan(box, N, ws)
    part2, _, _ = dg.partition_plan(box, N, ws, type_weight=[1.0, 2.5, 1.7, 0.8])
    assert np.any(part != part2)                   # the new weights do move elements


def test_partitioned_navier_stokes_two_exchanges(tmp_path):
    sys.path.insert(0, ROOT)
    import dg_inputs as di
    import paper_2511_08020_gb300 as dg
    from oracle.mesh import from_box
    from oracle.navier_stokes import NSOracle
    ws = 2
    torch.multiprocessing.spawn(_ns_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    box = di.box_mesh(3, "mixed", seed=3)
    N = 2
    o = NSOracle(from_box(box, N), mu=0.05)
    m = o.mesh
    Qg = o.project(lambda x: di.perturbed_tgv_state(x, seed=4, amp=0.05))
    R = o.rhs(Qg)
    part, off, halo = dg.partition_plan(box, N, ws)
    seen = np.zeros(box.n_elems, dtype=int)
    for r in range(ws):
        own = np.load(tmp_path / f"nsown{r}.npy")
        seen[own] += 1
        ref = np.concatenate([R[m.dof_off[e]:m.dof_off[e + 1]] for e in own])
        assert np.array_equal(np.load(tmp_path / f"nsR{r}.npy"), ref)
        held = set(np.load(tmp_path / f"nsheld{r}.npy").tolist())
        assert held == set(own.tolist()) | set(halo[off[r]:off[r + 1]].tolist())
        assert len(halo[off[r]:off[r + 1]]) > 0
    assert np.all(seen == 1)


def test_partition_plan_properties():
    """Contiguous Hilbert runs, balanced weights, symmetric halos."""
    sys.path.insert(0, ROOT)
    import dg_inputs as di
    import paper_2511_08020_gb300 as dg
    box = di.box_mesh(6, "mixed", seed=2)
    N = 2
    _, _, slots = dg.check_mesh(box, N)
    order = np.argsort(slots)                      # caller elements in Hilbert order
    tw = np.array([1.0, 1.6, 1.3, 1.0])
    for P in (1, 4, 7):
        part, off, halo = dg.partition_plan(box, N, P, type_weight=tw)
        seq = part[order]
        assert np.all(np.diff(seq) >= 0) and seq[0] == 0 and seq[-1] == P - 1    # contiguous runs
        w = np.bincount(part, weights=tw[box.etype], minlength=P)
        assert w.max() - w.min() <= 2 * tw.max() + 1e-12                          # within one element or two
        for p in range(P):
            h = halo[off[p]:off[p + 1]]
            assert np.all(part[h] != p) and np.all(np.diff(h) > 0)
    with pytest.raises(dg.DGError):
        dg.partition_plan(box, N, 0)
