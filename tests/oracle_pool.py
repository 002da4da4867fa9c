"""The oracle's residual of a whole mesh spread over spawned worker processes
(test infrastructure: the oracle itself is unchanged).

Every worker builds its own oracle of the mesh and always evaluates the same
contiguous part of the element list, so its face tables stay warm; states
and residuals (real or complex) travel through shared memory, and a pipe per
worker carries only the go and done tokens.  Used for the oracle's
complex-step directional derivative through many LSERK steps of a mesh too
large for one process.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np


def _worker(conn, box, N, flux, elems, q_name, r_name, n_dof):
    from oracle.dg import Oracle
    from oracle.mesh import from_box
    o = Oracle(from_box(box, N), flux=flux)
    q_shm = shared_memory.SharedMemory(name=q_name)
    r_shm = shared_memory.SharedMemory(name=r_name)
    Q = np.ndarray((n_dof,), dtype=np.complex128, buffer=q_shm.buf)
    R = np.ndarray((n_dof,), dtype=np.complex128, buffer=r_shm.buf)
    off = o.mesh.dof_off
    conn.send("ready")
    while conn.recv() == "go":
        Rl = o.rhs(Q.copy(), elems=elems)
        for e in elems:
            R[off[e]:off[e + 1]] = Rl[off[e]:off[e + 1]]
        conn.send("done")
    del Q, R
    q_shm.close()
    r_shm.close()


class PooledOracle:
    """rhs(Q) of the whole mesh in complex arithmetic by `procs` workers;
    run(Q, dt, nsteps) the oracle's LSERK(5,4) steps with it."""

    def __init__(self, box, N, flux="lf", procs=None):
        from oracle.dg import LSERK_A, LSERK_B
        from oracle.mesh import from_box
        self.A, self.B = LSERK_A, LSERK_B
        m = from_box(box, N)
        self.n_dof = m.n_dof()
        procs = procs or os.cpu_count() or 1
        parts = [p for p in np.array_split(np.arange(box.n_elems), procs) if len(p)]
        nbytes = 16 * self.n_dof
        self.q_shm = shared_memory.SharedMemory(create=True, size=nbytes)
        self.r_shm = shared_memory.SharedMemory(create=True, size=nbytes)
        self.Q = np.ndarray((self.n_dof,), dtype=np.complex128, buffer=self.q_shm.buf)
        self.R = np.ndarray((self.n_dof,), dtype=np.complex128, buffer=self.r_shm.buf)
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for part in parts:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_worker, args=(b, box, N, flux, part, self.q_shm.name, self.r_shm.name,
                                                  self.n_dof), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    def rhs(self, Q):
        self.Q[:] = Q
        for c in self.conns:
            c.send("go")
        for c in self.conns:
            assert c.recv() == "done"
        return self.R.copy()

    def run(self, Q, dt, nsteps):
        Q = np.asarray(Q, dtype=np.complex128)
        for _ in range(nsteps):
            K = np.zeros_like(Q)
            for s in range(5):
                K = self.A[s] * K + dt * self.rhs(Q)
                Q = Q + self.B[s] * K
        return Q

    def close(self):
        for c in self.conns:
            c.send("stop")
        for p in self.procs:
            p.join(timeout=60)
        del self.Q, self.R
        self.q_shm.close()
        self.q_shm.unlink()
        self.r_shm.close()
        self.r_shm.unlink()
