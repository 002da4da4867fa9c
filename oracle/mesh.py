"""Mesh geometry and face connectivity for the oracle.

Each element is an affine image x = X0 + A (xi + 1)/2 of its reference element
(the mapping x = chi(xi) of Sec. 2; all meshes here are affine).  The map is
fitted by least squares to all element vertices and rejected when the residual
is not at rounding level.  J = |det A| / 8 and d xi / d x = 2 A^{-1}.

Faces are matched by the set of their vertex positions reduced modulo the box
periods.  The owner of a face is the element with the smaller caller index;
flux and face points are taken on the owner's side (reading c6).  The
neighbour's reference coordinates of each owner face point are obtained by
inverting the neighbour's affine map at the (periodically shifted) physical
point, independently of any combinatorial vertex matching.

Parity: pinned through the RHS invariants (free-stream preservation,
conservation, convergence) and the divergence-theorem check of the face rules.
"""
from __future__ import annotations

import numpy as np

from .elements import FACES, REF_VERTS, n_modes
from .quadrature import face_rule

QUANT = float(1 << 24)


def _corner(ref_verts, point):
    """Index of the reference vertex at `point`."""
    hit = np.where(np.all(np.abs(ref_verts - point) < 1e-12, axis=1))[0]
    if hit.size != 1:
        raise ValueError("reference vertex not found")
    return int(hit[0])


class OracleMesh:
    def __init__(self, xyz, etype, elem_vert_off, elem_verts, period, N):
        self.xyz = np.asarray(xyz, dtype=float)
        self.etype = np.asarray(etype, dtype=np.int64)
        self.N = int(N)
        self.period = None if period is None else np.asarray(period, dtype=float)
        off = np.asarray(elem_vert_off)
        ev = np.asarray(elem_verts)
        E = self.etype.size
        self.n_elems = E
        self.verts = [ev[off[e]:off[e + 1]] for e in range(E)]
        self.nM = np.array([n_modes(t, N) for t in self.etype])
        self.dof_off = np.zeros(E + 1, dtype=np.int64)
        self.dof_off[1:] = np.cumsum(5 * self.nM)

        # affine maps
        self.X0 = np.zeros((E, 3))
        self.A = np.zeros((E, 3, 3))
        for e in range(E):
            R = REF_VERTS[self.etype[e]]
            X = self.xyz[self.verts[e]]
            if X.shape[0] != R.shape[0]:
                raise ValueError(f"element {e}: wrong vertex count")
            # X_m = X0 + A (R_m + 1)/2 : least squares in the 12 unknowns
            M = np.hstack([np.ones((R.shape[0], 1)), (R + 1) / 2])
            sol, *_ = np.linalg.lstsq(M, X, rcond=None)
            resid = M @ sol - X
            scale = np.abs(X - X.mean(0)).max()
            if np.abs(resid).max() > 1e-10 * scale:
                raise ValueError(f"element {e} is not an affine image of its reference element")
            # The map is affine, so it is fixed exactly by the vertex at the
            # reference origin corner and the vertices one reference edge away
            # along each axis; exact vertex differences avoid the fit's rounding.
            o = _corner(R, -np.ones(3))
            self.X0[e] = X[o]
            for k in range(3):
                tip = -np.ones(3)
                tip[k] = 1.0
                self.A[e][:, k] = X[_corner(R, tip)] - X[o]
        det = np.linalg.det(self.A)
        if np.any(np.abs(det) < 1e-300):
            raise ValueError("degenerate element")
        self.J = np.abs(det) / 8.0
        self.dxi_dx = 2.0 * np.linalg.inv(self.A)   # [E, 3(xi_k), 3(x_d)]
        self.centroid = np.array([self.xyz[v].mean(0) for v in self.verts])

        self._match_faces()

    # ------------------------------------------------------------ faces
    def _key(self, vids):
        """Reduced face centroid plus the sorted reduced vertex positions (the
        centroid separates faces whose vertex sets coincide modulo a period,
        as on a box only two cells wide)."""
        P = self.xyz[vids]
        P = np.vstack([P.mean(0, keepdims=True), P])
        if self.period is not None:
            q = np.rint(P / self.period * QUANT).astype(np.int64) % int(QUANT)
        else:
            q = np.rint(P / (np.abs(self.xyz).max() + 1.0) * QUANT).astype(np.int64)
        rows = list(map(tuple, q.tolist()))
        return (rows[0],) + tuple(sorted(rows[1:]))

    def _match_faces(self):
        table = {}
        for e in range(self.n_elems):
            for lf, fv in enumerate(FACES[self.etype[e]]):
                table.setdefault(self._key(self.verts[e][fv]), []).append((e, lf))
        faces = []
        for key, sides in table.items():
            if len(sides) != 2:
                raise ValueError(f"face {key} has {len(sides)} sides; the mesh must be conforming and closed")
            (e0, l0), (e1, l1) = sorted(sides)
            faces.append((e0, l0, e1, l1))
        faces.sort()
        self.faces = faces
        self.elem_faces = [[] for _ in range(self.n_elems)]
        for f, (e0, l0, e1, l1) in enumerate(faces):
            self.elem_faces[e0].append((f, 0))
            self.elem_faces[e1].append((f, 1))

    def face_centroid(self, e, lf):
        return self.xyz[self.verts[e][FACES[self.etype[e]][lf]]].mean(0)

    def to_physical(self, e, ref):
        return self.X0[e] + 0.5 * (ref + 1.0) @ self.A[e].T

    def to_reference(self, e, x):
        return 2.0 * np.linalg.solve(self.A[e], (x - self.X0[e]).T).T - 1.0

    def face_geometry(self, f):
        """Owner-side face data: owner reference points, neighbour reference
        points (of the same physical points), weights w*S, outward normal."""
        e0, l0, e1, l1 = self.faces[f]
        ref0, w, ts, tt = face_rule(self.etype[e0], l0, self.N)
        x = self.to_physical(e0, ref0)
        dxds = 0.5 * self.A[e0] @ ts
        dxdt = 0.5 * self.A[e0] @ tt
        cr = np.cross(dxds, dxdt)
        S = np.linalg.norm(cr)
        nrm = cr / S
        if np.dot(nrm, self.face_centroid(e0, l0) - self.centroid[e0]) < 0:
            nrm = -nrm
        shift = np.zeros(3)
        if self.period is not None:
            d = self.face_centroid(e0, l0) - self.face_centroid(e1, l1)
            shift = np.rint(d / self.period) * self.period
        # invert the neighbour's map at the same physical points, measured from
        # the neighbour's origin vertex (local differences keep the rounding of
        # absolute coordinates and of the periodic shift out of the result)
        x_rel = (self.X0[e0] - shift - self.X0[e1]) + 0.5 * (ref0 + 1.0) @ self.A[e0].T
        ref1 = 2.0 * np.linalg.solve(self.A[e1], x_rel.T).T - 1.0
        return ref0, ref1, w * S, nrm

    def n_dof(self):
        return int(self.dof_off[-1])

    def block(self, Q, e):
        """View of element e's coefficients as [5, nM]."""
        return Q[self.dof_off[e]:self.dof_off[e + 1]].reshape(5, self.nM[e])


def from_box(box, N):
    return OracleMesh(box.xyz, box.etype, box.elem_vert_off, box.elem_verts, box.period, N)
