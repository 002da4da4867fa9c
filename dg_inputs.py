"""Seeded synthetic inputs for the modal DG hot path.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds none of the discretisation's arithmetic (no basis, quadrature, flux or
time stepping): it only builds periodic box meshes out of cubes and evaluates
pointwise initial states at caller-supplied physical points.

Mesh recipe (periodic box [-pi, pi]^3 of m^3 cubes of side 2*pi/m):
  * 'mixed'  - every (i, j) cube column is, by a seeded hash, either a prism
               column (each cube split along its x=y diagonal plane into two
               prisms) or a hex column; every cube of a hex column is, by a
               second hash, kept as a hexahedron or split into 6 pyramids whose
               bases are the cube faces and whose apex is the cube centre.
  * 'kuhn'   - every cube split into the 6 Kuhn tetrahedra that share the
               v000-v111 diagonal (same orientation in every cube, so the mesh
               is conforming across cubes and across the periodic boundary).
  * 'four'   - all four types in one conforming mesh: the x-slab of cubes
               i < w (w = max(1, m // 4)) is split into Kuhn tetrahedra; the
               two neighbouring slabs (i = w and i = m - 1) are pyramid cubes
               whose pyramid facing the tet slab is split along the base
               diagonal the Kuhn split puts on that cube face (two tets); the
               remaining cubes follow the 'mixed' recipe (needs m >= 4).
  * 'hex', 'prism', 'pyramid' - all cubes of one kind (test meshes).
perturb_vertices() moves the vertices of any of these (curved geometry).
The hash is splitmix64(seed ^ id) compared with p * 2^64 (a decision is taken
when the hash is below the threshold).  Column ids are i + m*j; cube ids are
i + m*(j + m*k) + 2^32 so the two hash streams never share an input.

Element vertex orders follow the reference elements of the paper's polytopal
DGSEM (Sec. 2): hex lexicographic (x fastest); prism = bottom triangle then the
same triangle extruded; pyramid = base quadrilateral in lexicographic order of
its two in-plane axes, then the apex; tet = the 4 vertices along the Kuhn path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1

HEX, PRISM, PYR, TET = 0, 1, 2, 3
TYPE_NAMES = ("hex", "prism", "pyramid", "tet")
NVERT = (8, 6, 5, 4)


def splitmix64(x: int) -> int:
    """splitmix64 (Steele, Lea, Flood 2014) finaliser of x + golden gamma."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _decide(seed: int, ident: int, p: float) -> bool:
    return splitmix64((seed ^ ident) & MASK64) < int(p * 2.0 ** 64)


@dataclass
class BoxMesh:
    """Mesh in the layout dg_mesh_create reads (caller order)."""
    xyz: np.ndarray            # [n_vertices, 3] float64
    etype: np.ndarray          # [n_elems] int8
    elem_vert_off: np.ndarray  # [n_elems + 1] int64 (CSR)
    elem_verts: np.ndarray     # [sum nvert] int64
    period: np.ndarray         # [3] float64 box lengths (periodic in x, y, z)
    m: int
    kind: str
    seed: int

    @property
    def n_elems(self) -> int:
        return int(self.etype.shape[0])

    def verts_of(self, e: int) -> np.ndarray:
        return self.elem_verts[self.elem_vert_off[e]:self.elem_vert_off[e + 1]]

    def type_counts(self) -> dict:
        return {TYPE_NAMES[t]: int((self.etype == t).sum()) for t in range(4)}


def box_mesh(m: int, kind: str = "mixed", seed: int = 1, p_prism: float = 0.5,
             p_pyr: float = 0.5, length: float = 2.0 * math.pi,
             origin: float = -math.pi) -> BoxMesh:
    """Periodic box of m^3 cubes split per the recipe in the module docstring."""
    h = length / m
    n1 = m + 1
    gi = np.arange(n1, dtype=np.float64)
    X, Y, Z = np.meshgrid(gi, gi, gi, indexing="ij")
    # vertex id = i + n1*(j + n1*k)
    grid = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                     Z.transpose(2, 1, 0).ravel()], axis=1)
    xyz = [origin + h * grid]
    n_grid = n1 ** 3
    centres = []

    def vid(i, j, k):
        return i + n1 * (j + n1 * k)

    types, conn = [], []
    for k in range(m):
        for j in range(m):
            for i in range(m):
                v = {}
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            v[(dx, dy, dz)] = vid(i + dx, j + dy, k + dz)
                split_face = None   # (axis, side) of a pyramid cube's face split into two tets
                if kind == "four":
                    if m < 4:
                        raise ValueError("'four' meshes need m >= 4")
                    w = max(1, m // 4)
                    if i < w:
                        sub = "kuhn"
                    elif i == w:
                        sub, split_face = "pyramid", (0, 0)
                    elif i == m - 1:
                        sub, split_face = "pyramid", (0, 1)
                    elif _decide(seed, i + m * j, p_prism):
                        sub = "prism"
                    else:
                        cube_id = i + m * (j + m * k) + (1 << 32)
                        sub = "pyramid" if _decide(seed, cube_id, p_pyr) else "hex"
                elif kind == "mixed":
                    is_prism_col = _decide(seed, i + m * j, p_prism)
                    if is_prism_col:
                        sub = "prism"
                    else:
                        cube_id = i + m * (j + m * k) + (1 << 32)
                        sub = "pyramid" if _decide(seed, cube_id, p_pyr) else "hex"
                elif kind == "kuhn":
                    sub = "kuhn"
                elif kind in ("hex", "prism", "pyramid"):
                    sub = kind
                else:
                    raise ValueError(f"unknown mesh kind {kind!r}")

                if sub == "hex":
                    types.append(HEX)
                    conn.append([v[(b & 1, (b >> 1) & 1, (b >> 2) & 1)] for b in range(8)])
                elif sub == "prism":
                    # split along the x=y plane through the v000-v001 and v110-v111 edges
                    for tri in (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))):
                        types.append(PRISM)
                        conn.append([v[(a, b, 0)] for (a, b) in tri] + [v[(a, b, 1)] for (a, b) in tri])
                elif sub == "pyramid":
                    c_id = n_grid + len(centres)
                    centres.append(origin + h * np.array([i + 0.5, j + 0.5, k + 0.5]))
                    for axis in range(3):
                        for side in (0, 1):
                            u, w = [d for d in range(3) if d != axis]
                            base = []
                            for bw in (0, 1):
                                for bu in (0, 1):
                                    d = [0, 0, 0]
                                    d[axis], d[u], d[w] = side, bu, bw
                                    base.append(v[tuple(d)])
                            if split_face == (axis, side):
                                # the Kuhn split of the neighbouring cube puts the
                                # diagonal base[0]-base[3] on this face
                                for tri in ((0, 1, 3), (0, 2, 3)):
                                    types.append(TET)
                                    conn.append([base[t] for t in tri] + [c_id])
                            else:
                                types.append(PYR)
                                conn.append(base + [c_id])
                elif sub == "kuhn":
                    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
                        d = [0, 0, 0]
                        path = [v[tuple(d)]]
                        for ax in perm[:2]:
                            d[ax] = 1
                            path.append(v[tuple(d)])
                        path.append(v[(1, 1, 1)])
                        types.append(TET)
                        conn.append(path)
    if centres:
        xyz.append(np.array(centres))
    xyz = np.concatenate(xyz, axis=0)
    etype = np.array(types, dtype=np.int8)
    off = np.zeros(len(conn) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(c) for c in conn])
    verts = np.array([x for c in conn for x in c], dtype=np.int64)
    return BoxMesh(xyz=xyz, etype=etype, elem_vert_off=off, elem_verts=verts,
                   period=np.array([length] * 3), m=m, kind=kind, seed=seed)



# Vertex reorderings that map each reference element onto itself (so the
# element stays an affine image of its reference element, possibly with the
# opposite orientation).  hex: the 48 symmetries of the cube act on the 3
# vertex bits (axis permutation + per-axis flip); prism: the 6 symmetries of
# the triangle (top follows bottom); pyramid: the 8 symmetries of the base
# square (apex last); tet: all 24 vertex permutations.
def _hex_syms():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for flip in range(8):
            m = []
            for b in range(8):
                bits = [(b >> k) & 1 for k in range(3)]
                nb = [bits[perm[k]] ^ ((flip >> k) & 1) for k in range(3)]
                m.append(nb[0] | (nb[1] << 1) | (nb[2] << 2))
            out.append(m)
    return out


def _prism_syms():
    import itertools
    return [list(p) + [q + 3 for q in p] for p in itertools.permutations(range(3))]


def _pyr_syms():
    out = []
    for sw in (0, 1):
        for fx in (0, 1):
            for fy in (0, 1):
                m = []
                for b in range(4):
                    x, y = b & 1, b >> 1
                    if sw:
                        x, y = y, x
                    x ^= fx
                    y ^= fy
                    m.append(x | (y << 1))
                out.append(m + [4])
    return out


def _tet_syms():
    import itertools
    return [list(p) for p in itertools.permutations(range(4))]


def reorder_vertices(box: BoxMesh, seed: int) -> BoxMesh:
    """Apply a seeded random self-map of the reference element to every
    element's vertex list (exercises every face orientation case)."""
    syms = {HEX: _hex_syms(), PRISM: _prism_syms(), PYR: _pyr_syms(), TET: _tet_syms()}
    rng = np.random.Generator(np.random.PCG64(seed))
    verts = box.elem_verts.copy()
    for e in range(box.n_elems):
        lo, hi = box.elem_vert_off[e], box.elem_vert_off[e + 1]
        opts = syms[int(box.etype[e])]
        m = opts[rng.integers(len(opts))]
        verts[lo:hi] = box.elem_verts[lo:hi][m]
    return BoxMesh(xyz=box.xyz, etype=box.etype, elem_vert_off=box.elem_vert_off, elem_verts=verts,
                   period=box.period, m=box.m, kind=box.kind + "+reordered", seed=box.seed)


def perturb_vertices(box: BoxMesh, amp: float, seed: int = 11, smooth: bool = False) -> BoxMesh:
    """Curved-geometry variant of a box mesh: every vertex is moved, so hex,
    prism and pyramid elements are no longer affine images of their reference
    elements (tetrahedra stay affine).  Periodic images of a lattice vertex
    move together, so the mesh stays conforming and periodic.

      smooth = False: lattice vertex (i, j, k) moves by amp * h * (u0, u1, u2),
        u_d uniform on [-1, 1) from splitmix64(seed ^ (3 v + d)) with
        v = (i mod m) + m ((j mod m) + m (k mod m)); a cube centre (pyramid
        apex) by the same rule with v = m^3 + cube id.
      smooth = True: every vertex x moves by amp * (sin y sin z, sin z sin x,
        sin x sin y) (a fixed smooth periodic deformation of the box, so the
        elements become affine as the mesh is refined)."""
    m = box.m
    h = float(box.period[0]) / m
    n1 = m + 1
    xyz = box.xyz.copy()
    n_grid = n1 ** 3
    if smooth:
        X = box.xyz
        d = np.stack([np.sin(X[:, 1]) * np.sin(X[:, 2]), np.sin(X[:, 2]) * np.sin(X[:, 0]),
                      np.sin(X[:, 0]) * np.sin(X[:, 1])], axis=1)
        xyz = X + amp * d
    else:
        origin = float(box.xyz[0, 0])
        for v in range(box.xyz.shape[0]):
            if v < n_grid:
                i, j, k = v % n1, (v // n1) % n1, v // (n1 * n1)
                key = (i % m) + m * ((j % m) + m * (k % m))
            else:
                c = np.rint((box.xyz[v] - origin) / h - 0.5).astype(np.int64)
                key = m ** 3 + int(c[0] + m * (c[1] + m * c[2]))
            for dd in range(3):
                u = splitmix64((seed ^ (3 * key + dd)) & MASK64) / 2.0 ** 64
                xyz[v, dd] += amp * h * (2.0 * u - 1.0)
    return BoxMesh(xyz=xyz, etype=box.etype, elem_vert_off=box.elem_vert_off, elem_verts=box.elem_verts,
                   period=box.period, m=box.m, kind=box.kind + ("+smooth" if smooth else "+jitter"), seed=box.seed)


# --------------------------------------------------------------------------
# Pointwise initial states (conservative variables rho, rho u, rho v, rho w, E)
# --------------------------------------------------------------------------

def primitive_to_conservative(rho, u, v, w, p, gamma=1.4):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def tgv_primitive(x, gamma=1.4, mach=0.1, rho0=1.0, v0=1.0):
    """Taylor-Green vortex (Sec. 4): rho = rho0, p0 = rho0 V0^2 / (gamma Ma^2)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    p0 = rho0 * v0 * v0 / (gamma * mach * mach)
    rho = np.full_like(X, rho0)
    u = v0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -v0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(X)
    p = p0 + rho0 * v0 * v0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return rho, u, v, w, p


def tgv_state(x, gamma=1.4, mach=0.1):
    return primitive_to_conservative(*tgv_primitive(x, gamma, mach), gamma=gamma)


def perturbation_coeffs(seed: int):
    """Random amplitudes (alpha, beta) ~ U(-1, 1) for 5 variables x 4 modes x 3 axes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(2, 5, 4, 3))


def perturbed_tgv_state(x, seed: int, amp: float = 1e-2, gamma=1.4, mach=0.1):
    """TGV plus a smooth perturbation of the primitive variables built from the
    4 lowest Fourier modes per axis: delta_v = amp * s_v * sum_m sum_d
    (alpha sin(m x_d) + beta cos(m x_d)), normalised so that its bound
    sum |alpha| + |beta| equals 1, with s = (1, 1, 1, 1, p0)."""
    x = np.asarray(x, dtype=np.float64)
    rho, u, v, w, p = tgv_primitive(x, gamma, mach)
    ab = perturbation_coeffs(seed)
    p0 = 1.0 / (gamma * mach * mach)
    scale = (1.0, 1.0, 1.0, 1.0, p0)
    prim = [rho, u, v, w, p]
    out = []
    for var in range(5):
        d = np.zeros_like(rho)
        for mm in range(4):
            for ax in range(3):
                d += ab[0, var, mm, ax] * np.sin((mm + 1) * x[..., ax]) + \
                     ab[1, var, mm, ax] * np.cos((mm + 1) * x[..., ax])
        bound = np.abs(ab[:, var]).sum()
        out.append(prim[var] + amp * scale[var] * d / bound)
    return primitive_to_conservative(*out, gamma=gamma)


def advected_density_state(x, t=0.0, amp=0.2, vel=(1.0, 1.0, 1.0), p=1.0, gamma=1.4):
    """Smooth density wave rho = 1 + amp sin(x+y+z - (u+v+w) t) at constant
    velocity and pressure; an exact solution of the Euler equations."""
    x = np.asarray(x, dtype=np.float64)
    ph = x[..., 0] + x[..., 1] + x[..., 2] - (vel[0] + vel[1] + vel[2]) * t
    rho = 1.0 + amp * np.sin(ph)
    ones = np.ones_like(rho)
    return primitive_to_conservative(rho, vel[0] * ones, vel[1] * ones, vel[2] * ones, p * ones, gamma)


def random_modal_state(n_modes_per_elem, seed: int, mean=(1.0, 0.1, -0.05, 0.02, 180.0), amp=1e-3):
    """Modal coefficients in caller layout: for each element 5 blocks of
    nM coefficients; the first coefficient of each block is the given mean
    value, the others are amp * mean-scale * U(-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    blocks = []
    scale = np.array([1.0, 1.0, 1.0, 1.0, mean[4]])
    for nm in n_modes_per_elem:
        b = amp * scale[:, None] * rng.uniform(-1.0, 1.0, size=(5, nm))
        b[:, 0] = mean
        blocks.append(b.ravel())
    return np.concatenate(blocks)


def random_vector(n: int, seed: int, amp=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.uniform(-1.0, 1.0, size=n)


def batch_workload(n_instances: int = 64, seed: int = 5, m_min: int = 4, m_max: int = 20,
                   degrees=(2, 3, 4, 5)):
    """Serving-style batch recipe: instance i gets m_i cubes per direction,
    uniform on [m_min, m_max] from splitmix64(seed ^ (2i + 2^40)), a degree
    N_i uniform on `degrees` from splitmix64(seed ^ (2i + 1 + 2^40)), and a
    'mixed' box mesh hashed with seed + i.  Returns [(m_i, N_i, mesh_seed_i)]."""
    out = []
    span = m_max - m_min + 1
    for i in range(n_instances):
        hm = splitmix64((seed ^ (2 * i + (1 << 40))) & MASK64)
        hn = splitmix64((seed ^ (2 * i + 1 + (1 << 40))) & MASK64)
        out.append((m_min + hm % span, int(degrees[hn % len(degrees)]), seed + i))
    return out


def vertex_velocities(xyz, amp=0.1):
    """Constant vertex velocities of a mesh in motion: the periodic field
    amp (sin y sin z, sin z sin x, sin x sin y) at every vertex (periodic
    images move alike, so the mesh stays conforming and periodic)."""
    x = np.asarray(xyz, dtype=np.float64)
    return amp * np.stack([np.sin(x[:, 1]) * np.sin(x[:, 2]), np.sin(x[:, 2]) * np.sin(x[:, 0]),
                           np.sin(x[:, 0]) * np.sin(x[:, 1])], axis=1)
