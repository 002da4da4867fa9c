"""Host-side pins of the moving-mesh geometry (dg_geometry_at, no device):
the metric, J, inverse mass matrices, normals and face weights that the
library evaluates at time t from its polynomial coefficients must equal the
static pointwise geometry of the mesh with every vertex moved to
x_v + t u_v (the coefficients come from det and the adjugate of F0 + t F1,
the static builder inverts dx/dxi at the moved points: two independent
routes).  An element turned inside out is reported, tetrahedra rejected."""
import copy

import numpy as np
import pytest

import dg_inputs as di


@pytest.fixture(scope="module")
def dg():
    import paper_2511_08020_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("kind,N", [("hex", 2), ("prism", 3), ("pyramid", 2), ("mixed", 3), ("mixed", 4),
                                    ("mixed", 1)])
def test_geometry_at_equals_static_geometry_of_moved_vertices(dg, kind, N):
    box = di.perturb_vertices(di.box_mesh(2, kind, seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 0.3)
    for t in (0.0, 0.07, -0.11, 0.3):
        e1, f1 = dg.geometry_at(box, N, vel, t)
        moved = copy.copy(box)
        moved.xyz = box.xyz + t * vel
        e0, f0 = dg.geometry_at(moved, N)
        assert e1.shape == e0.shape and f1.shape == f0.shape
        assert np.abs(e1 - e0).max() < 1e-13 * np.abs(e0).max(), (kind, N, t)
        assert np.abs(f1 - f0).max() < 1e-13 * np.abs(f0).max(), (kind, N, t)


def test_zero_velocity_is_the_static_geometry(dg):
    box = di.perturb_vertices(di.box_mesh(2, "mixed", seed=2), 0.1)
    e0, f0 = dg.geometry_at(box, 3)
    e1, f1 = dg.geometry_at(box, 3, np.zeros_like(box.xyz), 0.8)
    assert np.abs(e1 - e0).max() < 1e-14 * np.abs(e0).max()
    assert np.abs(f1 - f0).max() < 1e-14 * np.abs(f0).max()


def test_inside_out_and_tetrahedra_are_rejected(dg):
    box = di.perturb_vertices(di.box_mesh(3, "hex", seed=1), 0.1)
    vel = di.vertex_velocities(box.xyz, 1.0)
    dg.geometry_at(box, 2, vel, 0.05)
    with pytest.raises(dg.DGError, match="inside out"):
        dg.geometry_at(box, 2, vel, 2.0)
    four = di.box_mesh(4, "four", seed=1)
    with pytest.raises(dg.DGError, match="hexahedra, prisms and pyramids"):
        dg.geometry_at(four, 2, di.vertex_velocities(four.xyz, 0.1), 0.1)
