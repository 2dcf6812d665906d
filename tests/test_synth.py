"""The seeded input generators (synth/) against the recipe they implement:
mesh orientation, region radii, boundary nodes, jitter bound, radial split,
workload sizes and the ranges of the batched cables.  The generators hold
none of the method's arithmetic; these checks pin the inputs both the oracle
and the GPU path consume."""

import numpy as np
import pytest

from synth import (BRAUER_BMAX, RADII, REGION_AIR, REGION_CORE, REGION_INSULATION, REGION_SHEATH, batched_cables,
                   coax_mesh, radial_intervals, workload)


@pytest.mark.parametrize("nr,ntheta,seed", [(5, 8, 0), (20, 40, 3), (37, 91, 11)])
def test_mesh_is_a_valid_polar_triangulation(nr, ntheta, seed):
    m = coax_mesh(nr, ntheta, seed=seed)
    xy, tri = m.xy, m.tri
    assert xy.shape[0] == 1 + nr * ntheta
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    det = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])
    assert np.all(det > 0)                                    # counter-clockwise, non-degenerate
    # the triangles tile the disc of radius 4 mm (polygonal boundary)
    area = 0.5 * det.sum()
    ring = np.hypot(*xy[m.dirichlet == 1].T)
    assert np.allclose(ring, RADII[3])
    assert area == pytest.approx(0.5 * ntheta * RADII[3] ** 2 * np.sin(2 * np.pi / ntheta), rel=1e-12)
    # every triangle's region matches its centroid radius
    c = (p0 + p1 + p2) / 3.0
    r = np.hypot(c[:, 0], c[:, 1])
    edges = (0.0,) + tuple(RADII)
    for reg in (REGION_CORE, REGION_INSULATION, REGION_SHEATH, REGION_AIR):
        sel = m.region == reg
        assert sel.any()
        assert np.all(r[sel] > edges[reg] - 0.15 * RADII[3] / nr) and np.all(r[sel] < edges[reg + 1])
    # Dirichlet nodes are exactly the outer ring
    assert int(m.dirichlet.sum()) == ntheta


def test_radial_split_follows_the_region_thicknesses():
    for nr in range(5, 300):
        c = radial_intervals(nr)
        assert sum(c) == nr and min(c) >= 1 and c[REGION_SHEATH] >= 2
    assert radial_intervals(100) == radial_intervals(100)
    with pytest.raises(ValueError):
        radial_intervals(4)


def test_workload_sizes_match_the_recipe():
    expect = {"tiny": 33, "small": 761, "medium": 19801, "paper": 2269}
    for name, ndof in expect.items():
        p = workload(name)
        assert int((p.mesh.dirichlet == 0).sum()) == ndof, name
        assert p.bmax[REGION_SHEATH] == BRAUER_BMAX and p.sigma[REGION_SHEATH] > 0
    p = workload("medium")
    assert (p.N, p.n_fine, p.sigma[REGION_SHEATH]) == (64, 50, 2e7)


def test_batched_cables_are_seeded_and_within_their_ranges():
    a, b = batched_cables(), batched_cables()
    assert len(a) == 32
    for p, q in zip(a, b):
        assert np.array_equal(p.mesh.xy, q.mesh.xy) and p.N == q.N and p.amp[0] == q.amp[0]
        assert 20 <= p.mesh.nr <= 200 and 40 <= p.mesh.ntheta <= 400
        assert 1.0 <= p.amp[0] <= 50.0 and 1e6 <= p.sigma[REGION_SHEATH] <= 3e7
        assert p.N in (16, 32, 64) and 20 <= p.n_fine <= 50
    assert len({(p.mesh.nr, p.mesh.ntheta) for p in a}) > 20          # uneven sizes
