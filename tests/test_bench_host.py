"""Host logic of bench.py on the CPU: the cell counts behind the roofline.

The roofline's algorithmic bytes count only the cells the bulk sweep updates,
i.e. all cells minus those the near-particle kernel takes (every cell whose
centre lies within R + 2 of the sphere centre along each axis, minimum image
in the periodic x and y, z closed).  bench.near_cells restates that rule in
closed form; here it is checked against a brute-force count over cell
centres.
"""
import numpy as np
import pytest

import bench


def _brute_force(particle, shape, halo=2.0):
    nx, ny, nz = shape
    R = 0.5 * particle["diameter"]
    inside = []
    for a, (n, periodic) in enumerate(((nx, True), (ny, True), (nz, False))):
        d = np.arange(n) + 0.5 - particle["x"][a]
        if periodic:
            d -= n * np.round(d / n)
        inside.append(int(np.count_nonzero(np.abs(d) <= R + halo)))
    return inside[0] * inside[1] * inside[2]


@pytest.mark.parametrize("seed", range(6))
def test_near_cells_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        D = float(rng.uniform(4.0, 30.0))
        shape = tuple(int(v) for v in rng.integers(int(D) + 8, 3 * int(D) + 20, size=3))
        x = [float(rng.uniform(0.0, shape[0])), float(rng.uniform(0.0, shape[1])),
             float(rng.uniform(0.5 * D + 0.1, shape[2] - 0.5 * D - 0.1))]
        p = {"x": x, "diameter": D}
        assert bench.near_cells(p, shape) == _brute_force(p, shape), (p, shape)


def test_near_cells_of_the_settling_workload():
    """The benchmark's own sphere (D = 24 at (64, 64, 448) in 128 x 128 x 512):
    28 cells per axis (centres x + 1/2 in [50, 78], within 14 of the sphere
    centre)."""
    p = {"x": (64.0, 64.0, 448.0), "diameter": 24.0}
    assert bench.near_cells(p, (128, 128, 512)) == 28 ** 3 == _brute_force(p, (128, 128, 512))
