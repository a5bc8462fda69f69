"""The chunked full-size products of tests/oracle_rows.py equal the products
of the oracle's full assembly (same rows, assembled per chunk with the
chunk's face neighbours), on small meshes of every kind the full-size tests
use: the jittered square, the jittered cube and the periodic shell."""
import numpy as np
import pytest

import oracle_rows
from oracle import sipg
from paper_2602_16312_gb300 import workloads as W

CASES = [
    ("W.jittered_square_2d(n=12, degree=2, n_levels=2)", (3, 2)),
    ("W.jittered_cube_3d(n=5, degree=2, n_levels=2, group=4)", (2, 2, 2)),
    ("W.ventricle_shell(n_circ=8, n_long=5, n_trans=3, n_levels=2)", (2, 2, 1)),
]


@pytest.mark.parametrize("expr,pieces", CASES)
def test_chunked_products_equal_full_assembly(expr, pieces):
    wl = eval(expr)
    disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements, wl.conductivity, wl.degree, wl.penalty_mode,
                         wl.penalty_coeff)
    rng = np.random.default_rng(5)
    xs = [rng.standard_normal(disc.n) for _ in range(2)]
    out = oracle_rows.oracle_products(expr, wl.mesh.grid_shape, pieces, xs, [(0, "MA"), (1, "A")], workers=2)
    for (mv, av), (k, ops) in zip(out, [(0, "MA"), (1, "A")]):
        ref_a = disc.A @ xs[k]
        assert np.abs(av - ref_a).max() <= 1e-14 * np.abs(ref_a).max()
        if "M" in ops:
            ref_m = disc.M @ xs[k]
            assert np.abs(mv - ref_m).max() <= 1e-14 * np.abs(ref_m).max()
        else:
            assert mv is None


def test_face_neighbours_across_the_periodic_seam():
    wl = W.ventricle_shell(n_circ=8, n_long=3, n_trans=2, n_levels=2)
    nu = wl.mesh.grid_shape[0]
    # element 0 (u index 0) neighbours element nu-1 across the seam
    got = oracle_rows.face_neighbours(wl.mesh.elements, np.array([0]), 3)
    assert nu - 1 in got and 1 in got and nu in got
    assert len(got) == 1 + 4      # seam, +u, +v, +s (v = 0 and s = 0 are boundaries)
