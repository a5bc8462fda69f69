"""The library's R*-tree agglomeration (agg_rtree_agglomerate, host C++)
against the oracle's, map for map and bit for bit: the same insertion order
and the same tie-breaking rules give the same tree."""
import dataclasses

import numpy as np
import pytest

from oracle import rtree
from paper_2602_16312_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2602_16312_gb300 import build
    build.build()


def _permuted(wl, seed):
    perm = np.random.default_rng(seed).permutation(wl.mesh.n_elements)
    return dataclasses.replace(wl, mesh=dataclasses.replace(wl.mesh, elements=wl.mesh.elements[perm]),
                               conductivity=wl.conductivity[perm])


CASES = {
    "jsquare2d_24": lambda: W.jittered_square_2d(n=24, n_levels=2),
    "jsquare2d_24_permuted": lambda: _permuted(W.jittered_square_2d(n=24, n_levels=2), 5),
    "jcube3d_7": lambda: W.jittered_cube_3d(n=7, degree=1, n_levels=2, group=1),
    "shell_q1": lambda: W.ventricle_shell(16, 8, 4, degree=1, n_levels=2),
}


@pytest.mark.parametrize("M", [4, 8, 13])
@pytest.mark.parametrize("name", list(CASES))
def test_maps_match_oracle(name, M):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    tree = rtree.build(wl.mesh.vertices, wl.mesh.elements, M)
    ref = rtree.agglomeration_maps(tree, wl.mesh.n_elements, tree.root.level + 1)
    got = aggmg.rtree_maps(aggmg.Mesh.from_workload(wl), M)
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        assert a.dtype == np.int32 and np.array_equal(a, b)


def test_rejections():
    from paper_2602_16312_gb300 import aggmg
    mesh = aggmg.Mesh.from_workload(W.square_2d_fhn(8, 1))
    with pytest.raises(aggmg.AggError) as e:
        aggmg.rtree_maps(mesh, 3)
    assert e.value.status == aggmg.AGG_EINVAL
    with pytest.raises(aggmg.AggError):
        aggmg.rtree_maps(mesh, 4, n_maps=50)
