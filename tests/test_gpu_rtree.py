"""Multigrid on R*-tree agglomerates (Section 4.1): the oracle's R*-tree maps
(irregular agglomerates, irregular coarse neighbourhoods) drive both the
oracle and the CUDA path; V-cycle and time steps must agree as on the
structured hierarchies."""
import dataclasses

import numpy as np
import pytest

from oracle import monodomain as omd
from oracle import multigrid as omg
from oracle import rtree
from paper_2602_16312_gb300 import workloads as W

from gpu_util import oracle_setup, rel, step_opts

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _rtree_workload(wl, M):
    tree = rtree.build(wl.mesh.vertices, wl.mesh.elements, M)
    maps = rtree.agglomeration_maps(tree, wl.mesh.n_elements, tree.root.level + 1)
    return dataclasses.replace(wl, maps=maps)


CASES = {
    "jsquare2d_q2_30_M8": lambda: _rtree_workload(W.jittered_square_2d(n=30, n_levels=2), 8),
    "jcube3d_q2_6_M8": lambda: _rtree_workload(W.jittered_cube_3d(n=6, degree=2, n_levels=2, group=2), 8),
    "shell_q2_M6": lambda: _rtree_workload(W.ventricle_shell(16, 8, 4, n_levels=2), 6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_and_trajectory_on_rtree_hierarchy(name):
    from paper_2602_16312_gb300 import aggmg
    wl = CASES[name]()
    disc, ho = oracle_setup(wl)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    assert hier.n_levels == len(wl.maps) + 1
    r = np.random.default_rng(61).standard_normal(disc.n)
    z = torch.empty(disc.n, dtype=torch.float64, device="cuda")
    hier.vcycle_apply(_dev(r), z)
    torch.cuda.synchronize()
    assert rel(z.cpu().numpy(), omg.vcycle(ho, r)) <= 1e-10
    opts = step_opts(wl)
    mask = wl.stim_mask_nodal()
    n_steps = 6
    u_ref, w_ref, its_ref = omd.run(disc, ho, opts, np.zeros(disc.n), np.zeros(disc.n), mask, n_steps)
    sim = aggmg.Monodomain(hier, wl.dt, wl.ionic, iapp_mask=_dev(mask), iapp_value=wl.iapp_value,
                           iapp_steps=wl.iapp_steps, rtol=wl.rtol)
    u = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    w = torch.zeros(disc.n, dtype=torch.float64, device="cuda")
    its = sim.step(u, w, n_steps)
    sim.close()
    assert its == its_ref
    assert rel(u.cpu().numpy(), u_ref) <= 1e-10
