"""The coarse-cycle kernels against the separate per-level kernels: the
persistent kernel (agg_mg_opts.coarse_persistent: levels >= 1 and the
coarsest solve in one cooperative launch) and the cluster kernel
(agg_mg_opts.coarse_cluster, the default: the smallest levels and the
coarsest solve on one thread-block cluster). The same
V-cycle and the same PCG solve, bit for bit, in every V-cycle precision and
for 2D and 3D blocks; fewer launches per V-cycle; and the bounded grid
barrier: when its arrivals never come, the solve ends with AGG_ECUDA instead
of hanging, and the device stays usable."""
import os

import numpy as np
import pytest

from paper_2602_16312_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aggmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import aggmg as mod
    from paper_2602_16312_gb300 import build
    build.build()
    return mod


def _hier(aggmg, wl, form, env=None, persistent=True, cluster=False):
    old = {}
    for k, v in (env or {}).items():
        old[k] = os.environ.get(k)
        os.environ[k] = v
    try:
        fine = "mf" if form != "f64" else "bsr"
        return aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=form, fine=fine,
                               coarse_persistent=persistent, coarse_cluster=cluster)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


CASES = {
    "square_q2_L4": lambda: W.jittered_square_2d(n=40, degree=2, n_levels=4),
    "cube_q2_L3": lambda: W.jittered_cube_3d(n=8, degree=2, n_levels=3, group=2),
    "square_q1_L3": lambda: W.jittered_square_2d(n=24, degree=1, n_levels=3),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("form", ["f64", "f32", "bf16s"])
def test_persistent_equals_separate_kernels_bitwise(aggmg, case, form):
    wl = CASES[case]()
    hp = _hier(aggmg, wl, form)
    hs = _hier(aggmg, wl, form, persistent=False)
    lp, ls = hp.launches(), hs.launches()
    assert lp["persistent"] and not ls["persistent"]
    L = wl.n_levels
    # 9 per level above the coarsest, less the segmented sums that the row-lane
    # levels 1 .. L-2 fuse into their first smoother step, + 2 for the coarsest
    assert ls["per_vcycle"] == 9 * (L - 1) + 2 - max(L - 2, 0)
    assert lp["per_vcycle"] == 9 + 1
    n = wl.n_dofs
    rng = np.random.default_rng(11)
    r = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
    zp, zs = torch.empty_like(r), torch.empty_like(r)
    for _ in range(2):                      # twice: the barrier resets between calls
        hp.vcycle_apply(r, zp)
        hs.vcycle_apply(r, zs)
        torch.cuda.synchronize()
        assert torch.equal(zp, zs), float((zp - zs).abs().max())
    b = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
    xp, xs = torch.zeros_like(b), torch.zeros_like(b)
    rp = hp.pcg_solve(b, xp, rtol=1e-10, flexible=(form != "f64"))
    rs = hs.pcg_solve(b, xs, rtol=1e-10, flexible=(form != "f64"))
    assert rp["iterations"] == rs["iterations"]
    assert torch.equal(xp, xs)
    hp.close()
    hs.close()


def test_barrier_timeout_ends_the_solve_with_an_error(aggmg):
    wl = W.jittered_square_2d(n=24, degree=2, n_levels=3)
    n = wl.n_dofs
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    # every barrier waits for one arrival that never comes
    h = _hier(aggmg, wl, "f64", {"AGG_PERSIST_TEST_EXTRA": "1"})
    assert h.launches()["persistent"]
    x = torch.zeros_like(b)
    with pytest.raises(aggmg.AggError) as e:
        h.pcg_solve(b, x, rtol=1e-8)
    assert e.value.status == aggmg.AGG_ECUDA
    assert "timed out" in str(e.value)
    h.close()
    # the device is still usable: a normal hierarchy solves
    h2 = _hier(aggmg, wl, "f64")
    assert h2.launches()["persistent"]
    x = torch.zeros_like(b)
    res = h2.pcg_solve(b, x, rtol=1e-8)
    assert res["status"] == 0 and res["iterations"] > 0
    h2.close()


CLUSTER_CASES = dict(CASES, square_q2_L2=lambda: W.jittered_square_2d(n=12, degree=2, n_levels=2),
                     shell_q2_L4=lambda: W.ventricle_shell(16, 8, 4, n_levels=4))


@pytest.mark.parametrize("case", list(CLUSTER_CASES))
@pytest.mark.parametrize("form", ["f64", "f32", "bf16s"])
def test_cluster_kernel_equals_separate_kernels_bitwise(aggmg, case, form):
    wl = CLUSTER_CASES[case]()
    hc = _hier(aggmg, wl, form, persistent=False, cluster=True)
    hs = _hier(aggmg, wl, form, persistent=False, cluster=False)
    lc, ls = hc.launches(), hs.launches()
    assert ls["cluster_level"] == -1 and not ls["persistent"]
    assert lc["cluster_level"] >= 1 and lc["cluster_ctas"] in (8, 16)
    L = wl.n_levels
    # 9 per level above the coarsest, less the segmented sums that the row-lane
    # levels 1 .. L-2 fuse into their first smoother step, + 2 for the coarsest
    assert ls["per_vcycle"] == 9 * (L - 1) + 2 - max(L - 2, 0)
    assert lc["per_vcycle"] == 9 * lc["cluster_level"] - (lc["cluster_level"] - 1) + 1
    n = wl.n_dofs
    rng = np.random.default_rng(12)
    r = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
    zc, zs = torch.empty_like(r), torch.empty_like(r)
    for _ in range(2):
        hc.vcycle_apply(r, zc)
        hs.vcycle_apply(r, zs)
        torch.cuda.synchronize()
        assert torch.equal(zc, zs), float((zc - zs).abs().max())
    b = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
    xc, xs = torch.zeros_like(b), torch.zeros_like(b)
    rc = hc.pcg_solve(b, xc, rtol=1e-10, flexible=(form != "f64"))
    rs = hs.pcg_solve(b, xs, rtol=1e-10, flexible=(form != "f64"))
    assert rc["iterations"] == rs["iterations"]
    assert torch.equal(xc, xs)
    hc.close()
    hs.close()
