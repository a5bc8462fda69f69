"""The cost model behind bench.py's roofline figures (agg_kernel_cost), checked
through the C ABI: the float64 SpMV's algorithmic bytes against a count made
here from the mesh (every stored entry of the face-structured operator, its
neighbour ids and face codes, x and y once), the whole-iteration figure
(id 4) against the per-kernel figures it must contain, and the ids that
agg_profile_kernel and single-level hierarchies reject."""
import pytest

from paper_2602_16312_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_16312_gb300 import build
    build.build()


def test_fp64_spmv_bytes_match_a_count_from_the_mesh():
    from paper_2602_16312_gb300 import aggmg
    n, p = 32, 2
    wl = W.jittered_square_2d(n=n, degree=p, n_levels=3)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f32", fine="mf")
    B, NF, E = (p + 1) ** 2, p + 1, n * n
    sides = 2 * 2 * n * (n - 1)                          # interior faces, each seen from both elements
    entries = E * B * B + sides * (2 * NF * B - NF * NF)  # diagonal blocks; face rows and columns
    ids = E * 4 * 5                                      # neighbour id (int32) + face code per face slot
    N = E * B
    b0, f0 = hier.kernel_cost(0)
    assert b0 == entries * 8 + ids + 2 * N * 8
    assert f0 == 2 * entries
    hier.close()


@pytest.mark.parametrize("precision,fine", [("f32", "mf"), ("f64", "bsr"), ("bf16s", "mf")])
def test_iteration_cost_contains_its_kernels(precision, fine):
    from paper_2602_16312_gb300 import aggmg
    wl = W.jittered_square_2d(n=32, degree=2, n_levels=3)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=precision, fine=fine)
    c = [hier.kernel_cost(k)[0] for k in range(5)]
    # one iteration: the float64 SpMV, five level-0 steps with an operator
    # product besides the residual + restriction, one prolongation, and more
    assert c[4] > c[0] + 5 * c[1] + c[2] + c[3]
    assert all(x > 0 for x in c)
    with pytest.raises(aggmg.AggError) as err:
        hier.profile_kernel(4, 1)
    assert err.value.status == aggmg.AGG_EINVAL
    hier.close()


def test_single_level_hierarchy_has_no_vcycle_kernels():
    from paper_2602_16312_gb300 import aggmg
    wl = W.jittered_square_2d(n=8, degree=2, n_levels=2)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, [], precision="f64")
    assert hier.kernel_cost(0)[0] > 0
    for k in (1, 4):
        with pytest.raises(aggmg.AggError) as err:
            hier.kernel_cost(k)
        assert err.value.status == aggmg.AGG_EUNSUPPORTED
    hier.close()
