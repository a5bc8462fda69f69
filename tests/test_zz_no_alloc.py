"""agg_operator_apply_static against agg_operator_apply, through the C ABI.

The static variant exists for callers that may not allocate device memory
while they run (for example an embedding whose device-memory budget is fixed
after start-up). It must give the same product as the allocating
entry point, call after call, since it reuses one static scratch array.
This file sorts last so that a stop-at-first-failure run has already run
every other test.
"""
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


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_static_apply_matches_operator_apply_on_consecutive_calls(aggmg, form):
    wl = W.jittered_square_2d(n=30, n_levels=3)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision=form)
    B = (wl.degree + 1) ** 2
    units = hier.stats()["units"]
    for level in range(hier.n_levels - 1):
        n = units[level] * B
        for call in range(2):
            x = torch.tensor(np.random.default_rng(100 * level + call).standard_normal(n),
                             dtype=torch.float64, device="cuda")
            y_ref = torch.empty(n, dtype=torch.float64, device="cuda")
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            hier.operator_apply(level, x, y_ref)
            hier.operator_apply_static(level, x, y)
            torch.cuda.synchronize()
            err = float((y - y_ref).abs().max() / y_ref.abs().max())
            assert err <= 1e-13, (form, level, call, err)
    hier.close()


def test_static_apply_rejects_levels_beyond_its_maximum(aggmg):
    # 352^2 Q2 elements: 1,115,136 fine DoFs > 2^20 entries of the static scratch
    wl = W.jittered_square_2d(n=352, n_levels=3)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    n = wl.n_dofs
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(aggmg.AggError) as e:
        hier.operator_apply_static(0, x, y)
    assert e.value.status == aggmg.AGG_EINVAL
    assert "at most" in str(e.value)
    # the coarser level fits and still works
    n1 = hier.stats()["units"][1] * 9
    x1 = torch.ones(n1, dtype=torch.float64, device="cuda")
    y1 = torch.empty(n1, dtype=torch.float64, device="cuda")
    y1r = torch.empty(n1, dtype=torch.float64, device="cuda")
    hier.operator_apply_static(1, x1, y1)
    hier.operator_apply(1, x1, y1r)
    torch.cuda.synchronize()
    assert torch.equal(y1, y1r)
    hier.close()


def test_static_apply_leaves_free_device_memory_unchanged(aggmg):
    """After the first call, repeated static products on every level leave the
    device's free memory (cudaMemGetInfo) exactly where it was."""
    wl = W.jittered_square_2d(n=30, n_levels=3)
    hier = aggmg.Hierarchy(aggmg.Mesh.from_workload(wl), 1.0 / wl.dt, wl.maps, precision="f64")
    B = (wl.degree + 1) ** 2
    units = hier.stats()["units"]
    bufs = []
    for level in range(hier.n_levels - 1):
        n = units[level] * B
        bufs.append((level, torch.ones(n, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.float64, device="cuda")))
    for level, x, y in bufs:
        hier.operator_apply_static(level, x, y)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        for level, x, y in bufs:
            hier.operator_apply_static(level, x, y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    hier.close()
