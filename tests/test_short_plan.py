"""Host planning of the short-axis kernel (no GPU): which axes each pass over
the state transforms, the CTA size and the shared memory, queried through
the C-ABI (mg_short_axis_plan)."""
import pytest

SMEM_CAP = 227 * 1024


@pytest.fixture(scope="module")
def capi():
    import os

    from paper_1909_06412_gb300 import _build, capi as c

    if not os.path.exists(c.LIB_PATH):
        _build.build()
    return c


def test_groups_of_the_eight_dimensional_workloads(capi):
    # 16^8 FP32: four groups, so a TVT stage makes 8 passes over the 34 GB state
    p = capi.mg_short_axis_plan((16,) * 8, capi.MG_FP32_MIXED)
    assert p["groups"] == [(5, 3), (3, 2), (1, 2), (0, 1)] and p["threads"] == 256
    # 12^8 FP64: three groups; two 288-line chunks per set on 12 warps
    p = capi.mg_short_axis_plan((12,) * 8, capi.MG_FP64)
    assert p["groups"] == [(5, 3), (2, 3), (0, 2)] and p["threads"] == 384
    # the 7D profiling cases
    assert capi.mg_short_axis_plan((16,) * 7, capi.MG_FP32_MIXED)["groups"] == [(4, 3), (2, 2), (0, 2)]
    assert capi.mg_short_axis_plan((12,) * 7, capi.MG_FP64)["groups"] == [(4, 3), (1, 3), (0, 1)]


@pytest.mark.parametrize("n", [8, 12, 16])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("D", [3, 4, 5, 6, 7, 8])
def test_every_plan_partitions_the_axes(capi, n, prec, D):
    p = capi.mg_short_axis_plan((n,) * D, prec)
    assert p is not None
    # consecutive runs from the back: group 0 ends at the last axis, each next
    # group ends where the previous one starts, the last starts at axis 0
    end = D
    for first, nax in p["groups"]:
        assert 1 <= nax <= 4 and first + nax == end
        end = first
    assert end == 0
    assert 0 < p["smem_bytes"] <= SMEM_CAP
    expect = 256 if n != 12 else (384 if prec == 0 else 288)
    assert p["threads"] == expect


def test_grids_the_short_kernel_does_not_take(capi):
    assert capi.mg_short_axis_plan((256, 256)) is None       # D < 3
    assert capi.mg_short_axis_plan((16, 16, 12)) is None     # mixed lengths
    assert capi.mg_short_axis_plan((32, 32, 32)) is None     # axes longer than 16
    with pytest.raises(capi.MgError):
        capi.mg_short_axis_plan((10, 10, 10))                # factor 5
