"""Host-side logic of the serving layer: lane planning and argument checks (no GPU needed)."""
import pytest

import paper_1202_6158_gb300 as di


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1202_6158_gb300 import build
    build.build()
    return di.load()


def test_no_budget_gives_64_lanes():
    assert di.di_plan_lanes([100, 1000, 5], [1, 2, 3], 0) == [64, 64, 64]
    assert di.di_plan_lanes([100], [0], -5) == [64]


def test_budget_halves_the_costliest_pool_first():
    # 64*100 + 64*1000 = 70400 > 22400: the second pool goes 64 -> 32 -> 16 (its lanes cost the most)
    assert di.di_plan_lanes([100, 1000], [0, 0], 64 * 100 + 16 * 1000) == [64, 16]
    # one byte less: the second pool, still the costliest, goes down to 8
    assert di.di_plan_lanes([100, 1000], [0, 0], 64 * 100 + 16 * 1000 - 1) == [64, 8]
    assert di.di_plan_lanes([100, 1000], [0, 0], 32 * 100 + 8 * 1000) == [32, 8]


def test_ties_halve_the_lowest_index_and_fixed_bytes_count():
    assert di.di_plan_lanes([10, 10], [0, 0], 32 * 10 + 64 * 10) == [32, 64]
    assert di.di_plan_lanes([10, 10], [100, 100], 64 * 20 + 200) == [64, 64]
    assert di.di_plan_lanes([10, 10], [100, 100], 64 * 20 + 199) == [32, 64]


def test_budget_too_small_is_enomem():
    with pytest.raises(di.DiError) as e:
        di.di_plan_lanes([10, 10], [0, 0], 8 * 20 - 1)
    assert e.value.status == di.DI_ENOMEM
    assert di.di_plan_lanes([10, 10], [0, 0], 8 * 20) == [8, 8]


def test_invalid_plans_and_servers():
    with pytest.raises(di.DiError):
        di.di_plan_lanes([-1], [0], 100)
    with pytest.raises(di.DiError):
        di.di_plan_lanes([], [], 100)
    with pytest.raises(di.DiError, match="at least one graph"):
        di.di_server_create([], 0)
    with pytest.raises(di.DiError, match="NULL"):
        di.di_server_create([None], 0)
    with pytest.raises(di.DiError, match="server is NULL"):
        di.di_server_submit(None, 0, [1], 1e-6)
    with pytest.raises(di.DiError, match="server is NULL"):
        di.di_server_poll(None)
    di.di_server_free(None)


def test_clock_is_monotonic():
    a = di.di_clock()
    b = di.di_clock()
    assert b >= a > 0
