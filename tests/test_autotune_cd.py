"""The coordinate-descent batch tuner (tune_batch) on a synthetic timing
landscape: a stand-in batch records the plan it is given and a stand-in
timer prices it, so the search logic runs without a GPU."""
import pytest

import paper_2002_12115_gb300.autotune as at
from paper_2002_12115_gb300 import JacError

DIMS = [(17, 33, 49), (129, 17, 17), (65, 65, 129), (17, 129, 65), (129, 33, 33)]
BEST_TI = {17: 16, 65: 64, 129: 128}
BEST_KD = {17: 8, 33: 16, 49: 16, 65: 32, 129: 64}


class StandInBatch:
    prec = "f32"

    def __init__(self, dims, refuse=None):
        self.dims = dims
        self.plan = None
        self.refuse = refuse or (lambda warps, ti, kd: False)
        self.measured = 0

    def set_plan(self, warps, tile_i, kdepth):
        if self.refuse(warps, tile_i, kdepth):
            raise JacError(1, "unsupported plan")
        self.plan = (warps, list(tile_i), list(kdepth))

    def sweep(self, n, residuals=True):
        pass


@pytest.fixture
def priced(monkeypatch):
    """time_call prices the stand-in batch's current plan: every tile width
    and depth away from the best one for its class costs time; 4 warps cost
    a constant more than 8."""
    state = {}

    def time_call(fn, reps=3, stream=None):
        b = state["batch"]
        b.measured += 1
        warps, ti, kd = b.plan
        cost = 1.0 + (0.5 if warps == 4 else 0.0)
        for (I, _, K), t, d in zip(b.dims, ti, kd):
            cost += abs(t - BEST_TI[I]) / 128 + abs(d - min(BEST_KD[K], K - 2)) / 64
        return cost

    monkeypatch.setattr(at, "time_call", time_call)
    monkeypatch.setattr(at, "_gpu_name", lambda: "stand-in")
    return state


def test_coordinate_descent_finds_each_class_optimum(priced):
    b = StandInBatch(DIMS)
    priced["batch"] = b
    plan = at.tune_batch(b, cache_path=None, passes=2)
    assert plan["warps"] == 8
    assert plan["tile_i"] == {str(I): BEST_TI[I] for I in (17, 65, 129)}
    for K in (17, 33, 49, 65, 129):
        assert plan["kdepth"][str(K)] == BEST_KD[K]
    # the batch is left on the plan found, with depths clipped to K - 2
    warps, ti, kd = b.plan
    assert warps == 8 and ti == [BEST_TI[I] for I, _, _ in DIMS]
    assert kd == [min(BEST_KD[K], K - 2) for _, _, K in DIMS]


def test_refused_plans_are_never_chosen(priced):
    """A plan the library refuses (JacError) counts as infinitely slow."""
    def refuse(warps, ti, kd):
        return any(t == 128 for t in ti)
    b = StandInBatch(DIMS, refuse)
    priced["batch"] = b
    plan = at.tune_batch(b, cache_path=None, passes=1)
    assert 128 not in plan["tile_i"].values()
    assert plan["tile_i"]["129"] == 64          # the next best width for I = 129


def test_cached_plan_is_reused_without_measuring(priced, tmp_path):
    cache = str(tmp_path / "cache.json")
    b = StandInBatch(DIMS)
    priced["batch"] = b
    first = at.tune_batch(b, cache_path=cache, passes=1)
    assert b.measured > 0
    b2 = StandInBatch(DIMS)
    priced["batch"] = b2
    second = at.tune_batch(b2, cache_path=cache, passes=1)
    assert b2.measured == 0 and second == first and b2.plan is not None
