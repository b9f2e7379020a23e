"""Host-side logic of the serving loop, on the CPU: memory admission (lazy
allocation under a budget, eviction of idle slots of other classes, refusal of
a class that can never fit) and the request trace."""
import math

import numpy as np
import pytest
import torch

import synth


class FakeScene:
    def __init__(self, n):
        self.n = n


@pytest.fixture(scope="module")
def serving():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_22159_gb300 import serving
    return serving


def test_pool_admission_eviction_and_refusal(serving):
    import paper_2503_22159_gb300 as d4
    cfg = d4.config_struct(16, 256)
    scenes = {"A": FakeScene(1000), "B": FakeScene(2000)}
    cam_s, cam_l = synth.pinhole(64, 64), synth.pinhole(256, 256)
    caps = {("A", 64, 64): 10_000, ("B", 256, 256): 200_000}
    pool = serving.WorkspacePool(cfg, scenes, caps, budget_bytes=0, device="cpu")
    need_s = pool._bytes(("A", 64, 64), cam_s)
    need_l = pool._bytes(("B", 256, 256), cam_l)
    pool.budget = 2 * need_s + need_l - 1          # room for two small slots, or one large + one small
    assert need_s < need_l
    a1 = pool.acquire(("A", 64, 64), cam_s)
    a2 = pool.acquire(("A", 64, 64), cam_s)
    assert a1 is not None and a2 is not None and a1 is not a2 and pool.used == 2 * need_s
    # both small slots busy: the large class does not fit beside them and nothing is idle to evict
    assert pool.acquire(("B", 256, 256), cam_l) is None and pool.used == 2 * need_s and pool.evicted == 0
    # one small slot idle again: it is evicted to admit the large one
    pool.release(a1)
    b = pool.acquire(("B", 256, 256), cam_l)
    assert b is not None and pool.evicted == 1 and pool.used <= pool.budget
    # a free slot of the same class is reused without allocating
    pool.release(b)
    used = pool.used
    assert pool.acquire(("B", 256, 256), cam_l) is b and pool.used == used
    with pytest.raises(MemoryError):
        serving.WorkspacePool(cfg, scenes, caps, need_l - 1, "cpu").acquire(("B", 256, 256), cam_l)


def test_trace_is_seeded_poisson(serving):
    scenes = {"A": FakeScene(10), "B": FakeScene(10)}
    r1 = serving.make_trace(scenes, n_requests=4000, rate_hz=500.0, seed=4)
    r2 = serving.make_trace(scenes, n_requests=4000, rate_hz=500.0, seed=4)
    assert [r.arrival for r in r1] == [r.arrival for r in r2]
    gaps = np.diff([0.0] + [r.arrival for r in r1])
    assert abs(gaps.mean() - 1 / 500.0) < 0.1 / 500.0        # exponential with mean 2 ms
    assert abs(np.median(gaps) / gaps.mean() - math.log(2)) < 0.06
    res = {r.res for r in r1}
    assert res == {(640, 480), (1352, 1014), (1920, 1080), (2704, 2028)}
    assert {r.scene for r in r1} == {"A", "B"}
    assert all(0.0 <= r.t <= 1.0 for r in r1)


def test_trace_at_another_rate_has_the_same_requests(serving):
    """The saturated replay offers the same requests faster: with the same seed, a different rate
    changes only the arrival times (all drawn first), by exactly the rate ratio."""
    scenes = {"A": FakeScene(10), "B": FakeScene(10)}
    slow = serving.make_trace(scenes, n_requests=500, rate_hz=500.0, seed=4)
    fast = serving.make_trace(scenes, n_requests=500, rate_hz=20000.0, seed=4)
    for a, b in zip(slow, fast):
        assert (a.scene, a.res, a.t) == (b.scene, b.res, b.t)
        assert np.array_equal(a.cam.R, b.cam.R) and np.array_equal(a.cam.T, b.cam.T)
        assert b.arrival == pytest.approx(a.arrival * 500.0 / 20000.0, rel=1e-9)
