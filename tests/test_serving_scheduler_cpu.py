"""Host-only tests of the shot server's admission and batching (ShotServer._take and
ShotServer._admit), with fake meshes whose device footprint is given; no GPU and no library
calls."""
import collections
import threading

import numpy as np
import pytest

from paper_2108_10946_gb300.serving import Request, ShotServer


class FakeMesh:
    def __init__(self, per_shot, fixed=0):
        self.per_shot, self.fixed = per_shot, fixed

    def batch_bytes(self, S, R):
        return self.fixed + self.per_shot * S


class FakeBatch:
    def __init__(self):
        self.closed = False

    def close(self):
        self.closed = True


def server(meshes, budget, max_batch, rolling=False):
    srv = ShotServer.__new__(ShotServer)  # the scheduler alone: no worker threads
    srv.meshes = {k: (m, np.zeros((1, 2))) for k, m in meshes.items()}
    srv.budget, srv.used, srv.max_batch = budget, 0, max_batch
    srv.rolling, srv.segment, srv.idle = rolling, None, 0
    srv.rolling_free = collections.Counter()
    srv.pending = collections.OrderedDict((k, collections.deque()) for k in meshes)
    srv.cv = threading.Condition()
    srv.pool, srv.nbytes, srv.completed = {}, {}, []
    return srv


def req(i, mesh, t, observed=False):
    return Request(i, mesh, [0.0, 0.0], np.zeros(4), observed=np.zeros((5, 1)) if observed else None,
                   arrival=t)


def test_largest_fitting_size_is_admitted():
    srv = server({"a": FakeMesh(100)}, budget=250, max_batch=4)
    for i in range(6):
        srv.pending["a"].append(req(i, "a", float(i)))
    kind, name, key, batch, reqs, _ = srv._take()
    assert (kind, name, key, batch) == ("batch", "a", ("a", 2), None) and [r.rid for r in reqs] == [0, 1]
    assert srv.used == 200
    # nothing else fits until a batch comes back
    assert srv._take() is None
    srv.pool[key] = [FakeBatch()]
    kind, name, key, batch, reqs, _ = srv._take()
    assert key[1] == 2 and batch is not None and [r.rid for r in reqs] == [2, 3]
    assert srv.used == 200


def test_one_shot_batch_when_only_that_fits():
    srv = server({"a": FakeMesh(100)}, budget=150, max_batch=4)
    for i in range(3):
        srv.pending["a"].append(req(i, "a", float(i)))
    _, _, key, _, reqs, _ = srv._take()
    assert key[1] == 1 and len(reqs) == 1 and srv.used == 100


def test_idle_batches_of_other_meshes_are_evicted():
    srv = server({"a": FakeMesh(100), "b": FakeMesh(100)}, budget=250, max_batch=2)
    idle = FakeBatch()
    srv.pool[("b", 2)] = [idle]
    srv.nbytes[("b", 2)] = 200
    srv.used = 200
    srv.pending["a"].append(req(0, "a", 0.0))
    srv.pending["a"].append(req(1, "a", 1.0))
    _, _, key, batch, reqs, _ = srv._take()
    assert idle.closed and key[1] == 2 and batch is None and srv.used == 200


def test_gradient_requests_share_a_batch_and_forward_requests_roll():
    """Gradient requests of one mesh pack into one batch (each lane returns its own
    gradient); a forward request starts a rolling batch of its mesh sized by the forward
    demand, after which as many of that mesh's forward requests as the batch has free lanes
    wait for its segment boundaries instead of new jobs."""
    srv = server({"a": FakeMesh(1), "b": FakeMesh(1)}, budget=1000, max_batch=4, rolling=True)
    srv.pending["a"].append(req(0, "a", 5.0))
    srv.pending["b"].append(req(1, "b", 1.0, observed=True))
    srv.pending["b"].append(req(2, "b", 2.0, observed=True))
    srv.pending["b"].append(req(3, "b", 3.0))
    srv.pending["b"].append(req(4, "b", 4.0, observed=True))
    srv.pending["b"].append(req(5, "b", 6.0))
    kind, name, key, _, reqs, _ = srv._take()
    assert (kind, name, key) == ("batch", "b", ("b", 4)) and [r.rid for r in reqs] == [1, 2, 4]
    assert [r.rid for r in srv.pending["b"]] == [3, 5]
    kind, name, key, _, reqs, src = srv._take()
    assert (kind, name, key, reqs) == ("roll", "b", ("b", 2), []) and srv.rolling_free["b"] == 2
    kind, name, key, _, _, _ = srv._take()
    assert (kind, name, key) == ("roll", "a", ("a", 1))
    assert srv._take() is None  # b's forward requests wait for its rolling batch
    assert [r.rid for r in srv._admit("b", 2)] == [3, 5]
    # a third forward request of b beyond the free lanes starts another rolling batch
    srv.rolling_free["b"] = 0
    srv.pending["b"].append(req(6, "b", 7.0))
    kind, name, key, _, _, _ = srv._take()
    assert (kind, name, key) == ("roll", "b", ("b", 1))


def test_rolling_admission_yields_to_older_requests_of_other_meshes():
    srv = server({"a": FakeMesh(1), "b": FakeMesh(1)}, budget=1000, max_batch=4, rolling=True)
    srv.rolling_free["a"] = 4
    srv.pending["a"].append(req(0, "a", 1.0))
    srv.pending["b"].append(req(1, "b", 2.0, observed=True))
    srv.pending["a"].append(req(2, "a", 3.0, observed=True))
    srv.pending["a"].append(req(3, "a", 4.0))
    # request 0 is the oldest: admitted; request 3 is younger than b's request 1 and no
    # worker is idle, so the rolling batch stops admitting (and drains)
    assert [r.rid for r in srv._admit("a", 4)] == [0]
    assert [r.rid for r in srv.pending["a"]] == [2, 3]
    srv.idle = 1  # an idle worker will serve b: the rolling batch may go on
    assert [r.rid for r in srv._admit("a", 4)] == [3]
    assert [r.rid for r in srv.pending["a"]] == [2]


def test_request_that_can_never_fit_is_reported():
    srv = server({"a": FakeMesh(100)}, budget=50, max_batch=2)
    r = req(0, "a", 0.0)
    srv.pending["a"].append(r)
    assert srv._take() is None
    assert r.event.is_set() and isinstance(r.error, MemoryError)
    assert not srv.pending["a"]


@pytest.mark.parametrize("budget", [100, 199, 400, 1000])
def test_used_never_exceeds_budget(budget):
    rng = np.random.default_rng(budget)
    srv = server({"a": FakeMesh(60, 40), "b": FakeMesh(30, 10)}, budget=budget, max_batch=8)
    running = []
    t = 0.0
    for _ in range(200):
        for _ in range(rng.integers(0, 4)):
            t += 1
            name = "a" if rng.random() < 0.5 else "b"
            srv.pending[name].append(req(int(t), name, t))
        job = srv._take()
        assert srv.used <= budget
        if job is not None:
            running.append(job)
        if running and rng.random() < 0.6:
            kind, name, key, batch, reqs, _ = running.pop(rng.integers(len(running)))
            srv.pool.setdefault(key, []).append(batch or FakeBatch())
