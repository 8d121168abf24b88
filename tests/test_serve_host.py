"""Host logic of the solve server (serve.SolveServer) around the library's
batch, with the batch replaced by a fake that keeps the same contract
(admission against a memory budget, steps, polling): every request is
served once, first come first served, the budget is never exceeded and a
request is never admitted before it arrives. CPU only."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding, serve


class _Mesh:
    dim = 2

    def __init__(self, n):
        self.n = n


class FakeBatch:
    """Admits while the bytes fit (the first request always); a request
    finishes after a number of steps proportional to its size."""
    log = []

    def __init__(self, budget, dim=2, device=0, precision=0, mode=0, lib=None):
        self.budget, self.used, self.next, self.running = budget, 0, 1, {}
        FakeBatch.log = []

    def admit(self, mesh, U0, t_final, bnd_state=None):
        need = mesh.n
        if self.running and self.used + need > self.budget:
            return None
        ticket, self.next = self.next, self.next + 1
        self.running[ticket] = dict(n=mesh.n, left=max(1, mesh.n // 100), t_final=t_final, steps=0)
        self.used += need
        FakeBatch.log.append(("admit", ticket, self.used, mesh.n))
        assert self.used <= self.budget or len(self.running) == 1
        return ticket

    def advance(self, steps=1):
        for r in self.running.values():
            take = min(steps, r["left"])
            r["left"] -= take
            r["steps"] += take
        return sum(1 for r in self.running.values() if r["left"] == 0)

    def poll(self, ticket):
        r = self.running[ticket]
        if r["left"]:
            return None
        del self.running[ticket]
        self.used -= r["n"]
        FakeBatch.log.append(("done", ticket, self.used, r["n"]))
        return np.full((4, r["n"]), float(ticket)), r["t_final"], r["steps"]

    def close(self):
        pass


@pytest.fixture
def fake_batch(monkeypatch):
    monkeypatch.setattr(binding, "Batch", FakeBatch)
    return FakeBatch


def _requests(sizes, arrivals):
    return [serve.Request(_Mesh(n), None, None, 0.5, a, f"r{k}") for k, (n, a) in enumerate(zip(sizes, arrivals))]


def test_every_request_is_served_once_within_the_budget(fake_batch):
    sizes = [300, 800, 200, 500, 700, 100, 400]
    reqs = _requests(sizes, [0.0] * len(sizes))
    srv = serve.SolveServer(1000, poll_every=2, lib=object())
    results = srv.run(reqs)
    assert sorted(r.name for r in results) == sorted(r.name for r in reqs)
    assert all(r.t == 0.5 and r.U.shape == (4, r.n) for r in results)
    assert all(used <= 1000 for _, _, used, _ in fake_batch.log)
    # first come, first served: admitted in arrival order, and a request that
    # does not fit holds back the ones behind it
    assert [n for kind, _, _, n in fake_batch.log if kind == "admit"] == sizes


def test_requests_wait_for_their_arrival(fake_batch):
    reqs = _requests([200, 200, 200], [0.0, 0.05, 0.1])
    ticks = iter(np.arange(0.0, 100.0, 0.004))
    results = serve.SolveServer(10_000, poll_every=1, lib=object()).run(reqs, clock=lambda: next(ticks))
    assert len(results) == 3
    for r in results:
        assert r.admitted >= r.arrival and r.finished >= r.admitted


def test_empty_trace():
    assert serve.SolveServer(1, lib=object()).run([]) == []


def test_trace_meshes_built_in_worker_processes_equal_serial():
    """poisson_trace with workers > 0 builds the distinct meshes in spawned
    processes; the trace equals the one built in this process."""
    kw = dict(count=6, rate=1e3, seed=3, n_range=(800, 3000), t_final=0.01, size_grid=3)
    a = serve.poisson_trace(**kw, workers=0)
    b = serve.poisson_trace(**kw, workers=2)
    assert [r.name for r in a] == [r.name for r in b]
    for x, y in zip(a, b):
        assert x.arrival == y.arrival and x.t_final == y.t_final
        assert np.array_equal(x.mesh.row_ptr, y.mesh.row_ptr) and np.array_equal(x.mesh.col, y.mesh.col)
        assert np.array_equal(x.mesh.cij, y.mesh.cij) and np.array_equal(x.U0, y.U0)
