"""The continuous-batching solve server: requests that arrive while others run
are admitted as memory allows, run concurrently, stop at their own final time,
and each result is the same (bitwise) as the request solved alone. Needs a GPU."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import serve

pytestmark = pytest.mark.gpu


def test_served_results_equal_solves_alone():
    B.build()
    reqs = serve.poisson_trace(6, rate=200.0, seed=5, n_range=(800, 6000), t_final=0.03)
    budget = sum(sorted(serve.device_bytes(r.mesh) for r in reqs)[-3:])  # ~3 requests at a time
    results = serve.SolveServer(budget, poll_every=2).run(reqs)
    assert len(results) == len(reqs)
    by_name = {r.name: r for r in results}
    for req in reqs:
        res = by_name[req.name]
        assert res.t == req.t_final
        assert res.admitted >= req.arrival - 1e-9 and res.finished >= res.admitted
        U, _ = serve.solve_alone(req)
        assert np.array_equal(res.U, U), req.name


def test_admission_respects_the_memory_budget():
    reqs = serve.poisson_trace(5, rate=1e6, seed=6, n_range=(1500, 2500), t_final=0.01)
    need = max(serve.device_bytes(r.mesh) for r in reqs)
    srv = serve.SolveServer(need, poll_every=1)  # one request at a time
    results = srv.run(reqs)
    spans = sorted((r.admitted, r.finished) for r in results)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-9  # never two at once


def test_batch_api_budget_tickets_and_results():
    # the C batch directly: a second request does not fit a one-request budget
    # until the first has been polled; unknown tickets are refused; the
    # result equals the solve alone
    reqs = serve.poisson_trace(2, rate=1e6, seed=7, n_range=(1500, 2500), t_final=0.01)
    need = max(serve.device_bytes(r.mesh) for r in reqs)
    b = B.Batch(need)
    t0 = b.admit(reqs[0].mesh, reqs[0].U0, reqs[0].t_final, reqs[0].bnd_state)
    assert t0 is not None
    assert b.admit(reqs[1].mesh, reqs[1].U0, reqs[1].t_final, reqs[1].bnd_state) is None
    assert b.active() == (1, serve.device_bytes(reqs[0].mesh))
    with pytest.raises(B.EulerError):
        b.poll(t0 + 100)
    assert b.poll(t0) is None  # still running
    while b.advance(3) == 0:
        pass
    U, t, steps = b.poll(t0)
    assert t == reqs[0].t_final and steps > 0
    assert np.array_equal(U, serve.solve_alone(reqs[0])[0])
    assert b.active() == (0, 0)
    assert b.admit(reqs[1].mesh, reqs[1].U0, reqs[1].t_final, reqs[1].bnd_state) is not None
    b.close()
