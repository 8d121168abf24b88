"""The continuous-batching solve server, in both batch modes (merged: the
running requests are the instances of one batched context, repacked as they
come and go; per-request streams): requests that arrive while others run are
admitted as memory allows, run concurrently, stop at their own final time,
and each result is the same (bitwise) as the request solved alone. Needs a GPU."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import serve

pytestmark = pytest.mark.gpu


MODES = [B.EH_BATCH_MERGED, B.EH_BATCH_PER_REQUEST_STREAMS]


@pytest.mark.parametrize("mode", MODES)
def test_served_results_equal_solves_alone(mode):
    B.build()
    reqs = serve.poisson_trace(6, rate=200.0, seed=5, n_range=(800, 6000), t_final=0.03)
    budget = sum(sorted(serve.device_bytes(r.mesh, mode=mode) for r in reqs)[-3:])  # ~3 requests at a time
    results = serve.SolveServer(budget, poll_every=2, mode=mode).run(reqs)
    assert len(results) == len(reqs)
    by_name = {r.name: r for r in results}
    for req in reqs:
        res = by_name[req.name]
        assert res.t == req.t_final
        assert res.admitted >= req.arrival - 1e-9 and res.finished >= res.admitted
        U, steps = serve.solve_alone(req)
        assert np.array_equal(res.U, U), req.name
        assert res.steps == steps, (req.name, res.steps, steps)


@pytest.mark.parametrize("mode", MODES)
def test_admission_respects_the_memory_budget(mode):
    reqs = serve.poisson_trace(5, rate=1e6, seed=6, n_range=(1500, 2500), t_final=0.01)
    need = max(serve.device_bytes(r.mesh, mode=mode) for r in reqs)
    srv = serve.SolveServer(need, poll_every=1, mode=mode)  # one request at a time
    results = srv.run(reqs)
    spans = sorted((r.admitted, r.finished) for r in results)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-9  # never two at once


@pytest.mark.parametrize("mode", MODES)
def test_batch_api_budget_tickets_and_results(mode):
    # the C batch directly: a second request does not fit a one-request budget
    # until the first has been polled; unknown tickets are refused; the
    # result equals the solve alone
    reqs = serve.poisson_trace(2, rate=1e6, seed=7, n_range=(1500, 2500), t_final=0.01)
    need = max(serve.device_bytes(r.mesh, mode=mode) for r in reqs)
    b = B.Batch(need, mode=mode)
    t0 = b.admit(reqs[0].mesh, reqs[0].U0, reqs[0].t_final, reqs[0].bnd_state)
    assert t0 is not None
    assert b.admit(reqs[1].mesh, reqs[1].U0, reqs[1].t_final, reqs[1].bnd_state) is None
    assert b.active() == (1, serve.device_bytes(reqs[0].mesh, mode=mode))
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


def test_merged_batch_repacks_as_requests_come_and_go():
    """Merged mode: requests admitted between advances join the one batched
    context, finished ones leave it; every result equals its solve alone, and
    a request larger than the whole budget is refused outright."""
    reqs = serve.poisson_trace(5, rate=1e6, seed=8, n_range=(900, 4000), t_final=0.02)
    b = B.Batch(1 << 32)
    tickets = [b.admit(reqs[0].mesh, reqs[0].U0, reqs[0].t_final, reqs[0].bnd_state)]
    b.advance(2)
    for r in reqs[1:3]:  # join a running batch
        tickets.append(b.admit(r.mesh, r.U0, r.t_final, r.bnd_state))
    results = {}
    k = 3
    while len(results) < len(reqs):
        b.advance(3)
        for t in list(tickets):
            out = b.poll(t)
            if out is not None:
                results[t] = out
                tickets.remove(t)
                if k < len(reqs):  # a freed slot is filled at once
                    tickets.append(b.admit(reqs[k].mesh, reqs[k].U0, reqs[k].t_final, reqs[k].bnd_state))
                    k += 1
    assert b.repacks() >= 4
    b.close()
    for (ticket, (U, t, steps)), req in zip(sorted(results.items()), reqs):
        Ua, steps_a = serve.solve_alone(req)
        assert t == req.t_final and steps == steps_a
        assert np.array_equal(U, Ua), req.name
    tiny = B.Batch(1 << 20)
    with pytest.raises(B.EulerError) as e:
        tiny.admit(reqs[0].mesh, reqs[0].U0, reqs[0].t_final, reqs[0].bnd_state)
    assert e.value.status == B.EH_ERR_INVALID_ARG
    tiny.close()


def _alone_requests(kind):
    from paper_2106_02159_gb300 import meshes as M
    from paper_2106_02159_gb300 import workloads as W
    out = []
    if kind == "3d":
        for k, (nx, ny, nz) in enumerate(((6, 5, 4), (8, 4, 5))):
            mesh = M.structured_q1_3d(nx, ny, nz, periodic=(False, False, True))
            U0 = W.perturbed_state(mesh, 20 + k, base=dict(rho=1.0, vel=(0.4, 0.1, 0.0), p=1.0), amplitude=0.2)
            out.append(serve.Request(mesh, U0, None, 0.02 + 0.01 * k, 0.0, f"box3d-{k}"))
    elif kind == "nonreflecting":
        for k, (case, bc) in enumerate((("i", M.BC_GODUNOV), ("ii", M.BC_CHARACTERISTIC))):
            mesh, U0, bs = W.nrbc_vortex_problem(16 + 4 * k, case, bc)
            out.append(serve.Request(mesh, U0, bs, 0.05 + 0.03 * k, 0.0, f"nrbc-{case}"))
    else:
        out = serve.poisson_trace(3, rate=1e6, seed=9, n_range=(900, 4000), t_final=0.02)
    return out


@pytest.mark.parametrize("kind", ["mixed", "3d", "nonreflecting"])
def test_merged_batch_other_configurations(kind):
    """The merged batch's union assembly with mixed precision, 3D requests
    (27-entry rows) and the non-reflecting boundary kinds (boundary states,
    normals and indices placed at offsets): every result equals its solve
    alone bit for bit, with the same step count."""
    B.build()
    reqs = _alone_requests(kind)
    dim = reqs[0].mesh.dim
    precision = B.EH_PRECISION_MIXED if kind == "mixed" else B.EH_PRECISION_FP64
    b = B.Batch(1 << 32, dim=dim, precision=precision)
    tickets = [b.admit(r.mesh, r.U0, r.t_final, r.bnd_state) for r in reqs]
    results = {}
    while len(results) < len(reqs):
        b.advance(3)
        for t in tickets:
            if t not in results:
                out = b.poll(t)
                if out is not None:
                    results[t] = out
    b.close()
    for t, req in zip(tickets, reqs):
        U, tt, steps = results[t]
        Ua, steps_a = serve.solve_alone(req, precision)
        assert tt == req.t_final and steps == steps_a, (req.name, steps, steps_a)
        assert np.array_equal(U, Ua), req.name
