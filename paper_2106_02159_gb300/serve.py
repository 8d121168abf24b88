"""Continuous-batching solve server on one GPU.

Requests (a mesh, an initial state, boundary data and a final time) arrive
over time. The server hands every arrived request to the library's batch
(eh_batch_admit), which admits it as soon as its device memory fits in the
budget next to the requests already running and keeps its mesh and state
resident on the device. In merged mode (the default) the running requests are
the instances of one batched context, so eh_batch_advance takes each SSPRK(3,3)
step of all of them with one set of kernel launches (one CUDA-graph replay);
requests that arrive or finish are merged in or taken out between advances. In
per-request-stream mode (the comparison) every request has a context and a
stream of its own and the advance launches one step of each in turn. Each
request stops on the device at its final time (the last step is shortened);
eh_batch_poll returns its state and frees its memory. Admission, stepping and
retirement run in the library; this module keeps the arrival clock and the
results.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import binding


@dataclasses.dataclass
class Request:
    """One flow solve. arrival: seconds after the server starts."""
    mesh: object
    U0: np.ndarray
    bnd_state: np.ndarray | None
    t_final: float
    arrival: float = 0.0
    name: str = ""


@dataclasses.dataclass
class Result:
    name: str
    n: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    t: float
    U: np.ndarray

    @property
    def time_to_solution(self) -> float:
        return self.finished - self.arrival


def device_bytes(mesh, precision=binding.EH_PRECISION_FP64, mode=binding.EH_BATCH_MERGED) -> int:
    """Device memory a batch in ``mode`` counts for this mesh at admission
    (eh_estimate_request_bytes)."""
    return binding.estimate_request_bytes(mesh.dim, precision, mode, mesh.n, mesh.nnz, mesh.n_bnd)


class SolveServer:
    def __init__(self, hbm_budget_bytes: int, precision=binding.EH_PRECISION_FP64, device=0, poll_every=4,
                 mode=binding.EH_BATCH_MERGED, lib=None):
        self.budget = int(hbm_budget_bytes)
        self.precision = precision
        self.mode = mode
        self.device = device
        self.poll_every = poll_every
        self.lib = lib or binding.load()

    def run(self, requests, clock=time.perf_counter):
        """Serve the requests (sorted by arrival); returns the Results in
        completion order. Arrival times are honoured against ``clock``."""
        pending = sorted(requests, key=lambda r: r.arrival)
        if not pending:
            return []
        dims = {r.mesh.dim for r in pending}
        assert len(dims) == 1, "one batch serves one dimension"
        batch = binding.Batch(self.budget, dim=dims.pop(), device=self.device, precision=self.precision,
                              mode=self.mode, lib=self.lib)
        waiting, active, done = [], {}, []
        t0 = clock()
        try:
            while pending or waiting or active:
                now = clock() - t0
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.pop(0))
                # admission by free device memory (first come, first served)
                while waiting:
                    ticket = batch.admit(waiting[0].mesh, waiting[0].U0, waiting[0].t_final, waiting[0].bnd_state)
                    if ticket is None:
                        break
                    active[ticket] = (waiting.pop(0), clock() - t0)
                if not active:
                    if pending:  # idle until the next arrival
                        time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                    continue
                if batch.advance(self.poll_every) == 0:
                    continue
                for ticket in list(active):
                    out = batch.poll(ticket)
                    if out is None:
                        continue
                    U, t, steps = out
                    req, admitted = active.pop(ticket)
                    done.append(Result(req.name, req.mesh.n, req.arrival, admitted, clock() - t0, steps, t, U))
        finally:
            batch.close()
        return done


def solve_alone(req: Request, precision=binding.EH_PRECISION_FP64, device=0, lib=None):
    """The same solve in a context of its own (for the alone-vs-mix check and
    for the sequential baseline): SSPRK(3,3) steps until t_final."""
    s = binding.Solver(dim=req.mesh.dim, precision=precision, device=device, lib=lib)
    s.upload_mesh(req.mesh, req.bnd_state)
    s.set_instances([0, req.mesh.n], [req.t_final])
    s.set_state(req.U0)
    s.apply_boundary_conditions()
    while True:
        s.run(4)
        inst = s.instances()
        if inst["t"][0] >= req.t_final:
            break
    U = s.get_state()
    s.close()
    return U, int(inst["steps"][0])


def _build_mesh(args):
    """(m, p1) -> the P1 or Q1 cylinder channel of size m (a worker task)."""
    from . import meshes
    m, p1 = args
    return meshes.cylinder_channel_p1(m) if p1 else meshes.cylinder_channel_q1(m)


def poisson_trace(count, rate, seed, n_range, t_final, mach_range=(1.5, 4.0), size_grid=0, workers=0):
    """Seeded request trace: Poisson arrivals at ``rate`` per second, vertex
    counts log-uniform in n_range, P1 or Q1 (probability 1/2 each), inflow Mach
    uniform in mach_range, all to ``t_final``. size_grid > 0 snaps each drawn
    vertex count to the nearest of that many log-spaced sizes spanning n_range
    (so that meshes repeat and are built once); workers > 0 builds the distinct
    meshes in that many processes (spawned: safe after CUDA is initialised; the
    spawned workers import the caller's main module, so a script that calls
    this with workers > 0 must do so under ``if __name__ == "__main__":``).
    Inside a worker process, or when the workers cannot start, the meshes are
    built in the calling process."""
    from . import meshes, workloads
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    arrivals -= arrivals[0]
    grid = np.exp(np.linspace(np.log(n_range[0]), np.log(n_range[1]), size_grid)) if size_grid > 0 else None
    specs = []
    for k in range(count):
        n_target = float(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        if grid is not None:
            n_target = float(grid[np.argmin(np.abs(np.log(grid) - np.log(n_target)))])
        m = meshes.cylinder_m_for_vertices(int(n_target))
        p1 = bool(rng.uniform() < 0.5)
        mach = float(rng.uniform(*mach_range))
        specs.append((m, p1, mach))
    keys = sorted({(m, p1) for m, p1, _ in specs}, key=lambda t: -t[0])
    import multiprocessing as mp
    built = None
    if workers > 0 and len(keys) > 1 and mp.parent_process() is None:
        from concurrent.futures import ProcessPoolExecutor
        from concurrent.futures.process import BrokenProcessPool
        try:
            with ProcessPoolExecutor(min(workers, len(keys)), mp_context=mp.get_context("spawn")) as ex:
                built = dict(zip(keys, ex.map(_build_mesh, keys)))
        except BrokenProcessPool:  # a worker could not start (say, a main module that cannot be imported)
            built = None
    if built is None:
        built = {key: _build_mesh(key) for key in keys}
    out = []
    for k, (m, p1, mach) in enumerate(specs):
        mesh = built[(m, p1)]
        U0 = workloads.uniform_state(mesh, 1.4, (mach, 0.0), 1.0)
        out.append(Request(mesh, U0, np.ascontiguousarray(U0[:, mesh.bnd_node]), t_final, float(arrivals[k]),
                           f"req{k}-{'p1' if p1 else 'q1'}-m{m}-M{mach:.2f}"))
    return out
