"""Continuous-batching solve server on one GPU.

Requests (a mesh, an initial state, boundary data and a final time) arrive
over time. The server admits a waiting request as soon as its device memory
fits in the budget next to the requests already running, keeps every admitted
request's mesh and state resident in its own solver context on its own CUDA
stream, and advances all admitted requests together: each loop iteration
launches one SSPRK(3,3) step (one CUDA-graph launch) for every active request,
and the launches of different requests overlap on the device. Each request
stops on the device at its final time (the last step is shortened, see
eh_set_instances); the server retires it between iterations, frees its memory
and admits the next ones. Every step runs in the CUDA library; this module
only orchestrates.
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


def device_bytes(mesh, precision=binding.EH_PRECISION_FP64) -> int:
    """Device memory a context needs for this mesh (the arrays eh_upload_mesh
    allocates, rounded up)."""
    S, SP = mesh.dim + 2, (4 if mesh.dim == 2 else 6)
    per_entry = 4 + 4 + 8 * mesh.dim + 8 * 4 + 8 * SP * 2 + 8 * 3 + 8 + 5
    per_node = 8 * (24 + 8 * SP + 3 * S + 13)
    if precision == binding.EH_PRECISION_MIXED:
        per_entry += 4 * (mesh.dim + 2 + SP + 1)
        per_node += 4 * (24 + SP)
    return int(1.1 * (per_entry * mesh.nnz + per_node * mesh.n)) + (1 << 20)


class SolveServer:
    def __init__(self, hbm_budget_bytes: int, precision=binding.EH_PRECISION_FP64, device=0, poll_every=4,
                 lib=None):
        import torch  # streams only
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.precision = precision
        self.device = device
        self.poll_every = poll_every
        self.lib = lib or binding.load()

    def _start(self, req):
        stream = self.torch.cuda.Stream(device=self.device)
        s = binding.Solver(dim=req.mesh.dim, precision=self.precision, device=self.device,
                           stream=stream.cuda_stream, lib=self.lib)
        s.upload_mesh(req.mesh, req.bnd_state)
        s.set_instances([0, req.mesh.n], [req.t_final])
        s.set_state(req.U0)
        s.apply_boundary_conditions()
        return s, stream

    def run(self, requests, clock=time.perf_counter):
        """Serve the requests (sorted by arrival); returns the Results in
        completion order. Arrival times are honoured against ``clock``."""
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting, active, done = [], [], []
        used = 0
        t0 = clock()
        it = 0
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.pop(0))
            # admission by free device memory (first come, first served)
            while waiting:
                need = device_bytes(waiting[0].mesh, self.precision)
                if active and used + need > self.budget:
                    break
                req = waiting.pop(0)
                s, stream = self._start(req)
                active.append(dict(req=req, solver=s, stream=stream, need=need, admitted=clock() - t0, steps=0))
                used += need
            if not active:
                if pending:  # idle until the next arrival
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
            # one step for every active request; the launches overlap on the device
            for a in active:
                a["solver"].run(1)
                a["steps"] += 1
            it += 1
            if it % self.poll_every:
                continue
            still = []
            for a in active:
                info = a["solver"].instances()
                if info["t"][0] >= a["req"].t_final:
                    U = a["solver"].get_state()
                    done.append(Result(a["req"].name, a["req"].mesh.n, a["req"].arrival, a["admitted"],
                                       clock() - t0, a["steps"], float(info["t"][0]), U))
                    a["solver"].close()
                    used -= a["need"]
                else:
                    still.append(a)
            active = still
        return done


def solve_alone(req: Request, precision=binding.EH_PRECISION_FP64, device=0, lib=None):
    """The same solve in a context of its own (for the alone-vs-mix check and
    for the sequential baseline): SSPRK(3,3) steps until t_final."""
    s = binding.Solver(dim=req.mesh.dim, precision=precision, device=device, lib=lib)
    s.upload_mesh(req.mesh, req.bnd_state)
    s.set_instances([0, req.mesh.n], [req.t_final])
    s.set_state(req.U0)
    s.apply_boundary_conditions()
    steps = 0
    while True:
        s.run(4)
        steps += 4
        if s.instances()["t"][0] >= req.t_final:
            break
    U = s.get_state()
    s.close()
    return U, steps


def poisson_trace(count, rate, seed, n_range, t_final, mach_range=(1.5, 4.0)):
    """Seeded request trace: Poisson arrivals at ``rate`` per second, vertex
    counts log-uniform in n_range, P1 or Q1 (probability 1/2 each), inflow Mach
    uniform in mach_range, all to ``t_final``."""
    from . import meshes, workloads
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    arrivals -= arrivals[0]
    out = []
    for k in range(count):
        n_target = float(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))
        m = meshes.cylinder_m_for_vertices(int(n_target))
        p1 = bool(rng.uniform() < 0.5)
        mach = float(rng.uniform(*mach_range))
        mesh = meshes.cylinder_channel_p1(m) if p1 else meshes.cylinder_channel_q1(m)
        U0 = workloads.uniform_state(mesh, 1.4, (mach, 0.0), 1.0)
        out.append(Request(mesh, U0, np.ascontiguousarray(U0[:, mesh.bnd_node]), t_final, float(arrivals[k]),
                           f"req{k}-{'p1' if p1 else 'q1'}-m{m}-M{mach:.2f}"))
    return out
