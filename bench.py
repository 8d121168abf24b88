#!/usr/bin/env python
"""Benchmark of the hyperbolic (Euler) step: DOF-updates per second per RK stage.

Workload (default): Mach-3 flow past a cylinder, Q1 quadrilaterals, channel
[0,4]x[0,1] minus the disc r = 0.25 at (0.6, 0.5), ~4.0M vertices, inflow
rho = 1.4, u = (3, 0), p = 1, slip walls, do-nothing outflow, SSPRK(3,3) at
CFL 0.5, FP64, strict local bounds. One "step" is one SSPRK(3,3) step = three
forward-Euler stages (all kernels of the hot path).

value   : vertices x 3 stages x steps x ranks / max-over-ranks device time of
          the timed steps (CUDA events on the solver's stream, inputs resident).
e2e     : the same metric through the C ABI with host buffers: every step
          copies the state from pinned host memory in (eh_set_state) and back
          out (eh_get_state), inside the timed region.
roofline: the kernel with the largest share of the step time (CUDA events
          around each kernel on the solver's stream): its FP64 operations,
          counted once from the method's formulas (method_fp64_flops), over
          its mean duration against the FP64 peak (the path is bound by FP64
          issue on GB300); beside it the HBM fraction by the planned
          schedule's per-unit bytes (survey_bytes) and the whole step's
          minimum-bytes fraction (survey_min_bytes_per_stage).
developed_flow: the same mesh from a seeded perturbed state (no identical-
          state edge, so no kernel takes the exact identical-state shortcut):
          time per step and the same roofline -- the FP64 fraction of the
          kernels doing all of their work.
cpu_baseline : the FP64 oracle on the host cores (all threads, and one
          thread), on a window of the same mesh, from the inflow state.

--impl reference runs the oracle (the CPU reference of this repository) for
the same workload and metric. Multi-GPU (torchrun): independent replicas, one
per GPU, no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage"
UNIT = "DOF-updates/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("cylinder", "vortex", "batch", "serve", "cylinder3d", "nrbc", "adaptive",
                                           "ns"),
                    default="cylinder")
    ap.add_argument("--requests", type=int, default=128, help="serve workload: requests in the trace")
    ap.add_argument("--serve-t-final", type=float, default=0.005, help="serve workload: t_final of every request")
    ap.add_argument("--serve-max-vertices", type=float, default=4e6,
                    help="serve workload: largest vertex count of the trace")
    ap.add_argument("--instances", type=int, default=256, help="batch workload: number of instances")
    ap.add_argument("--batch-small", action="store_true", help="batch workload: 32x8 to 64x16-cell instances only")
    ap.add_argument("--start3d", type=int, default=100,
                    help="cylinder3d workload: untimed steps from the inflow state before the warm-up")
    ap.add_argument("--vertices", type=int, default=4_000_000)
    ap.add_argument("--start-step", type=int, default=1000,
                    help="cylinder workload: untimed steps from the inflow state before the warm-up, so that the "
                         "timed steps sit in the middle of the 2000-step run (0: time from the inflow state)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-seconds-single", type=float, default=10.0,
                    help="seconds of the single-thread oracle leg of cpu_baseline (0: skip)")
    ap.add_argument("--repeats", type=int, default=4, help="repeats of the K timed steps (median of 1 + repeats)")
    ap.add_argument("--no-perturbed", action="store_true",
                    help="skip the measurement on the perturbed state of the same mesh")
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="fp64",
                    help="fp64: everything in FP64; mixed: FP32 c_ij, lambda_max, d_ij, high-order fluxes")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group(backend="nccl" if self._cuda() else "gloo")
            self.pg = td

    @staticmethod
    def _cuda():
        import torch
        return torch.cuda.is_available()

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if self._cuda() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows if len(r) >= 9 for q in range(4)
                          if r[5 + q].strip().lower() in ("active", "1")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": reasons}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(args):
    from paper_2106_02159_gb300 import meshes, workloads
    if args.workload == "vortex":
        w = workloads.vortex_workload(64)
        desc = "2D isentropic vortex, P1 64x64-vertex periodic mesh of [-5,5]^2, CFL 0.5, FP64"
    else:
        m = meshes.cylinder_m_for_vertices(args.vertices)
        mesh, U0, bs = workloads.cylinder_problem(m)
        w = workloads.Workload(f"cylinder-q1-m{m}", mesh, U0, bs, 2000)
        prec = "FP64" if args.precision == "fp64" else "mixed FP32/FP64"
        desc = ("2D Mach-3 cylinder channel, Q1, ring-graded O-grid + Cartesian blocks, "
                f"{mesh.n} vertices, CFL 0.5, {prec}, strict local bounds")
    return w, desc


def survey_bytes(kernel: str, n: int, nnz: int, dim: int) -> float:
    """Algorithmic HBM bytes of one launch by the per-unit figures of the
    method's planned schedule (the scope table's measurement section): the
    viscosity and low-order passes each read col + c_ij and write or read d_ij
    (12 + 8 dim B per entry), the first limiter pass reads col, m_ij, d_ij and
    writes l (28 B), the symmetrising pass and the final pass read col, m_ij,
    d_ij, l, the transpose index and l_ji (48 B); per node, every state-sized
    vector (S = dim + 2 doubles) the pass reads or writes, once."""
    S = dim + 2
    v = 8 * S
    per_entry, per_node = {
        "prep": (0, 2 * v),
        "visc": (12 + 8 * dim, v),
        "low": (12 + 8 * dim, v + 2 * v + 24),  # U read; U^L, F^H written; bounds
        "lim1": (28, 2 * v + 24),               # U^L, F^H read; bounds read
        "pass": (48, 2 * v),
        "final": (48, 3 * v),                   # limited state and U0 read, result written
        "tau": (0, 0),
        "lsearch": (0, 0),
    }[kernel]
    return per_entry * nnz + per_node * n


def survey_min_bytes_per_stage(n: int, nnz: int, dim: int) -> float:
    """The minimum the method must move per forward-Euler stage: static edge
    data read once (c_ij 8 dim + m_ij 8 + col 4 B per entry), the state read and
    written once (2 x 8 S per node), m_i (8) and row_ptr (4) per node (C2:
    328 B per node, C3: 1064)."""
    S = dim + 2
    return (8 * dim + 8 + 4) * nnz + (2 * 8 * S + 8 + 4) * n


def method_fp64_flops(kernel: str, n: int, nnz: int, dim: int) -> float:
    """FP64 operations of one launch counted ONCE from the method's formulas
    (Algorithm 1 with the readings of the scope table), independently of how
    the kernels evaluate them: +, -, x, /, sqrt and each elementary function
    (pow, log) = 1; comparisons, min/max and |x| = 0; data-dependent branches
    (shock square roots, the density division, the entropy iteration) not
    counted. Per node: primitives v, eps, p, a (3d + 7), a p^-z (2), Phi (2),
    eta (3), q (d), f(U) (d^2 + 2d + 1), eta'(U) (3d + 10). Per unique edge:
    n_ij (3d), the normal velocities (4d - 2), p_tr (7), the two outer wave
    speeds (14), d_ij (1). Per off-diagonal entry: (f_j - f_i) c_ij (S(3d - 1)),
    (q_j - q_i).c_ij (3d - 1), eta'.(.) (2S - 1), N and D (4); bar states and
    the low-order sum (7S + 1), d^H and F^H (4S + 3); P_ij (6S + 3); the l = 1
    check of each pass (S + 2d + 6); the limited updates (3S each) and the
    shrink (S + 1). Per node also: U^L (2S + 2), P's prefactor (2), the CFL
    bound (3), the SSP combination (3S)."""
    d, S = dim, dim + 2
    e = nnz - n
    check = S + 2 * d + 6
    per_entry, per_node = {
        "prep": (0.0, d * d + 9 * d + 25),
        "visc": ((7 * d + 20) / 2.0 + S * (3 * d - 1) + (3 * d - 1) + (2 * S - 1) + 4, 1),
        "low": ((7 * S + 1) + (4 * S + 3) + 1, 3),
        "lim1": ((6 * S + 3) + check, (2 * S + 2) + 2),
        "pass": (3 * S + (S + 1) + check, 0),
        "final": (3 * S, 3 * S),
        "tau": (0.0, 0),
        "lsearch": (0.0, 0),
    }[kernel]
    return per_entry * e + per_node * n


# FP64 peak: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (the recipe's
# 1.25 TFLOP/s; a throughput probe of independent FMA chains measured 1.01)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def peaks():
    try:
        d = json.load(open(MEASURED_PEAKS))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a window of the same mesh
# ---------------------------------------------------------------------------

def window_sample(mesh, U0, bs, x0=0.35, x1=0.85):
    """Rows with x in [x0, x1] (the cylinder and its bow shock) and the
    entries among them; the cut rows keep fewer neighbours (a timing sample)."""
    import dataclasses
    keep = (mesh.coords[:, 0] >= x0) & (mesh.coords[:, 0] <= x1)
    old = np.nonzero(keep)[0]
    new_of_old = np.full(mesh.n, -1, dtype=np.int64)
    new_of_old[old] = np.arange(old.size)
    rows = mesh.row_of_entry()
    sel = keep[rows] & keep[mesh.col]
    r2 = new_of_old[rows[sel]]
    row_ptr = np.zeros(old.size + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r2, minlength=old.size))
    bsel = keep[mesh.bnd_node]
    sm = dataclasses.replace(mesh, name=mesh.name + "-window", coords=mesh.coords[old], row_ptr=row_ptr,
                             col=new_of_old[mesh.col[sel]].astype(np.int32),
                             cij=np.ascontiguousarray(mesh.cij[:, sel]), mij=mesh.mij[sel], mi=mesh.mi[old],
                             bnd_node=new_of_old[mesh.bnd_node[bsel]].astype(np.int32),
                             bnd_kind=mesh.bnd_kind[bsel], bnd_normal=np.ascontiguousarray(mesh.bnd_normal[:, bsel]),
                             bnd_mass_full=mesh.bnd_mass_full[bsel],
                             bnd_normal_full=np.ascontiguousarray(mesh.bnd_normal_full[:, bsel]))
    return sm, np.ascontiguousarray(U0[:, old]), None if bs is None else np.ascontiguousarray(bs[:, bsel])


class OracleSample:
    """The oracle as it stands, on a sample of the workload (a window of the
    same mesh for large meshes, the full mesh otherwise), from the workload's
    initial state. ``threads`` OpenMP threads (0: all host cores)."""

    def __init__(self, w, threads=0):
        import oracle
        self.threads = oracle.set_threads(threads)
        if w.mesh.n > 200_000:
            mesh, U0, bs = window_sample(w.mesh, w.U0, w.bnd_state)
            self.sample = f"rows with x in [0.35, 0.85] of the same mesh ({mesh.n} vertices)"
        else:
            mesh, U0, bs = w.mesh, w.U0, w.bnd_state
            self.sample = f"the full mesh ({mesh.n} vertices)"
        self.n = mesh.n
        self.orc = oracle.Oracle(mesh, cfl=w.cfl, bnd_state=bs)
        self.U = self.orc.apply_bc(U0)

    def step(self):
        self.U, _, _ = self.orc.ssprk3_step(self.U)


STATE_NOTE = "from the inflow state (the same start as the reference arm)"


def cpu_baseline(w, seconds: float, threads=0):
    """Times the oracle: SSPRK(3,3) steps on the sample for ~``seconds``,
    from the workload's initial state."""
    smp = OracleSample(w, threads)
    steps = 0
    t0 = time.perf_counter()
    while True:
        smp.step()
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    value = smp.n * 3 * steps / el
    return {"value": value, "unit": UNIT, "cores": smp.threads, "kind": "oracle",
            "sample": f"{steps} SSPRK(3,3) steps on {smp.sample}, {STATE_NOTE}, FP64 C oracle, "
                      f"{smp.threads} OpenMP thread(s), {el:.1f} s"}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args, dist):
    """The oracle as the reference arm: each step is one SSPRK(3,3) step on
    the sample; rank 0 only."""
    if dist.rank != 0:
        return
    w, desc = make_workload(args)
    smp = OracleSample(w)
    for _ in range(args.warmup):
        smp.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.step()
    el = time.perf_counter() - t0
    value = smp.n * 3 * args.steps / el
    cb = {"value": value, "unit": UNIT, "cores": smp.threads, "kind": "oracle",
          "sample": f"{args.steps} SSPRK(3,3) steps on {smp.sample}, {STATE_NOTE}, FP64 C oracle, "
                    f"{smp.threads} OpenMP threads"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "vertices": w.mesh.n, "nnz": w.mesh.nnz},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per CSR entry of each kernel kind, from one ncu
# capture of the kernels as they stand (dram__bytes_read.sum +
# dram__bytes_write.sum, 2D Q1 cylinder, FP64, 4.0M vertices, the bench's own
# timed window; k_visc + k_alpha as "visc"); a launch moves about this times
# nnz. None where a kernel changed after the capture.
NCU_DRAM_BYTES_PER_ENTRY_2D_FP64 = {
    "prep": 24.3, "visc": 95.0, "low": 61.0, "lim1": 48.7, "pass": 32.4, "final": 18.3,
}
NCU_CAPTURE_NOTE = ("ncu launch list of the 4.0M-vertex cylinder at the bench's timed window "
                    "(dram__bytes_read.sum + dram__bytes_write.sum per launch, as bytes per CSR entry x nnz)")


def kernel_profile(solver, steps):
    """Per-kernel CUDA-event times (eager launches, events on the solver's
    stream) over ``steps`` steps: {kind: (total ms, launches)}."""
    solver.profile(True)
    solver.run(steps)
    prof = solver.profile_read()
    solver.profile(False)
    return prof


def roofline_of(prof, mesh, ms_per_step, hbm, hbm_src, precision):
    """The dominant kernel's FP64 fraction (method-fixed operation count over
    its mean CUDA-event time, against the FP64 peak) with its HBM fraction by
    the schedule's per-unit bytes, and the whole step's minimum-bytes HBM
    fraction."""
    total = sum(v[0] for v in prof.values())
    shares = {k: v[0] / total for k, v in prof.items() if v[1]}
    top = max((k for k in shares if k != "lsearch"), key=shares.get)
    top_ms = prof[top][0] / prof[top][1]
    flops = method_fp64_flops(top, mesh.n, mesh.nnz, mesh.dim)
    achieved = flops / (top_ms * 1e-3) / 1e12
    kbytes = survey_bytes(top, mesh.n, mesh.nnz, mesh.dim)
    step_bytes = 3 * survey_min_bytes_per_stage(mesh.n, mesh.nnz, mesh.dim)
    traffic = None
    if mesh.dim == 2 and precision == "fp64" and NCU_DRAM_BYTES_PER_ENTRY_2D_FP64.get(top) is not None:
        traffic = NCU_DRAM_BYTES_PER_ENTRY_2D_FP64[top] * mesh.nnz
    per_kernel = {}
    for k, (ms, cnt) in prof.items():
        if not cnt or k in ("tau", "lsearch"):
            continue
        t = ms / cnt * 1e-3
        per_kernel[k] = {"mean_launch_ms": round(ms / cnt, 4), "share": round(shares[k], 4),
                         "fp64_frac": round(method_fp64_flops(k, mesh.n, mesh.nnz, mesh.dim) / t / 1e12
                                            / FP64_PEAK_TFLOPS, 4),
                         "hbm_frac": round(survey_bytes(k, mesh.n, mesh.nnz, mesh.dim) / t / 1e9 / hbm, 4)}
    return {"bound": "alu", "kernel": f"k_{top}", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
            "traffic_source": NCU_CAPTURE_NOTE if traffic else None,
            "peak_source": "FP64 nominal: 152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz (the recipe's 1.25 TFLOP/s)",
            "count": "method-fixed FP64 operations per launch from the method's formulas (method_fp64_flops)",
            "method_fp64_flops_per_launch": flops, "mean_launch_ms": top_ms,
            "hbm": {"achieved": kbytes / (top_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": kbytes / (top_ms * 1e-3) / 1e9 / hbm, "peak_source": hbm_src,
                    "bytes_per_launch": kbytes, "bytes": "the planned schedule's per-unit figures (survey_bytes)"},
            "step_hbm_min": {"achieved": step_bytes / (ms_per_step * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm, "bytes_per_step": step_bytes,
                             "bytes": "minimum per stage x 3 (survey_min_bytes_per_stage)"},
            "kernel_shares": {k: round(v, 4) for k, v in sorted(shares.items(), key=lambda t: -t[1])},
            "per_kernel": per_kernel,
            "note": "the count is the method's for every entry; entries between bit-identical states are "
                    "evaluated by the exact identical-state shortcut (see identical_edge_share), so where that "
                    "share is large a fraction can exceed what the executed arithmetic alone would give -- "
                    "developed_flow has none of them; likewise the planned bytes of k_pass and k_final include "
                    "reads of P_ij that they skip where the limiter is 1 (the remainder (1 - l) P_ij is 0), so "
                    "their hbm_frac can exceed 1"}


def timed_steps(solver, stream, steps):
    """Device time of ``steps`` steps (one CUDA-graph replay each), CUDA events
    on the solver's stream, synchronised on both sides."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.run(steps)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def identical_edge_share(mesh, U):
    """Share of off-diagonal entries whose two states are equal bit for bit
    (the edges the kernels evaluate by the exact identical-state shortcut)."""
    rows = mesh.row_of_entry()
    off = mesh.col != rows
    same = np.all(U[:, mesh.col[off]] == U[:, rows[off]], axis=0)
    return float(same.mean())


def run_ours(args, dist):
    import torch
    from paper_2106_02159_gb300 import binding, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    w, desc = make_workload(args)
    mesh = w.mesh
    S = mesh.dim + 2
    stream = torch.cuda.Stream()
    precision = binding.EH_PRECISION_MIXED if args.precision == "mixed" else binding.EH_PRECISION_FP64
    solver = binding.Solver(dim=mesh.dim, cfl=w.cfl, gamma=w.gamma, device=dist.local_rank,
                            stream=stream.cuda_stream, precision=precision)
    solver.upload_mesh(mesh, w.bnd_state)
    solver.set_state(w.U0)
    solver.apply_boundary_conditions()
    # the limiter's work grows as the flow develops (the bow shock and its
    # wake spread over the channel), so the timed steps are taken from the
    # middle of the run, not from the uniform inflow state
    start = args.start_step if args.workload == "cylinder" else 0
    if start > 0:
        solver.run(start)
    solver.run(args.warmup)
    solver.synchronize()
    d_start = solver.diagnostics()
    t_window = d_start["t"]
    same_share = identical_edge_share(mesh, solver.get_state())

    # ---- device-timed steps (the contract's K steps) ----
    clocks = Clocks(dist.local_rank)
    dist.barrier()
    clocks.start()
    ms = timed_steps(solver, stream, args.steps)
    # repeats of the same K steps (the flow keeps developing): median and range
    repeats = [timed_steps(solver, stream, args.steps) for _ in range(args.repeats)]
    clk = clocks.stop()
    solver.synchronize()
    diag = solver.diagnostics()
    # share of the limiter line searches (one per off-diagonal entry, pass and
    # stage) that the l = 1 check did not settle, over the timed steps
    deferred = (diag["line_searches_deferred"] - d_start["line_searches_deferred"]) / (
        (args.steps * (1 + args.repeats)) * 3 * 2 * (mesh.nnz - mesh.n))
    dist.barrier()
    ms = dist.max(ms)
    per_step_ms = ms / args.steps
    value = mesh.n * 3 * args.steps * dist.world / (ms * 1e-3)
    rep_values = [mesh.n * 3 * args.steps / (r * 1e-3) for r in [ms] + repeats]

    # ---- per-kernel event timing (same kernels, eager launches) ----
    hbm, hbm_src = peaks()
    prof = kernel_profile(solver, args.profile_steps)
    roofline = roofline_of(prof, mesh, per_step_ms, hbm, hbm_src, args.precision)

    # ---- the same mesh with no identical-state edge: a seeded perturbed
    # state, so that every kernel evaluates every entry in full ----
    developed = None
    if args.workload == "cylinder" and not args.no_perturbed:
        U_keep = solver.get_state()
        Up = workloads.perturbed_state(mesh, 2106)
        solver.set_state(Up)
        solver.apply_boundary_conditions()
        same_p = identical_edge_share(mesh, solver.get_state())
        solver.run(args.warmup)
        pms = timed_steps(solver, stream, args.steps)
        pprof = kernel_profile(solver, args.profile_steps)
        developed = {"workload": "same mesh, seeded perturbed state (smooth density, pressure and velocity bumps "
                                 "on the inflow state), strict bounds: every entry evaluated in full",
                     "identical_edge_share": round(same_p, 4), "ms_per_step": pms / args.steps,
                     "value": mesh.n * 3 * args.steps / (pms * 1e-3), "unit": UNIT,
                     "roofline": roofline_of(pprof, mesh, pms / args.steps, hbm, hbm_src, args.precision)}
        developed["roofline"]["traffic"] = None
        developed["roofline"]["traffic_source"] = None
        solver.set_state(U_keep)

    # ---- end to end through the C ABI with host buffers ----
    host_in = torch.empty((S, mesh.n), dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty((S, mesh.n), dtype=torch.float64, pin_memory=True).numpy()
    solver.get_state(host_in)
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        solver.set_state(host_in)
        solver.step(sync=False)
        solver.get_state(host_out)
        host_in, host_out = host_out, host_in
    e2e_s = dist.max(time.perf_counter() - t0)
    e2e_value = mesh.n * 3 * args.e2e_steps * dist.world / e2e_s

    cb = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, args.cpu_seconds)
        if args.cpu_seconds_single > 0:
            cb1 = cpu_baseline(w, args.cpu_seconds_single, threads=1)
            cb["single_thread"] = {k: cb1[k] for k in ("value", "unit", "cores", "sample")}
    if dist.rank == 0:
        launches = solver.launches_per_step()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32/f64", "data": "synthetic",
            "config": {"workload": desc, "vertices": mesh.n, "nnz": mesh.nnz, "rk_stages_per_step": 3,
                       "limiter_passes": 2, "parallelism": f"replicas x{dist.world}",
                       "l2": "inputs larger than L2 (edge arrays ~{:.1f} GB per stage)".format(
                           mesh.nnz * 150 / 1e9),
                       "timed_steps": f"{start + args.warmup}..{start + args.warmup + args.steps} of the run "
                                      f"from the inflow state (t = {t_window:.4g} at the first timed step)",
                       "identical_edge_share": round(same_share, 4),
                       "line_searches_not_settled_at_l1": round(deferred, 4),
                       "invariant_violations": diag["not_admissible"],
                       "cfl_violations": diag["cfl_violations"]},
            "runs": {"what": f"the timed K steps and {args.repeats} repeats of K steps right after them",
                     "values": [round(v, 1) for v in rep_values], "median": float(np.median(rep_values)),
                     "min": float(min(rep_values)), "max": float(max(rep_values))},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * S * mesh.n,
                    "d2h_bytes_per_step": 8 * S * mesh.n},
            "gpu_launches": launches * args.steps,
            "roofline": roofline,
            "developed_flow": developed,
            "cpu_baseline": cb,
        }
        print(json.dumps(line), flush=True)
    solver.close()


def run_batch(args, dist):
    """Batched sweep (C4): independent Q1 cylinder instances (m log-uniform in
    [8, 256], i.e. 32x8 to 1024x256 cells; Mach uniform in [1.5, 4]; seed 4) in
    one context -- every kernel launch covers all instances, each with its own
    CFL step -- in FP64 and in mixed precision, against a per-instance launch
    loop of the plain FP64 path: the batching gain (batched FP64 / loop FP64)
    and the precision gain (batched mixed / batched FP64) separately.
    --batch-small: instances of 32x8 to 64x16 cells only (launch-bound)."""
    import torch
    from paper_2106_02159_gb300 import binding, meshes, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    m_range = (8, 16) if args.batch_small else (8, 256)
    sweep = workloads.batch_sweep(args.instances, m_range=m_range)
    inst = [workloads.cylinder_instance(m, mach) for m, mach in sweep]
    mesh, off, bs = meshes.concatenate([x[0] for x in inst], [x[2] for x in inst])
    U0 = np.concatenate([x[1] for x in inst], axis=1)
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for prec_name, precision in (("fp64", binding.EH_PRECISION_FP64), ("mixed", binding.EH_PRECISION_MIXED)):
        s = binding.Solver(dim=2, precision=precision, device=dist.local_rank, stream=stream.cuda_stream)
        s.upload_mesh(mesh, bs)
        s.set_instances(off)
        s.set_state(U0)
        s.apply_boundary_conditions()
        chosen = s.autotune(1)
        rows_cap = s.rows_per_sm()
        s.run(args.warmup)
        s.synchronize()
        clocks = Clocks(dist.local_rank)
        dist.barrier()
        clocks.start()
        e0.record(stream)
        s.run(args.steps)
        e1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        s.synchronize()
        ms = dist.max(e0.elapsed_time(e1))
        prof = kernel_profile(s, 2)
        kernel_ms = sum(v[0] for v in prof.values()) / 2
        out[prec_name] = {"value": mesh.n * 3 * args.steps * dist.world / (ms * 1e-3), "ms_per_step": ms / args.steps,
                          "eager_kernel_ms_per_step": kernel_ms,
                          "block_sizes": chosen, "rows_per_sm": rows_cap, "clocks": clk,
                          "invariant_violations": s.diagnostics()["not_admissible"]}
        s.close()
    # the baseline: a loop over instances, one plain FP64 context each
    loop = []
    for m, u, b in inst:
        q = binding.Solver(dim=2, device=dist.local_rank, stream=stream.cuda_stream)
        q.upload_mesh(m, b)
        q.set_state(u)
        q.apply_boundary_conditions()
        loop.append(q)
    for q in loop:
        q.run(args.warmup)
    torch.cuda.synchronize()
    loop_steps = max(1, args.steps // 4)
    clocks = Clocks(dist.local_rank)
    clocks.start()
    e0.record(stream)
    for _ in range(loop_steps):
        for q in loop:
            q.step(sync=False)
    e1.record(stream)
    stream.synchronize()
    loop_clk = clocks.stop()
    loop_ms = dist.max(e0.elapsed_time(e1))
    loop_value = mesh.n * 3 * loop_steps * dist.world / (loop_ms * 1e-3)
    for q in loop:
        q.close()
    if dist.rank == 0:
        cells = [4 * m * m for m, _ in sweep]
        main = out["mixed"]
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic", "clocks": main["clocks"],
            "config": {"workload": f"batched sweep: {len(inst)} independent Q1 cylinder instances, n_y = m cells "
                                   f"(m log-uniform in [{m_range[0]}, {m_range[1]}]), Mach uniform in [1.5, 4], "
                                   "seed 4, CFL 0.5, one launch per kernel for all instances (CUDA graph)",
                       "instances": len(inst), "vertices": mesh.n, "nnz": mesh.nnz,
                       "cells_min_max": [min(cells), max(cells)]},
            "batched": out,
            "per_instance_loop": {"value": loop_value, "unit": UNIT, "steps": loop_steps,
                                  "ms_per_step": loop_ms / loop_steps, "dtype": "f64", "clocks": loop_clk,
                                  "what": "one plain FP64 context per instance, eh_step launched instance after instance"},
            "batching_gain_fp64": out["fp64"]["value"] / loop_value,
            "precision_gain_batched": out["mixed"]["value"] / out["fp64"]["value"],
            "speedup_vs_loop": main["value"] / loop_value,
        }
        print(json.dumps(line), flush=True)


def run_serve(args, dist):
    """Served stream: a seeded Poisson trace (mean 50 requests/s, seed 5) of 2D
    Euler solves on P1/Q1 cylinder meshes (vertices log-uniform in [1e4, 4e6],
    snapped to 16 log-spaced sizes; Mach uniform in [1.5, 4]) to a common
    t_final, served with continuous batching -- merged mode (all running
    requests are the instances of one batched context, repacked as they come
    and go) in mixed precision and in FP64, and the per-request-stream mode --
    against the same requests solved one after another with the plain FP64
    path (their service times replayed against the same arrivals). Every run
    is timed with clock samples."""
    import torch
    from paper_2106_02159_gb300 import binding, serve
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    if dist.rank != 0:
        return
    reqs = serve.poisson_trace(args.requests, rate=50.0, seed=5, n_range=(1e4, args.serve_max_vertices),
                               t_final=args.serve_t_final, size_grid=16, workers=16)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    # warm the library and the caches once
    serve.solve_alone(reqs[0], binding.EH_PRECISION_MIXED)
    total_vertices = sum(r.mesh.n for r in reqs)

    def served(mode, precision):
        clocks = Clocks(dist.local_rank)
        clocks.start()
        t0 = time.perf_counter()
        results = serve.SolveServer(budget, precision=precision, device=dist.local_rank, mode=mode).run(reqs)
        makespan = time.perf_counter() - t0
        clk = clocks.stop()
        tts = np.array([r.time_to_solution for r in results])
        dof = sum(r.n * 3 * r.steps for r in results)
        return {"p50_s": float(np.percentile(tts, 50)), "p99_s": float(np.percentile(tts, 99)),
                "aggregate": dof / makespan, "unit": UNIT, "makespan_s": makespan,
                "served_requests_per_s": len(results) / makespan, "steps": int(sum(r.steps for r in results)),
                "clocks": clk}

    runs = {
        "merged_mixed": served(binding.EH_BATCH_MERGED, binding.EH_PRECISION_MIXED),
        "merged_fp64": served(binding.EH_BATCH_MERGED, binding.EH_PRECISION_FP64),
        "streams_mixed": served(binding.EH_BATCH_PER_REQUEST_STREAMS, binding.EH_PRECISION_MIXED),
    }
    # sequential plain FP64 baseline: each solve alone, then queueing replayed
    clocks = Clocks(dist.local_rank)
    clocks.start()
    service = []
    for r in reqs:
        a = time.perf_counter()
        _, steps = serve.solve_alone(r, binding.EH_PRECISION_FP64)
        service.append((time.perf_counter() - a, steps))
    clk = clocks.stop()
    finish, seq_tts = 0.0, []
    for r, (svc, _) in zip(reqs, service):
        finish = max(finish, r.arrival) + svc
        seq_tts.append(finish - r.arrival)
    seq_tts = np.array(seq_tts)
    seq_dof = sum(r.mesh.n * 3 * st for r, (_, st) in zip(reqs, service))
    runs["sequential_plain_fp64"] = {"p50_s": float(np.percentile(seq_tts, 50)),
                                     "p99_s": float(np.percentile(seq_tts, 99)),
                                     "aggregate": seq_dof / sum(x for x, _ in service), "unit": UNIT,
                                     "makespan_s": finish, "clocks": clk}
    main = runs["merged_mixed"]
    line = {
        "metric": "p50/p99 time-to-solution (served)", "value": main["p99_s"], "unit": "s",
        "p50_s": main["p50_s"], "p99_s": main["p99_s"], "n_gpus": 1, "steps": main["steps"], "warmup": 1,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "aggregate": {"value": main["aggregate"], "unit": UNIT, "makespan_s": main["makespan_s"]},
        "load": {"offered_requests_per_s": 50.0, "served_requests_per_s": main["served_requests_per_s"]},
        "clocks": main["clocks"],
        "config": {"workload": f"served stream: {len(reqs)} requests, Poisson arrivals (mean 50/s, seed 5), P1/Q1 "
                               f"cylinder meshes, vertices log-uniform in [1e4, {args.serve_max_vertices:.0e}] "
                               f"(16 log-spaced sizes), Mach uniform in [1.5, 4], t_final {args.serve_t_final:g}, "
                               "admission by device memory, states resident, merged continuous batching",
                   "requests": len(reqs), "total_vertices": total_vertices,
                   "distinct_sizes": sorted({r.mesh.n for r in reqs}), "hbm_budget_bytes": budget},
        "runs": runs,
    }
    print(json.dumps(line), flush=True)


def run_cylinder3d(args, dist):
    """3D Mach-3 cylinder: the 2D cross-section (~94k vertices) extruded over
    z in [0, 2] with periodic layers to ~30M vertices (27-point rows), inflow
    rho = 1.4, u = (3, 0, 0), p = 1, slip on walls and cylinder; the same
    steps in FP64 and in mixed precision, with the L1 error per field of the
    mixed run against the FP64 run."""
    import torch
    from paper_2106_02159_gb300 import binding, meshes, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    target = max(args.vertices, 1) if args.vertices != 4_000_000 else 30_000_000
    m2 = meshes.cylinder_m_for_vertices(94_000)
    base = meshes.cylinder_channel_q1(m2)
    nz = max(3, int(round(target / base.n)))
    mesh = meshes.extruded_q1(base, nz, 2.0)
    U0 = workloads.uniform_state(mesh, 1.4, (3.0, 0.0, 0.0), 1.0)
    bs = np.ascontiguousarray(U0[:, mesh.bnd_node])
    out = {}
    for prec in ("fp64", "mixed"):
        stream = torch.cuda.Stream()
        p = binding.EH_PRECISION_MIXED if prec == "mixed" else binding.EH_PRECISION_FP64
        s = binding.Solver(dim=3, precision=p, device=dist.local_rank, stream=stream.cuda_stream)
        s.upload_mesh(mesh, bs)
        s.set_state(U0)
        s.apply_boundary_conditions()
        # the timed steps start in the middle of the 200-step run (the bow
        # shock and its wake have formed), not at the uniform inflow state
        s.run(args.start3d + args.warmup)
        s.synchronize()
        same = identical_edge_share(mesh, s.get_state())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = Clocks(dist.local_rank)
        clocks.start()
        e0.record(stream)
        s.run(args.steps)
        e1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        s.synchronize()
        U = s.get_state()
        viol = s.diagnostics()["not_admissible"]
        s.profile(True)
        s.run(1)
        prof = s.profile_read()
        s.profile(False)
        tot = sum(v[0] for v in prof.values())
        shares = {k: round(v[0] / tot, 4) for k, v in sorted(prof.items(), key=lambda t: -t[1][0]) if v[1]}
        out[prec] = dict(value=mesh.n * 3 * args.steps / (ms * 1e-3), ms_per_step=ms / args.steps,
                         U=U, violations=viol, shares=shares, clocks=clk, identical_edge_share=same,
                         roofline=roofline_of(prof, mesh, ms / args.steps, *peaks(), prec))
        out[prec]["roofline"]["traffic"] = None
        out[prec]["roofline"]["traffic_source"] = None
        if prec == "fp64" and not args.no_perturbed:
            # the same mesh from a seeded perturbed state: every entry in full
            Up = workloads.perturbed_state(mesh, 2106, base=dict(rho=1.4, vel=(3.0, 0.0, 0.0), p=1.0))
            s.set_state(Up)
            s.apply_boundary_conditions()
            s.run(2)
            s.synchronize()
            e0.record(stream)
            s.run(args.steps)
            e1.record(stream)
            stream.synchronize()
            pms = e0.elapsed_time(e1)
            pprof = kernel_profile(s, 1)
            out["developed"] = {"workload": "same mesh, seeded perturbed state: every entry evaluated in full",
                                "identical_edge_share": identical_edge_share(mesh, s.get_state()),
                                "ms_per_step": pms / args.steps, "value": mesh.n * 3 * args.steps / (pms * 1e-3),
                                "roofline": roofline_of(pprof, mesh, pms / args.steps, *peaks(), prec)}
            out["developed"]["roofline"]["traffic"] = None
            out["developed"]["roofline"]["traffic_source"] = None
        s.close()
        del s
        torch.cuda.empty_cache()
    Uf, Um = out["fp64"]["U"], out["mixed"]["U"]
    names = ("rho", "m_x", "m_y", "m_z", "E")
    norms = np.abs(Uf).sum(1)
    err = np.abs(Um - Uf).sum(1) / np.maximum(norms, 1e-3 * norms.max())
    if dist.rank == 0:
        line = {"metric": METRIC, "value": out["fp64"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": out["fp64"]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"3D Mach-3 cylinder, Q1 hexes: the {base.n}-vertex 2D cross-section "
                                       f"extruded over z in [0,2] with {nz} periodic layers, {mesh.n} vertices, "
                                       f"27-point rows, CFL 0.5, strict local bounds",
                           "vertices": mesh.n, "nnz": mesh.nnz},
                "mixed": {"value": out["mixed"]["value"], "unit": UNIT, "ms_per_step": out["mixed"]["ms_per_step"],
                          "speedup_vs_fp64": out["mixed"]["value"] / out["fp64"]["value"],
                          "l1_rel_error_vs_fp64_run": dict(zip(names, err.tolist())),
                          "after_steps": args.warmup + args.steps},
                "invariant_violations": {"fp64": out["fp64"]["violations"], "mixed": out["mixed"]["violations"]},
                "clocks": out["fp64"]["clocks"], "clocks_mixed": out["mixed"]["clocks"],
                "identical_edge_share": out["fp64"]["identical_edge_share"],
                "timed_steps": f"{args.start3d + args.warmup}..{args.start3d + args.warmup + args.steps} of the run "
                               "from the inflow state",
                "developed_flow": out.get("developed"),
                "roofline": out["fp64"]["roofline"],
                "kernel_shares": {"fp64": out["fp64"]["shares"], "mixed": out["mixed"]["shares"]}}
        print(json.dumps(line), flush=True)


def nrbc_deltas(mesh, U, curl0_max):
    """delta_1 = max |v - v_inf| / |v_inf| and delta_2 = max |curl v| / max |curl v_0|
    over the nodes (Sec. 6, non-reflecting conditions), with v_inf = (1, 0) and
    the nodal curl of the lumped Galerkin projection, (curl v)_i = (1/m_i)
    sum_j (c_ij,x v_j,y - c_ij,y v_j,x)."""
    v = U[1:3] / U[0]
    d1 = float(np.sqrt((v[0] - 1.0) ** 2 + v[1] ** 2).max())
    rows = mesh.row_of_entry()
    cv = mesh.cij[0] * v[1, mesh.col] - mesh.cij[1] * v[0, mesh.col]
    curl = np.bincount(rows, weights=cv, minlength=mesh.n) / mesh.mi
    cmax = float(np.abs(curl).max())
    return d1, (cmax / curl0_max if curl0_max else cmax)


def run_nrbc(args, dist):
    """The non-reflecting boundary tests of Sec. 6: a vortex (r0 = 0.1) carried
    by a unit free stream out of [-1,1]^2 on an 80 x 80 Q1 mesh, CFL 0.75,
    strict bounds, to t = 4, for the four (Mach, perturbation) cases, with the
    characteristic and the Godunov post-processing on all four sides (and
    do-nothing as a reflecting reference): delta_1(t), delta_2(t)."""
    import torch
    from paper_2106_02159_gb300 import binding, meshes, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    if dist.rank != 0:
        return
    kinds = {"characteristic": meshes.BC_CHARACTERISTIC, "godunov": meshes.BC_GODUNOV,
             "do_nothing": meshes.BC_DO_NOTHING}
    samples = (0.5, 1.0, 1.5, 2.0, 3.0, 4.0)
    results, total_dof, total_ms = {}, 0.0, 0.0
    clocks = Clocks(dist.local_rank)
    clocks.start()
    for case in sorted(workloads.NRBC_CASES):
        for kname, kind in kinds.items():
            mesh, U0, bs = workloads.nrbc_vortex_problem(80, case, kind)
            v0 = U0[1:3] / U0[0]
            rows = mesh.row_of_entry()
            c0 = np.bincount(rows, weights=mesh.cij[0] * v0[1, mesh.col] - mesh.cij[1] * v0[0, mesh.col],
                             minlength=mesh.n) / mesh.mi
            c0max = float(np.abs(c0).max())
            stream = torch.cuda.Stream()
            s = binding.Solver(dim=2, cfl=0.75, stream=stream.cuda_stream)
            s.upload_mesh(mesh, bs)
            s.set_instances([0, mesh.n], [4.0])
            s.set_state(U0)
            s.apply_boundary_conditions()
            series, steps, k, failure, t = [], 0, 0, None, 0.0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            while True:
                e0.record(stream)
                s.run(20)
                e1.record(stream)
                stream.synchronize()
                try:
                    t_now = float(s.instances()["t"][0])
                except binding.EulerError as e:  # e.g. a non-admissible state: record it and stop this run
                    failure = {"after_steps": steps + 20, "last_t": t, "error": str(e)}
                    break
                total_ms += e0.elapsed_time(e1)
                steps += 20
                t = t_now
                while k < len(samples) and t >= samples[k] - 1e-12:
                    d1, d2 = nrbc_deltas(mesh, s.get_state(), c0max)
                    series.append({"t": round(t, 4), "delta_1": d1, "delta_2": d2})
                    k += 1
                if t >= 4.0 or k >= len(samples):
                    break
            total_dof += mesh.n * 3 * steps
            results[f"{case}/{kname}"] = {"mach": workloads.NRBC_CASES[case][0],
                                          "vbar": workloads.NRBC_CASES[case][1], "steps": steps,
                                          "failure": failure, "deltas": series}
            s.close()
    clk = clocks.stop()
    line = {"metric": "delta_1(t), delta_2(t) of the vortex leaving the box (non-reflecting conditions)",
            "clocks": clk,
            "value": None, "unit": "1", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "dtype": "f64",
            "config": {"workload": "Sec. 6 non-reflecting tests: [-1,1]^2, 80x80 Q1, rho=1, v_inf=(1,0), "
                                   "r0=0.1, CFL 0.75, strict bounds, t in [0, 4]",
                       "cases": {k: list(v) for k, v in workloads.NRBC_CASES.items()}},
            "throughput": {"value": total_dof / (total_ms * 1e-3), "unit": UNIT,
                           "what": "all 12 runs, device time of the steps (6561-vertex meshes: launch-bound)"},
            "results": results}
    print(json.dumps(line), flush=True)


def run_adaptive(args, dist):
    """Adaptive CFL (Sec. 3.1, remark on high aspect-ratio meshes): a periodic
    Q1 channel of 2000 x 500 cells with aspect ratio 50:1 (boundary-layer-like
    cells), slip walls, Mach-3 flow with seeded bumps; simulated time advanced
    per second by plain steps at c_cfl = 0.5 and by adaptive steps from
    cfl_max = 2, 4, 8 (restarts counted as work)."""
    import torch
    from paper_2106_02159_gb300 import binding, meshes, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    if dist.rank != 0:
        return
    nx, ny, aspect = 2000, 500, 50.0
    hy = 1.0 / nx / aspect
    mesh = meshes.structured_q1(nx, ny, 0.0, 1.0, 0.0, ny * hy, periodic_x=True,
                                kinds=(0, 0, meshes.BC_SLIP, meshes.BC_SLIP))
    U0 = workloads.perturbed_state(mesh, 4, base=dict(rho=1.4, vel=(3.0, 0.0), p=1.0), amplitude=0.3)
    stream = torch.cuda.Stream()
    out = {}
    clocks = Clocks(dist.local_rank)
    clocks.start()
    for label, cfl_max in (("plain c_cfl=0.5", None), ("adaptive cfl_max=2", 2.0), ("adaptive cfl_max=4", 4.0),
                           ("adaptive cfl_max=8", 8.0)):
        s = binding.Solver(dim=2, cfl=0.5, stream=stream.cuda_stream)
        s.upload_mesh(mesh, None)
        s.set_state(U0)
        s.apply_boundary_conditions()
        s.step()  # warm-up (and the graph for the plain path)
        s.run(1)
        s.synchronize()
        t_start = float(s.instances()["t"][0])
        steps, attempts, cfls = args.steps, 0, []
        t0 = time.perf_counter()
        if cfl_max is None:
            s.run(steps)
            s.synchronize()
            attempts = steps
        else:
            for _ in range(steps):
                _, c, r = s.step_adaptive(cfl_max)
                cfls.append(c)
                attempts += 1 + r
        el = time.perf_counter() - t0
        t_sim = float(s.instances()["t"][0]) - t_start
        d = s.diagnostics()
        out[label] = {"steps": steps, "attempts": attempts, "mean_cfl": float(np.mean(cfls)) if cfls else 0.5,
                      "simulated_time": t_sim, "wall_s": el, "simulated_time_per_s": t_sim / el,
                      "dof_updates_per_s": mesh.n * 3 * attempts / el,
                      "not_admissible": d["not_admissible"]}
        s.close()
    clk = clocks.stop()
    base = out["plain c_cfl=0.5"]["simulated_time_per_s"]
    for v in out.values():
        v["speedup_vs_plain"] = v["simulated_time_per_s"] / base
    line = {"metric": "simulated time advanced per second (adaptive CFL vs plain)", "clocks": clk, "value":
            max(v["speedup_vs_plain"] for v in out.values()), "unit": "x plain", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f64",
            "config": {"workload": f"periodic Q1 channel {nx}x{ny} cells, aspect ratio {aspect:g}:1, slip walls, "
                                   "Mach-3 flow with seeded bumps, strict bounds", "vertices": mesh.n,
                       "steps": args.steps},
            "results": out}
    print(json.dumps(line), flush=True)


def run_ns(args, dist):
    """Strang-split Navier-Stokes steps (eq. continuous_Strang, Sec. 5) on the Q1
    cylinder channel (--vertices), Mach-3 inflow, no-slip cylinder and walls in
    the parabolic step, mu = 1e-4, lambda = 0, kappa/c_v = 1.4e-4 (Pr ~ 1):
    vertices x 2 hyperbolic steps x 3 stages per second of NS steps, the
    parabolic sub-step's share and its CG iteration counts, against the plain
    Euler path's own steps on the same mesh."""
    import torch
    from paper_2106_02159_gb300 import binding, meshes, workloads
    torch.cuda.set_device(dist.local_rank)
    binding.build()
    if dist.rank != 0:
        return
    m = meshes.cylinder_m_for_vertices(args.vertices)
    mesh, U0, bs = workloads.cylinder_problem(m)
    wall = mesh.bnd_node[mesh.bnd_kind == meshes.BC_SLIP]
    pdata = meshes.parabolic_data(mesh)
    stream = torch.cuda.Stream()
    s = binding.Solver(dim=2, cfl=0.5, stream=stream.cuda_stream)
    s.upload_mesh(mesh, bs)
    mu, kc = 1e-4, 1.4e-4
    s.set_viscosity(pdata, mu, 0.0, kc, wall=wall)
    U0 = U0.copy()
    U0[1:3, wall] = 0.0
    s.set_state(U0)
    s.apply_boundary_conditions()
    for _ in range(args.warmup):
        s.step_ns()
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, par_ms = [], 0.0
    clocks = Clocks(dist.local_rank)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tau, info = s.step_ns()
        iters.append((info["cg_iter_velocity"], info["cg_iter_energy"], info["cg_iter_low"]))
    ns_wall = time.perf_counter() - t0
    # the parabolic sub-step alone, and the hyperbolic steps alone, on the same state
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.parabolic_step(2.0 * tau)
    par_wall = time.perf_counter() - t0
    e0.record(stream)
    s.run(2 * args.steps)
    e1.record(stream)
    stream.synchronize()
    euler_ms = e0.elapsed_time(e1) / (2 * args.steps)
    clk = clocks.stop()
    d = s.diagnostics()
    line = {"metric": "DOF-updates/s per RK stage (Navier-Stokes steps)", "unit": UNIT, "n_gpus": 1,
            "value": mesh.n * 2 * 3 * args.steps / ns_wall, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * ns_wall / args.steps, "higher_is_better": True, "data": "synthetic", "dtype": "f64",
            "config": {"workload": f"Q1 cylinder channel, {mesh.n} vertices, Mach-3 inflow, no-slip cylinder and "
                                   f"walls in the parabolic step, mu={mu:g}, lambda=0, kappa/c_v={kc:g}, CFL 0.5, "
                                   "strict bounds; one NS step = H(tau) P(2 tau) H(tau)",
                       "vertices": mesh.n, "nnz": mesh.nnz},
            "parabolic_ms_per_step": 1e3 * par_wall / args.steps,
            "euler_ms_per_ssprk3_step": euler_ms,
            "cg_iterations_velocity_energy_low": iters[-1],
            "cg_iterations_mean": [float(np.mean([it[q] for it in iters])) for q in range(3)],
            "not_admissible": d["not_admissible"], "clocks": clk,
            "timing": "host wall clock around synchronising calls (the CG loops read their control pair once per "
                      "batch of queued iterations)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        elif args.workload == "batch":
            run_batch(args, dist)
        elif args.workload == "serve":
            run_serve(args, dist)
        elif args.workload == "cylinder3d":
            run_cylinder3d(args, dist)
        elif args.workload == "nrbc":
            run_nrbc(args, dist)
        elif args.workload == "adaptive":
            run_adaptive(args, dist)
        elif args.workload == "ns":
            run_ns(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
