"""Seeded synthetic workloads: initial states and the benchmark configurations.

Only inputs live here (initial data, Dirichlet states, mesh choices); none of
the hyperbolic step's arithmetic. States are returned component-major,
``U[s, i]`` with s = 0 (rho), 1..dim (momentum), dim+1 (total energy), which
is the layout the C-ABI takes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import meshes


def conserved(rho, vel, p, gamma=1.4):
    """(rho, v, p) -> (rho, m, E) with E = p/(gamma-1) + rho |v|^2 / 2 (ideal gas)."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = [np.asarray(v, dtype=np.float64) for v in vel]
    p = np.asarray(p, dtype=np.float64)
    shape = np.broadcast(rho, p, *vel).shape
    ke = sum(np.broadcast_to(v, shape) ** 2 for v in vel) * 0.5 * np.broadcast_to(rho, shape)
    out = [np.broadcast_to(rho, shape)]
    out += [np.broadcast_to(rho, shape) * np.broadcast_to(v, shape) for v in vel]
    out.append(np.broadcast_to(p, shape) / (gamma - 1.0) + ke)
    return np.ascontiguousarray(np.stack(out))


def uniform_state(mesh, rho=1.4, vel=(3.0, 0.0), p=1.0, gamma=1.4):
    vel = tuple(vel) + (0.0,) * (mesh.dim - len(vel))
    one = np.ones(mesh.n)
    return conserved(rho * one, [v * one for v in vel[: mesh.dim]], p * one, gamma)


# --------------------------------------------------------------------------
# isentropic vortex (Shu 1998; Yee et al. 1999)
# --------------------------------------------------------------------------

def isentropic_vortex_primitive(x, y, t=0.0, beta=5.0, gamma=1.4, u_inf=(1.0, 1.0), lo=-5.0, hi=5.0):
    """Vortex of strength beta centred at (0,0) + u_inf t on the periodic box
    [lo,hi]^2: du = beta/(2 pi) e^{(1-r^2)/2} (-y, x),
    T = 1 - (gamma-1) beta^2/(8 gamma pi^2) e^{1-r^2}, rho = T^{1/(gamma-1)},
    p = rho T. Returns rho, u, v, p."""
    L = hi - lo
    xc = x - u_inf[0] * t
    yc = y - u_inf[1] * t
    xc = (xc - lo) % L + lo
    yc = (yc - lo) % L + lo
    r2 = xc * xc + yc * yc
    du = beta / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * math.pi * math.pi) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return rho, u_inf[0] - du * yc, u_inf[1] + du * xc, rho * T


def isentropic_vortex(mesh, t=0.0, beta=5.0, gamma=1.4):
    rho, u, v, p = isentropic_vortex_primitive(mesh.coords[:, 0], mesh.coords[:, 1], t, beta, gamma)
    return conserved(rho, [u, v], p, gamma)


# --------------------------------------------------------------------------
# 1D Riemann problems on a quasi-1D strip
# --------------------------------------------------------------------------

RIEMANN_CASES = {
    # name: (rho_L, u_L, p_L, rho_R, u_R, p_R, t_end) on x in [0, 1], interface at 0.5
    "sod": (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 0.2),
    "lax": (0.445, 0.698, 3.528, 0.5, 0.0, 0.571, 0.13),
    "strong_shock": (1.0, 0.0, 100.0, 1.0, 0.0, 0.01, 0.035),
    "double_rarefaction": (1.0, -2.0, 0.4, 1.0, 2.0, 0.4, 0.1),
}


def riemann_strip(nx: int, ny: int = 4):
    """Q1 strip [0,1] x [0, ny/nx], periodic in y, do-nothing at x = 0, 1."""
    return meshes.structured_q1(nx, ny, 0.0, 1.0, 0.0, ny / nx, periodic_y=True,
                                kinds=(meshes.BC_DO_NOTHING, meshes.BC_DO_NOTHING, 0, 0),
                                name=f"q1-strip-{nx}x{ny}")


def riemann_initial(mesh, case, gamma=1.4, x0=0.5):
    rl, ul, pl, rr, ur, pr, _ = RIEMANN_CASES[case] if isinstance(case, str) else case
    x = mesh.coords[:, 0]
    left = x < x0
    mid = np.isclose(x, x0)
    rho = np.where(left, rl, rr).astype(float)
    u = np.where(left, ul, ur).astype(float)
    p = np.where(left, pl, pr).astype(float)
    U = conserved(rho, [u, np.zeros_like(u)], p, gamma)
    if mid.any():  # the interface node carries the average of the two states
        UL = conserved(rl, [ul, 0.0], pl, gamma)
        UR = conserved(rr, [ur, 0.0], pr, gamma)
        U[:, mid] = 0.5 * (UL + UR)[:, None]
    return U


def random_riemann_case(rng, gamma=1.4):
    """Seeded Riemann data: rho, p log-uniform in [1e-3, 1e3]... kept moderate for the strip runs."""
    rl, rr = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 2))
    pl, pr = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 2))
    ul, ur = rng.uniform(-1.0, 1.0, 2)
    return (rl, ul, pl, rr, ur, pr, 0.1)


# --------------------------------------------------------------------------
# Mach-3 cylinder channel
# --------------------------------------------------------------------------

CYLINDER_INFLOW = dict(rho=1.4, vel=(3.0, 0.0), p=1.0)


def cylinder_problem(m: int, gamma=1.4):
    """Q1 cylinder channel with U0 = inflow state everywhere; returns
    (mesh, U0, bnd_state) where bnd_state holds the inflow state for every
    boundary node (only the Dirichlet ones read it)."""
    mesh = meshes.cylinder_channel_q1(m)
    U0 = uniform_state(mesh, gamma=gamma, **CYLINDER_INFLOW)
    bnd_state = np.ascontiguousarray(U0[:, mesh.bnd_node])
    return mesh, U0, bnd_state


# --------------------------------------------------------------------------
# non-reflecting boundary tests (Sec. 6: vortex leaving [-1,1]^2)
# --------------------------------------------------------------------------

# case: (Mach number of the free stream, velocity perturbation of the vortex)
NRBC_CASES = {"i": (0.5, 0.75), "ii": (0.5, 0.25), "iii": (0.05, 0.75), "iv": (0.05, 0.25)}


def nrbc_vortex_state(x, mach, vbar, r0=0.1, gamma=1.4, center=(0.0, 0.0)):
    """rho = 1, v = (1, 0) + vbar/r0 psi(r) (-(y - y0), x - x0), p = p_inf -
    vbar^2 psi(r)^2 / 2 with psi(r) = exp((1 - r^2/r0^2)/2) and p_inf =
    a_inf^2/gamma, a_inf = 1/mach. The paper leaves r0 and the centre to the
    cited test suite; here r0 = 0.1 and the centre is the origin (so the centre
    crosses x = 1 at t = 1)."""
    dx = x[:, 0] - center[0]
    dy = x[:, 1] - center[1]
    psi = np.exp(0.5 * (1.0 - (dx * dx + dy * dy) / (r0 * r0)))
    p_inf = (1.0 / mach) ** 2 / gamma
    vx = 1.0 - vbar / r0 * psi * dy
    vy = vbar / r0 * psi * dx
    return conserved(np.ones(x.shape[0]), [vx, vy], p_inf - 0.5 * vbar * vbar * psi * psi, gamma)


def nrbc_vortex_problem(n_cells=80, case="i", kind=None, r0=0.1, gamma=1.4):
    """The vortex of ``nrbc_vortex_state`` on an n_cells x n_cells Q1 mesh of
    [-1,1]^2 with a non-reflecting kind (default: characteristic) on all four
    sides and the free stream as far-field state. Returns (mesh, U0, bnd_state)."""
    kind = meshes.BC_CHARACTERISTIC if kind is None else kind
    mach, vbar = NRBC_CASES[case]
    mesh = meshes.structured_q1(n_cells, n_cells, -1.0, 1.0, -1.0, 1.0, kinds=(kind,) * 4,
                                name=f"nrbc-q1-{n_cells}-{case}-k{kind}")
    U0 = nrbc_vortex_state(mesh.coords, mach, vbar, r0, gamma)
    p_inf = (1.0 / mach) ** 2 / gamma
    far = conserved(np.ones(mesh.bnd_node.size), [np.ones(mesh.bnd_node.size), np.zeros(mesh.bnd_node.size)],
                    np.full(mesh.bnd_node.size, p_inf), gamma)
    return mesh, U0, np.ascontiguousarray(far)


@dataclasses.dataclass
class Workload:
    name: str
    mesh: object
    U0: np.ndarray
    bnd_state: np.ndarray | None
    steps: int
    cfl: float = 0.5
    gamma: float = 1.4


def vortex_workload(nv: int = 64, steps: int = 100) -> Workload:
    """2D isentropic vortex on the nv x nv-vertex periodic P1 mesh, CFL 0.5."""
    mesh = meshes.periodic_p1_square(nv)
    return Workload(f"vortex-p1-{nv}x{nv}", mesh, isentropic_vortex(mesh), None, steps)


def cylinder_workload(target_vertices: int = 4_000_000, steps: int = 2000) -> Workload:
    """Mach-3 flow past a cylinder, Q1, ~target_vertices vertices, CFL 0.5."""
    m = meshes.cylinder_m_for_vertices(target_vertices)
    mesh, U0, bs = cylinder_problem(m)
    return Workload(f"cylinder-q1-m{m}", mesh, U0, bs, steps)


def perturbed_state(mesh, seed: int, base=None, amplitude=0.3, n_bumps=12, gamma=1.4):
    """Seeded admissible state with smooth density / pressure / velocity bumps
    on top of ``base`` (default: the Mach-3 inflow state); exercises every
    branch of the step (shocks form, limiter active) from the first step."""
    rng = np.random.default_rng(seed)
    x = mesh.coords
    lo, hi = x.min(0), x.max(0)
    base = base or CYLINDER_INFLOW
    rho = np.full(mesh.n, base["rho"], dtype=float)
    p = np.full(mesh.n, base["p"], dtype=float)
    vel = [np.full(mesh.n, v, dtype=float) for v in tuple(base["vel"]) + (0.0,) * (mesh.dim - len(base["vel"]))]
    scale = (hi - lo).max()
    for _ in range(n_bumps):
        c = rng.uniform(lo, hi)
        r = rng.uniform(0.03, 0.15) * scale
        g = np.exp(-((x - c) ** 2).sum(1) / (r * r))
        rho *= 1.0 + amplitude * rng.uniform(-0.9, 1.0) * g
        p *= 1.0 + amplitude * rng.uniform(-0.9, 2.0) * g
        for d in range(mesh.dim):
            vel[d] += amplitude * rng.uniform(-2.0, 2.0) * g
    return conserved(rho, vel[: mesh.dim], p, gamma)


def cylinder_instance(m: int, mach: float, gamma=1.4):
    """Cylinder channel of size m with inflow rho = 1.4, p = 1 (sound speed 1)
    and u = (mach, 0); returns (mesh, U0, bnd_state)."""
    mesh = meshes.cylinder_channel_q1(m)
    U0 = uniform_state(mesh, 1.4, (mach, 0.0), 1.0, gamma)
    return mesh, U0, np.ascontiguousarray(U0[:, mesh.bnd_node])


def batch_sweep(count: int = 256, seed: int = 4, m_range=(8, 256), mach_range=(1.5, 4.0)):
    """Seeded sweep of independent Q1 cylinder instances: n_y = m cells across
    the channel, m log-uniform in m_range (cells n_x n_y ~ 4 m^2 log-uniform
    between 32x8 and 1024x256), inflow Mach uniform in mach_range. Returns a
    list of (m, mach)."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]), count)).round().astype(int)
    machs = rng.uniform(mach_range[0], mach_range[1], count)
    return list(zip(ms.tolist(), machs.tolist()))
