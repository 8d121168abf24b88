"""Pins of the oracle's parabolic sub-step (Sec. 5) and Strang step
(eq. continuous_Strang). Against closed forms: plane viscous waves (the
operator div sigma(v) = mu lap v + (lambda + mu/3) grad div v decays a
transverse wave at mu |k|^2 and a longitudinal one at (4 mu/3 + lambda) |k|^2)
and heat decay, at second order in h and dt together (Crank-Nicolson);
Lemma 5.x: density unchanged, momentum and total energy conserved on a
periodic box, no-slip nodes at rest, positivity of e through the FCT limiter
(min e^{n+1} >= min e^n); zero viscosity and conductivity give the identity;
the Strang step with no dissipation is two hyperbolic steps. CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W


SHEAR = 0.3  # sheared P1 box: lattice (1, 0), (0.3, 1); k = 2 pi (1, 0.7) is periodic on it


def _box(n, elem):
    if elem == "q1":
        return M.structured_q1(n, n, 0.0, 1.0, 0.0, 1.0, periodic_x=True, periodic_y=True)
    if elem == "p1sheared":
        return M.periodic_p1_square(n, 0.0, 1.0, shear=SHEAR)
    return M.periodic_p1_square(n, 0.0, 1.0)


def _orc(mesh, mu, lam, kc, wall=None):
    o = oracle.Oracle(mesh, cfl=0.5)
    o.set_viscosity(M.parabolic_data(mesh), mu, lam, kc, wall=wall)
    return o


def _state(mesh, vx, vy, e, rho=None):
    rho = np.ones(mesh.n) if rho is None else rho
    return W.conserved(rho, [vx, vy], (1.4 - 1.0) * rho * e)


def _plane_wave(x, t, mu, lam, k=(1.0, 1.0)):
    k = 2 * np.pi * np.array(k)
    a = np.array([1.0, 0.0]) * 0.1
    kh = k / np.linalg.norm(k)
    apar, aperp = (a @ kh) * kh, a - (a @ kh) * kh
    k2 = k @ k
    s = np.sin(x @ k)
    v = (apar * math.exp(-(4 * mu / 3 + lam) * k2 * t) + aperp * math.exp(-mu * k2 * t))[:, None] * s[None, :]
    return v


@pytest.mark.parametrize("elem", ["q1", "p1", "p1sheared"])
def test_viscous_plane_wave_second_order(elem):
    mu, lam, T = 0.01, 0.02, 0.2
    k = (1.0, 1.0 - SHEAR) if elem == "p1sheared" else (1.0, 1.0)
    errs = []
    for n in (16, 32, 64):
        mesh = _box(n, elem)
        x = mesh.coords
        v0 = _plane_wave(x, 0.0, mu, lam, k)
        U = _state(mesh, v0[0], v0[1], np.full(mesh.n, 10.0))
        o = _orc(mesh, mu, lam, 0.0)
        steps = n // 4
        for _ in range(steps):
            U, _ = o.parabolic_step(U, T / steps)
        v = U[1:3] / U[0]
        ex = _plane_wave(x, T, mu, lam, k)
        errs.append(np.sqrt((mesh.mi * ((v - ex) ** 2).sum(0)).sum()))
    rates = [math.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert min(rates) >= 1.8, (errs, rates)


@pytest.mark.parametrize("elem", ["q1", "p1"])
def test_heat_decay_second_order(elem):
    kc, T = 0.02, 0.25
    errs = []
    for n in (16, 32, 64):
        mesh = _box(n, elem)
        x = mesh.coords[:, 0]
        e0 = 2.0 + 0.5 * np.cos(2 * np.pi * x)
        U = _state(mesh, np.zeros(mesh.n), np.zeros(mesh.n), e0)
        o = _orc(mesh, 0.0, 0.0, kc)
        steps = n // 4
        for _ in range(steps):
            U, _ = o.parabolic_step(U, T / steps)
        e = U[3] / U[0]
        ex = 2.0 + 0.5 * math.exp(-4 * np.pi ** 2 * kc * T) * np.cos(2 * np.pi * x)
        errs.append(np.sqrt((mesh.mi * (e - ex) ** 2).sum()))
    rates = [math.log2(errs[q] / errs[q + 1]) for q in range(2)]
    assert min(rates) >= 1.8, (errs, rates)


def _random_smooth(mesh, seed):
    rng = np.random.default_rng(seed)
    x = mesh.coords
    vx = sum(rng.normal() * np.sin(2 * np.pi * (rng.integers(1, 3) * x[:, 0] + rng.integers(0, 3) * x[:, 1]))
             for _ in range(3))
    vy = sum(rng.normal() * np.cos(2 * np.pi * (rng.integers(0, 3) * x[:, 0] + rng.integers(1, 3) * x[:, 1]))
             for _ in range(3))
    e = 3.0 + np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1])
    rho = 1.0 + 0.3 * np.cos(2 * np.pi * x[:, 1])
    return _state(mesh, vx, vy, e, rho)


@pytest.mark.parametrize("elem", ["q1", "p1"])
def test_conservation_on_a_periodic_box(elem):
    mesh = _box(24, elem)
    U = _random_smooth(mesh, 1)
    o = _orc(mesh, 0.05, 0.03, 0.04)
    U1, info = o.parabolic_step(U, 0.01)
    assert np.array_equal(U1[0], U[0])
    for s in (1, 2, 3):
        assert abs((mesh.mi * U1[s]).sum() - (mesh.mi * U[s]).sum()) <= 1e-11 * (mesh.mi * np.abs(U[s])).sum()
    assert info["cg_iter_velocity"] > 0 and info["limited"] == 0


def test_conservation_with_traction_free_sides():
    """Homogeneous Neumann data for v and e on a non-periodic box: momentum and
    total energy are still conserved (the discrete dissipation a(v, v) equals
    sum_i m_i K_i, and sigma(const) = 0)."""
    mesh = M.structured_q1(14, 10, 0.0, 1.0, 0.0, 0.8)
    x = mesh.coords
    U = _state(mesh, np.sin(2.0 * x[:, 0]) * np.cos(1.5 * x[:, 1]), np.cos(2.5 * x[:, 0] * x[:, 1]),
               3.0 + x[:, 0] * x[:, 1], 1.0 + 0.2 * x[:, 0])
    o = _orc(mesh, 0.05, 0.03, 0.04)
    U1, _ = o.parabolic_step(U, 0.02)
    for s in (1, 2, 3):
        assert abs((mesh.mi * U1[s]).sum() - (mesh.mi * U[s]).sum()) <= 1e-11 * (mesh.mi * np.abs(U[s])).sum()


def test_no_slip_nodes_at_rest_and_energy_conserved_in_a_closed_channel():
    mesh = M.structured_q1(24, 12, 0.0, 2.0, 0.0, 1.0, periodic_x=True)
    wall = mesh.bnd_node  # the walls y = 0, 1
    x = mesh.coords
    vx = np.sin(np.pi * x[:, 1]) * (1.0 + 0.2 * np.cos(np.pi * x[:, 0]))
    vx[wall] = 0.0
    U = _state(mesh, vx, 0.1 * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 0]), np.full(mesh.n, 5.0))
    U[1:3, wall] = 0.0
    o = _orc(mesh, 0.05, 0.0, 0.02, wall=wall)
    U1, _ = o.parabolic_step(U, 0.02)
    assert np.all(U1[1:3, wall] == 0.0)
    E0, E1 = (mesh.mi * U[3]).sum(), (mesh.mi * U1[3]).sum()
    assert abs(E1 - E0) <= 1e-11 * E0
    ke0 = (mesh.mi * (U[1] ** 2 + U[2] ** 2) / U[0]).sum()
    ke1 = (mesh.mi * (U1[1] ** 2 + U1[2] ** 2) / U1[0]).sum()
    assert ke1 < ke0  # viscous dissipation into internal energy


def test_fct_keeps_the_internal_energy_positive():
    """A near-vacuum of internal energy next to hot cells and a long step:
    Crank-Nicolson undershoots below zero; the limited update stays >= the
    minimum of the old e and conserves the total energy."""
    mesh = _box(32, "q1")
    x = mesh.coords
    e = np.where(np.abs(x[:, 0] - 0.5) < 0.1, 50.0, 1e-3)
    U = _state(mesh, np.zeros(mesh.n), np.zeros(mesh.n), e)
    o = _orc(mesh, 0.0, 0.0, 5.0)
    U1, info = o.parabolic_step(U, 0.05)
    e1 = U1[3] / U1[0]
    assert info["limited"] == 1 and info["cg_iter_low"] > 0
    assert e1.min() >= e.min() * (1 - 1e-12)
    assert abs((mesh.mi * U1[3]).sum() - (mesh.mi * U[3]).sum()) <= 1e-11 * (mesh.mi * U[3]).sum()


def test_no_dissipation_is_the_identity():
    mesh = _box(16, "p1")
    U = _random_smooth(mesh, 2)
    o = _orc(mesh, 0.0, 0.0, 0.0)
    U1, info = o.parabolic_step(U, 0.1)
    assert info["cg_iter_velocity"] == 0 and info["cg_iter_energy"] == 0
    assert np.array_equal(U1[:3], U[:3])
    assert np.allclose(U1[3], U[3], rtol=1e-15, atol=0)


def test_strang_step_without_dissipation_is_two_hyperbolic_steps():
    w = W.vortex_workload(24)
    o = oracle.Oracle(w.mesh, cfl=0.5, bound_relaxation=True)
    o.set_viscosity(M.parabolic_data(w.mesh), 0.0, 0.0, 0.0)
    U1, tau, _ = o.ns_step(w.U0)
    ref, tau_ref, _ = o.ssprk3_step(w.U0)
    ref, _, _ = o.ssprk3_step(ref, tau_ref)
    assert tau == tau_ref
    assert np.abs(U1 - ref).max() <= 1e-12 * np.abs(ref).max()
