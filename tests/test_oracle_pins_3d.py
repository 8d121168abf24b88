"""Pins of the oracle's 3D path (Q1 hexes, 27-point rows; the dimension only
changes loop lengths and the mesh, so these mirror the 2D pins): uniform
states are exact fixed points, sum_i m_i U_i is conserved on a periodic box
and mass and energy in a closed slip box (Lemma 4.5), x-invariant data stay
invariant with zero transverse momentum, and a shock tube along x converges
to the exact Riemann solution. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from . import riemann_exact as RE

GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(0)


def _smooth_state(mesh, seed, amp=0.2):
    """Positive smooth seeded perturbation of a state at rest-ish (periodic in
    the unit box)."""
    rng = np.random.default_rng(seed)
    x, y, z = (mesh.coords[:, d] for d in range(3))
    ph = rng.uniform(0.0, 2.0 * np.pi, 6)
    s = lambda k, a, b: np.sin(2 * np.pi * a + ph[k]) * np.cos(2 * np.pi * b + ph[k + 1])  # noqa: E731
    rho = 1.0 + amp * s(0, x, y + z)
    vel = [0.3 * s(1, y, z), 0.2 * s(2, z, x), 0.25 * s(3, x, z)]
    p = 1.0 + amp * s(4, x + y, z)
    return W.conserved(rho, vel, p, GAMMA)


def test_uniform_states_are_exact_fixed_points_3d():
    box = M.structured_q1_3d(6, 5, 4, periodic=(True, True, True))
    slab = M.structured_q1_3d(6, 4, 3, periodic=(True, False, False), kinds=(M.BC_SLIP,) * 6)
    for mesh, vel in ((box, (0.7, -0.4, 0.2)), (slab, (0.9, 0.0, 0.0))):
        U = W.uniform_state(mesh, 1.3, vel, 2.0)
        orc = oracle.Oracle(mesh)
        U20, _ = orc.run(U, 20)
        assert np.array_equal(U20, U)


def test_periodic_box_conserves_every_component_3d():
    mesh = M.structured_q1_3d(8, 7, 6, periodic=(True, True, True))
    U0 = _smooth_state(mesh, 3)
    orc = oracle.Oracle(mesh)
    U, _ = orc.run(U0, 10)
    scale = (mesh.mi * np.abs(U0)).sum(1)
    assert np.all(np.abs((mesh.mi * U).sum(1) - (mesh.mi * U0).sum(1)) <= 1e-13 * scale)
    assert orc.count_not_admissible(U) == 0


def test_closed_slip_box_conserves_mass_and_energy_3d():
    """Lemma 4.5: with slip on every face, mass and total energy are conserved
    (momentum is not: the walls push back)."""
    mesh = M.structured_q1_3d(7, 6, 5, kinds=(M.BC_SLIP,) * 6)
    orc = oracle.Oracle(mesh)
    U0 = orc.apply_bc(_smooth_state(mesh, 5))
    U, _ = orc.run(U0, 10)
    for s in (0, 4):
        scale = (mesh.mi * np.abs(U0[s])).sum()
        assert abs((mesh.mi * U[s]).sum() - (mesh.mi * U0[s]).sum()) <= 1e-13 * scale, s


def _tube(nx, case):
    mesh = M.structured_q1_3d(nx, 2, 2, box=((0.0, 1.0), (0.0, 2.0 / nx), (0.0, 2.0 / nx)),
                              periodic=(False, True, True), kinds=(M.BC_DO_NOTHING,) * 2 + (M.BC_SLIP,) * 4)
    rl, ul, pl, rr, ur, pr, t_end = W.RIEMANN_CASES[case]
    x = mesh.coords[:, 0]
    left, mid = x < 0.5, np.isclose(x, 0.5)
    z = np.zeros(mesh.n)
    U = W.conserved(np.where(left, rl, rr), [np.where(left, ul, ur), z, z], np.where(left, pl, pr), GAMMA)
    if mid.any():
        UL = W.conserved(np.array([rl]), [np.array([ul]), np.zeros(1), np.zeros(1)], np.array([pl]), GAMMA)
        UR = W.conserved(np.array([rr]), [np.array([ur]), np.zeros(1), np.zeros(1)], np.array([pr]), GAMMA)
        U[:, mid] = 0.5 * (UL + UR)
    return mesh, U, t_end


def test_x_invariant_data_stay_one_dimensional_3d():
    """A shock tube along x: the solution stays constant on every x-plane and
    the y and z momenta stay 0 (to roundoff: the transverse c_ij of a row
    cancel only up to the rounding of the quadrature)."""
    mesh, U0, t_end = _tube(64, "sod")
    # relaxed bounds: with strict bounds the limiter amplifies the roundoff
    # that tells the nodes of a plane apart to ~1e-8 (section on conditioning)
    orc = oracle.Oracle(mesh, bound_relaxation=True)
    U, _, _ = orc.run_to(U0, t_end)
    mx = np.abs(U[1]).max()
    assert np.abs(U[2]).max() <= 1e-12 * mx and np.abs(U[3]).max() <= 1e-12 * mx
    x = np.round(mesh.coords[:, 0] * 64).astype(int)
    for s in (0, 1, 4):
        per_plane = np.full(65, -np.inf)
        np.maximum.at(per_plane, x, U[s])
        lo = np.full(65, np.inf)
        np.minimum.at(lo, x, U[s])
        assert np.all(per_plane - lo <= 1e-12 * np.abs(per_plane).max()), s


@pytest.mark.parametrize("case", ["sod", "lax"])
def test_shock_tube_converges_to_exact_solution_3d(case):
    """L1 density error along x decreases at a rate >= 0.6, as on the 2D strip."""
    data = W.RIEMANN_CASES[case]
    errs = []
    for nx in (100, 200, 400):
        mesh, U0, t_end = _tube(nx, case)
        orc = oracle.Oracle(mesh)
        U, t, _ = orc.run_to(U0, t_end)
        rho, _, _ = RE.sample(mesh.coords[:, 0], t, *data[:6])
        errs.append((mesh.mi * np.abs(U[0] - rho)).sum() / (mesh.mi * rho).sum())
        assert orc.count_not_admissible(U) == 0
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates >= 0.6), (errs, rates)
    assert errs[-1] < {"sod": 0.01, "lax": 0.02}[case]
