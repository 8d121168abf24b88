"""The parabolic sub-step (Sec. 5) and the Strang-split Navier-Stokes step on
the GPU against the oracle: Crank-Nicolson solves by CG on both sides to a
relative residual of 1e-13, so states agree to ~1e-11; the FCT branch,
no-slip walls, P1 and Q1 meshes; Navier-Stokes steps on the vortex (relaxed
bounds) and on the cylinder with no-slip walls (strict bounds, held like every
strict-bound run to 100 x the oracle's own spread). Needs a GPU."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from .test_gpu_parity import RUN_TOL, fma_twin, oracle_spread, rel_l1, solver_for, tolerance
from .test_oracle_parabolic import _box, _random_smooth, _state

pytestmark = pytest.mark.gpu

PAR_TOL = 1e-11


def _pair(mesh, mu, lam, kc, wall=None, bs=None, **kw):
    pdata = M.parabolic_data(mesh)
    o = oracle.Oracle(mesh, bnd_state=bs, **kw)
    o.set_viscosity(pdata, mu, lam, kc, wall=wall)
    s = solver_for(mesh, bs, **kw)
    s.set_viscosity(pdata, mu, lam, kc, wall=wall)
    return o, s


@pytest.mark.parametrize("elem", ["q1", "p1sheared"])
def test_parabolic_step_matches_oracle(elem):
    mesh = _box(24, elem)
    U = _random_smooth(mesh, 3)
    o, s = _pair(mesh, 0.05, 0.03, 0.04)
    ref, info_o = o.parabolic_step(U, 0.01)
    s.set_state(U)
    info = s.parabolic_step(0.01)
    assert info["limited"] == info_o["limited"] == 0
    assert abs(info["cg_iter_velocity"] - info_o["cg_iter_velocity"]) <= 1
    assert rel_l1(s.get_state(), ref).max() <= PAR_TOL


def test_cg_batching_leaves_the_result_bitwise_unchanged():
    # the first solve queues CG iterations in a batch of the default length,
    # the repeat in a batch as long as the first solve took: iterations queued
    # past convergence must do nothing
    mesh = _box(24, "q1")
    U = _random_smooth(mesh, 3)
    _, s = _pair(mesh, 0.05, 0.03, 0.04)
    s.set_state(U)
    info1 = s.parabolic_step(0.01)
    first = s.get_state()
    s.set_state(U)
    info2 = s.parabolic_step(0.01)
    assert info1 == info2
    assert np.array_equal(s.get_state(), first)


def test_fct_branch_matches_oracle():
    mesh = _box(32, "q1")
    x = mesh.coords
    e = np.where(np.abs(x[:, 0] - 0.5) < 0.1, 50.0, 1e-3)
    U = _state(mesh, np.zeros(mesh.n), np.zeros(mesh.n), e)
    o, s = _pair(mesh, 0.0, 0.0, 5.0)
    ref, info_o = o.parabolic_step(U, 0.05)
    s.set_state(U)
    info = s.parabolic_step(0.05)
    assert info["limited"] == info_o["limited"] == 1
    got = s.get_state()
    assert rel_l1(got, ref).max() <= PAR_TOL
    assert (got[3] / got[0]).min() >= e.min() * (1 - 1e-12)
    assert np.isclose(info["min_e"], info_o["min_e"], rtol=1e-10)


def test_no_slip_channel_matches_oracle():
    mesh = M.structured_q1(24, 12, 0.0, 2.0, 0.0, 1.0, periodic_x=True)
    wall = mesh.bnd_node
    x = mesh.coords
    vx = np.sin(np.pi * x[:, 1]) * (1.0 + 0.2 * np.cos(np.pi * x[:, 0]))
    U = _state(mesh, vx, 0.1 * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 0]), np.full(mesh.n, 5.0))
    U[1:3, wall] = 0.0
    o, s = _pair(mesh, 0.05, 0.0, 0.02, wall=wall)
    ref, _ = o.parabolic_step(U, 0.02)
    s.set_state(U)
    s.parabolic_step(0.02)
    got = s.get_state()
    assert np.all(got[1:3, wall] == 0.0)
    assert rel_l1(got, ref).max() <= PAR_TOL


def test_navier_stokes_steps_vortex_relaxed():
    w = W.vortex_workload(32)
    o, s = _pair(w.mesh, 2e-3, 0.0, 3e-3, bound_relaxation=True)
    U = w.U0
    s.set_state(U)
    for _ in range(5):
        U, tau_o, _ = o.ns_step(U)
        tau, info = s.step_ns()
        assert abs(tau - tau_o) <= 1e-12 * tau_o
    assert rel_l1(s.get_state(), U).max() <= 1e-10


def test_navier_stokes_steps_cylinder_no_slip():
    mesh, U0, bs = W.cylinder_problem(12)
    wall = mesh.bnd_node[mesh.bnd_kind == M.BC_SLIP]
    U0 = W.perturbed_state(mesh, 7)
    o, s = _pair(mesh, 1e-3, 0.0, 1e-3, wall=wall, bs=bs)
    U0 = o.apply_bc(U0)
    U0[1:3, wall] = 0.0
    ref = U0
    for _ in range(3):
        ref, _, _ = o.ns_step(ref)
    s.set_state(U0)
    for _ in range(3):
        s.step_ns()
    err = rel_l1(s.get_state(), ref).max()
    orf = fma_twin(o, mesh, bs)
    orf.set_viscosity(M.parabolic_data(mesh), 1e-3, 0.0, 1e-3, wall=wall)

    def run(fn_orc, U):
        for _ in range(3):
            U, _, _ = fn_orc.ns_step(U)
        return U
    spread = oracle_spread(lambda U: run(o, U), U0, fn_fma=lambda U: run(orf, U))
    assert err <= tolerance(RUN_TOL, spread), (err, spread)
    assert s.diagnostics()["not_admissible"] == 0
