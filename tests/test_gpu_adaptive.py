"""The adaptive CFL step (Sec. 3.1, remark on high aspect-ratio meshes) on the
GPU against the oracle: the same restarts and accepted CFL number, the same
state; CFL numbers <= 1 never restart and equal a plain step; the low-order
admissibility counter stays 0 for plain steps. Needs a GPU.

Above c_cfl = 1 the step is outside the CFL condition of Sec. 3.1 that makes
U^L a convex combination of the bar states: U^L can leave the local bounds,
and the line search then clamps l to 0 or 1 on entries whose bound is met to
rounding, so the state is not a continuous function of the arithmetic. An FP64
CPU build of the same algorithm with the flux differences written in the
algebraically equal form (X_j - X_i)(v_j.c) + X_i (v_j - v_i).c moves by
3.8e-11 (Lax, c = 6), 1.6e-10 (strong shock) and, with the SSP combinations
also rounded in their other form, 1.3e-8; accepted steps above 1 are held to
C_ABOVE_ONE_TOL, steps at c <= 1 to the strict parity bar."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import workloads as W

from .test_gpu_parity import STEP_TOL, fma_twin, oracle_spread, rel_l1, solver_for, tolerance

pytestmark = pytest.mark.gpu

C_ABOVE_ONE_TOL = 1e-7


def test_cfl_up_to_one_equals_a_plain_step():
    w = W.vortex_workload(24)
    a = solver_for(w.mesh)
    a.set_state(w.U0)
    dt, c, r = a.step_adaptive(0.75)
    p = solver_for(w.mesh, cfl=0.75)
    p.set_state(w.U0)
    dt_p = p.step()
    assert r == 0 and c == 0.75 and dt == dt_p
    assert np.array_equal(a.get_state(), p.get_state())


@pytest.mark.parametrize("case,cfl_max", [("strong_shock", 16.0), ("sod", 8.0), ("lax", 6.0)])
def test_restarts_match_the_oracle(case, cfl_max):
    mesh = W.riemann_strip(120)
    U0 = W.riemann_initial(mesh, case)
    orc = oracle.Oracle(mesh, cfl=0.5)
    ref, dt_ref, c_ref, r_ref = orc.ssprk3_step_adaptive(U0, cfl_max)
    s = solver_for(mesh)
    s.set_state(U0)
    dt, c, r = s.step_adaptive(cfl_max)
    assert (r, c) == (r_ref, c_ref)
    assert abs(dt - dt_ref) <= 1e-13 * dt_ref
    err = rel_l1(s.get_state(), ref).max()
    plain = oracle.Oracle(mesh, cfl=c)
    orf = fma_twin(plain, mesh, None, cfl=c)
    spread = oracle_spread(lambda U: plain.ssprk3_step(U)[0], U0, fn_fma=lambda U: orf.ssprk3_step(U)[0])
    assert err <= (tolerance(STEP_TOL, spread) if c <= 1.0 else max(C_ABOVE_ONE_TOL, 100.0 * spread)), (err, spread)
    d = s.diagnostics()
    assert d["not_admissible"] == 0 and d["low_order_not_admissible"] == 0


def test_time_is_restored_on_restart_and_advanced_once():
    mesh = W.riemann_strip(120)
    U0 = W.riemann_initial(mesh, "strong_shock")
    s = solver_for(mesh)
    s.set_state(U0)
    dt, c, r = s.step_adaptive(16.0)
    assert r >= 1
    assert s.instances()["t"][0] == dt


def test_plain_steps_keep_low_order_states_admissible():
    mesh, U0, bs = W.cylinder_problem(16)
    s = solver_for(mesh, bs)
    s.set_state(W.perturbed_state(mesh, 3))
    s.apply_boundary_conditions()
    s.run(30)
    d = s.diagnostics()
    assert d["low_order_not_admissible"] == 0 and d["not_admissible"] == 0


def test_adaptive_step_rejects_bad_arguments():
    w = W.vortex_workload(16)
    s = solver_for(w.mesh)
    s.set_state(w.U0)
    for bad in (0.0, -1.0, 65.0):
        with pytest.raises(B.EulerError):
            s.step_adaptive(bad)
