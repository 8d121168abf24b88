"""Pins of the oracle's adaptive CFL step (Sec. 3.1, remark on high
aspect-ratio meshes): a CFL number above 1 is tried first and halved while a
low-order state leaves the admissible set. The accepted step is a plain
SSPRK(3,3) step at the accepted CFL number (bitwise), admissible; CFL numbers
<= 1 never restart (the low-order update is then invariant-domain
preserving). CPU only."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from . import helpers as H


def _admissible(U):
    rho = U[0]
    eps = U[-1] - 0.5 * (U[1:-1] ** 2).sum(0) / rho
    return bool((rho > 0).all() and (eps > 0).all())


@pytest.mark.parametrize("cfl", [0.3, 0.75, 1.0])
def test_cfl_up_to_one_never_restarts(cfl):
    w = W.vortex_workload(24)
    ada = oracle.Oracle(w.mesh, cfl=0.5)
    plain = oracle.Oracle(w.mesh, cfl=cfl)
    U, dt, c, r = ada.ssprk3_step_adaptive(w.U0, cfl)
    ref, dt_ref, _ = plain.ssprk3_step(w.U0)
    assert r == 0 and c == cfl and dt == dt_ref
    assert np.array_equal(U, ref)


def test_strong_shock_restarts_until_admissible():
    mesh = W.riemann_strip(120)
    U0 = W.riemann_initial(mesh, "strong_shock")
    ada = oracle.Oracle(mesh, cfl=0.5)
    U, dt, c, r = ada.ssprk3_step_adaptive(U0, 16.0)
    assert r >= 1 and c == 16.0 / 2 ** r and c < 16.0
    assert _admissible(U)
    ref, dt_ref, _ = oracle.Oracle(mesh, cfl=c).ssprk3_step(U0)
    assert dt == dt_ref and np.array_equal(U, ref)
    # the accepted step: every stage's low-order state is admissible
    _, _, stages = H.ssprk3_with_traces(oracle.Oracle(mesh, cfl=c), U0)
    assert all(_admissible(tr["UL"]) for _, _, tr in stages)
    # the rejected CFL number: some stage's low-order state (or a stage input)
    # leaves the admissible set -- replayed stage by stage with traces
    try:
        _, _, stages = H.ssprk3_with_traces(oracle.Oracle(mesh, cfl=2 * c), U0)
        rejected_ok = any(not _admissible(tr["UL"]) for _, _, tr in stages)
    except oracle.OracleError:
        rejected_ok = True
    assert rejected_ok


def test_adaptive_steps_advance_a_smooth_flow_at_high_cfl():
    """Away from shocks the low-order update stays admissible well above
    c_cfl = 1 on this mesh: 10 steps at cfl_max = 1.5 pass without restart and
    stay admissible and conservative (periodic box)."""
    w = W.vortex_workload(24)
    ada = oracle.Oracle(w.mesh, cfl=0.5)
    U = w.U0
    mass0 = (w.mesh.mi * U[0]).sum()
    for _ in range(10):
        U, dt, c, r = ada.ssprk3_step_adaptive(U, 1.5)
        assert r == 0 and c == 1.5
    assert _admissible(U)
    assert abs((w.mesh.mi * U[0]).sum() - mass0) <= 1e-12 * mass0
