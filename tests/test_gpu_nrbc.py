"""Non-reflecting boundary post-processing (Sec. 4.2) on the GPU against the
oracle: node by node on states that cover all four characteristic regimes,
and SSPRK(3,3) runs of the vortex leaving [-1,1]^2 (Sec. 6) with either
post-processing on all four sides. Needs a GPU."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from .test_gpu_parity import RUN_TOL, STEP_TOL, fma_twin, oracle_spread, rel_l1, solver_for, tolerance

pytestmark = pytest.mark.gpu

KINDS = {"characteristic": M.BC_CHARACTERISTIC, "godunov": M.BC_GODUNOV}


def _regime_states(mesh, seed):
    """Admissible states whose velocity at every node is random in direction
    and in magnitude up to 3 sound speeds (inflow/outflow, sub/supersonic)."""
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(-0.5, 0.5, mesh.n))
    p = np.exp(rng.uniform(-0.5, 0.5, mesh.n))
    a = np.sqrt(1.4 * p / rho)
    th = rng.uniform(0, 2 * np.pi, mesh.n)
    sp = rng.uniform(0, 3, mesh.n) * a
    return W.conserved(rho, [sp * np.cos(th), sp * np.sin(th)], p)


@pytest.mark.parametrize("kind", sorted(KINDS))
def test_post_processing_matches_oracle_node_by_node(kind):
    mesh, _, bs = W.nrbc_vortex_problem(12, "i", KINDS[kind])
    orc = oracle.Oracle(mesh, cfl=0.75, bnd_state=bs)
    s = solver_for(mesh, bs, cfl=0.75)
    regimes = set()
    for seed in range(6):
        U = _regime_states(mesh, seed)
        s.set_state(U)
        s.apply_boundary_conditions()
        got, ref = s.get_state(), orc.apply_bc(U)
        b = mesh.bnd_node
        scale = np.abs(ref[:, b]).max(axis=0)
        assert np.all(np.abs(got[:, b] - ref[:, b]) <= 1e-13 * scale), kind
        inside = np.setdiff1d(np.arange(mesh.n), b)
        assert np.array_equal(got[:, inside], U[:, inside])
        rho, vn = U[0, b], (U[1:3, b] * mesh.bnd_normal).sum(0) / U[0, b]
        a = np.sqrt(1.4 * (0.4 * (U[3, b] - 0.5 * (U[1, b] ** 2 + U[2, b] ** 2) / rho)) / rho)
        regimes |= set(np.where(vn < 0, np.where(-vn > a, 1, 2), np.where(vn >= a, 4, 3)).tolist())
    assert regimes == {1, 2, 3, 4}  # supersonic/subsonic inflow, subsonic/supersonic outflow


@pytest.mark.parametrize("kind", sorted(KINDS))
@pytest.mark.parametrize("case", ["i", "iii"])
def test_vortex_leaving_the_box_matches_oracle(kind, case):
    """Strict bounds (the paper's), CFL 0.75: held to max(target, 100 x the
    oracle's own spread), as every strict-bound run."""
    steps = 120 if case == "i" else 900  # the vortex centre reaches x = 1 near t = 1
    mesh, U0, bs = W.nrbc_vortex_problem(16, case, KINDS[kind])
    orc = oracle.Oracle(mesh, cfl=0.75, bnd_state=bs)
    U0 = orc.apply_bc(U0)
    ref1 = orc.ssprk3_step(U0)[0]
    ref, _ = orc.run(U0, steps)
    s = solver_for(mesh, bs, cfl=0.75)
    s.set_state(U0)
    s.step()
    err1 = rel_l1(s.get_state(), ref1).max()
    s.set_state(U0)
    s.run(steps)
    err = rel_l1(s.get_state(), ref).max()
    assert s.diagnostics()["not_admissible"] == 0
    orf = fma_twin(orc, mesh, bs, cfl=0.75)
    spread1 = oracle_spread(lambda U: orc.ssprk3_step(U)[0], U0, fn_fma=lambda U: orf.ssprk3_step(U)[0])
    spread = oracle_spread(lambda U: orc.run(U, steps)[0], U0, fn_fma=lambda U: orf.run(U, steps)[0])
    assert err1 <= tolerance(STEP_TOL, spread1), (err1, spread1)
    assert err <= tolerance(RUN_TOL, spread), (err, spread)
