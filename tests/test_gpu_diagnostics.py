"""The state statistics of eh_get_diagnostics: min rho, min specific internal
energy and the lumped totals sum_i m_i U_i, against numpy on the state the
library returns; the totals are constant on a periodic mesh (no boundary
flux: conservation, Lemma 3.1) and are the same bits on repeated calls. Needs
a GPU."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _stats(mesh, U):
    rho = U[0]
    m2 = (U[1:-1] ** 2).sum(axis=0)
    e = U[-1] / rho - 0.5 * m2 / rho ** 2
    return rho.min(), e.min(), (mesh.mi[None, :] * U).sum(axis=1)


@pytest.mark.parametrize("case", ["vortex", "cylinder"])
def test_state_statistics_match_numpy(case):
    if case == "vortex":
        w = W.vortex_workload(40)
        mesh, U0, bs = w.mesh, w.U0, None
    else:
        mesh, U0, bs = W.cylinder_problem(12)
        U0 = W.perturbed_state(mesh, 4)
    s = B.Solver(dim=mesh.dim)
    s.upload_mesh(mesh, bs)
    assert s.diagnostics()["rho_min"] == 0.0  # no state yet
    s.set_state(U0)
    s.apply_boundary_conditions()
    s.run(7)
    d = s.diagnostics()
    U = s.get_state()
    rho_min, e_min, total = _stats(mesh, U)
    assert d["rho_min"] == rho_min
    assert abs(d["e_min"] - e_min) <= 1e-14 * abs(e_min)
    scale = (mesh.mi[None, :] * np.abs(U)).sum(axis=1)
    assert np.all(np.abs(np.array(d["total"]) - total) <= 1e-13 * scale)
    assert s.diagnostics()["total"] == d["total"]  # deterministic


def test_totals_are_conserved_on_a_periodic_mesh():
    w = W.vortex_workload(32)
    s = B.Solver(dim=2)
    s.upload_mesh(w.mesh, None)
    s.set_state(w.U0)
    before = np.array(s.diagnostics()["total"])
    s.run(40)
    after = np.array(s.diagnostics()["total"])
    scale = (w.mesh.mi[None, :] * np.abs(w.U0)).sum(axis=1)
    assert np.all(np.abs(after - before) <= 1e-12 * scale), (after - before) / scale
