"""Kept node records and skipped edges. k_prep keeps the record of a node
whose state has the bits it had at the previous stage, and k_visc skips an
edge between two such nodes whose values it stored from equal states: both are
exact, so a context that has been stepping must give, bit for bit, what a
fresh context (whose first stage keeps and skips nothing) gives from the same
state -- after plain steps, a new state set over part of the mesh, a refused
step, eh_cfl_dt and the autotuner, in FP64 and mixed precision, 2D and 3D.
(The merged served batch, whose context is rebuilt over other meshes, is
checked against solves alone in test_gpu_serve.py.) Needs a GPU."""
import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _problem(dim):
    if dim == 2:
        return W.cylinder_problem(14)
    mesh = M.extruded_q1(M.cylinder_channel_q1(10), 6, 0.5)
    U0 = W.uniform_state(mesh, 1.4, (3.0, 0.0, 0.0), 1.0)
    return mesh, U0, np.ascontiguousarray(U0[:, mesh.bnd_node])


def _fresh(mesh, bs, U, steps, precision):
    s = B.Solver(dim=mesh.dim, precision=precision)
    s.upload_mesh(mesh, bs)
    s.set_state(U)
    for _ in range(steps):
        s.step(sync=False)
    out = s.get_state()
    s.close()
    return out


def _steps(s, k):
    for _ in range(k):
        s.step(sync=False)
    return s.get_state()


@pytest.mark.parametrize("precision", [B.EH_PRECISION_FP64, B.EH_PRECISION_MIXED])
@pytest.mark.parametrize("dim", [2, 3])
def test_kept_records_equal_a_fresh_context(dim, precision):
    mesh, U0, bs = _problem(dim)
    s = B.Solver(dim=dim, precision=precision)
    s.upload_mesh(mesh, bs)
    s.set_state(U0)
    s.apply_boundary_conditions()
    U1 = _steps(s, 3)  # a bow shock forming at the cylinder, free stream elsewhere
    # many edges still join equal states: the shortcuts are in use
    i = np.repeat(np.arange(mesh.n), np.diff(mesh.row_ptr))
    off = mesh.col != i
    equal = np.all(U1[:, i[off]] == U1[:, mesh.col[off]], axis=0)
    assert equal.mean() > 0.4
    # (1) plain steps
    assert np.array_equal(_steps(s, 3), _fresh(mesh, bs, U1, 3, precision))
    # (2) a new state that differs from the current one on a band of nodes
    U2 = s.get_state()
    band = slice(mesh.n // 3, mesh.n // 3 + mesh.n // 8)
    U2[:, band] *= 1.01  # rho, m and E scaled together: admissible
    s.set_state(U2)
    assert np.array_equal(_steps(s, 3), _fresh(mesh, bs, U2, 3, precision))
    # (3) a refused step (tau above the CFL limit), the same state set again
    U3 = s.get_state()
    dt = s.cfl_dt()
    with pytest.raises(B.EulerError) as e:
        s.step(dt * 2.5)
    assert e.value.status == B.EH_ERR_CFL
    s.set_state(U3)
    assert np.array_equal(_steps(s, 2), _fresh(mesh, bs, U3, 2, precision))
    # (4) eh_cfl_dt between steps, then the autotuner (which restores the state)
    U4 = s.get_state()
    s.cfl_dt()
    s.autotune(1)
    assert np.array_equal(s.get_state(), U4)
    assert np.array_equal(_steps(s, 2), _fresh(mesh, bs, U4, 2, precision))
    s.close()
