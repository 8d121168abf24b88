"""Failure detection and checkpoint/resume through the C ABI. Faults are made
on the host (corrupted inputs, a too-large dt); nothing here faults, traps or
hangs the GPU. Needs a GPU."""
import dataclasses

import numpy as np
import pytest

from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver(mesh, bs=None, **kw):
    s = B.Solver(dim=mesh.dim, **kw)
    s.upload_mesh(mesh, bs)
    return s


@pytest.mark.parametrize("precision", [B.EH_PRECISION_FP64, B.EH_PRECISION_MIXED])
def test_checkpoint_resume_is_bitwise(precision):
    """10 steps, get_state, a new context, set_state, 10 steps == 20 steps."""
    mesh, U0, bs = W.cylinder_problem(12)
    a = _solver(mesh, bs, precision=precision)
    a.set_state(U0)
    a.apply_boundary_conditions()
    a.run(20)
    ref = a.get_state()
    b = _solver(mesh, bs, precision=precision)
    b.set_state(U0)
    b.apply_boundary_conditions()
    b.run(10)
    ckpt = b.get_state()
    b.close()
    c = _solver(mesh, bs, precision=precision)
    c.set_state(ckpt)
    c.run(10)
    assert np.array_equal(c.get_state(), ref)


def test_corrupted_mesh_data_is_rejected_on_the_host():
    mesh = M.periodic_p1_square(8)
    s = B.Solver()
    bad = [
        dataclasses.replace(mesh, mi=np.where(np.arange(mesh.n) == 3, -1.0, mesh.mi)),
        dataclasses.replace(mesh, cij=np.where(np.arange(mesh.nnz) == 5, np.nan, mesh.cij)),
        dataclasses.replace(mesh, col=np.where(np.arange(mesh.nnz) == 7, mesh.n + 4, mesh.col).astype(np.int32)),
        # the consistent mass matrix must be symmetric (m_ij = int phi_i phi_j);
        # entry 9 is off the diagonal (row 1, column 2)
        dataclasses.replace(mesh, mij=np.where(np.arange(mesh.nnz) == 9, mesh.mij * (1.0 + 1e-6), mesh.mij)),
    ]
    for m in bad:
        with pytest.raises(B.EulerError) as e:
            s.upload_mesh(m)
        assert e.value.status == B.EH_ERR_BAD_MESH
    cyl = M.cylinder_channel_q1(6)
    with pytest.raises(B.EulerError) as e:
        s.upload_mesh(dataclasses.replace(cyl, bnd_kind=np.full(cyl.n_bnd, 9, dtype=np.int32)))
    assert e.value.status == B.EH_ERR_BAD_MESH
    with pytest.raises(B.EulerError) as e:  # Dirichlet nodes without Dirichlet states
        s.upload_mesh(cyl, None)
    assert e.value.status == B.EH_ERR_BAD_MESH


def test_corrupted_states_are_rejected():
    w = W.vortex_workload(16)
    s = _solver(w.mesh)
    for k, v in ((0, np.nan), (0, 0.0), (3, -5.0)):  # NaN density, zero density, negative internal energy
        U = w.U0.copy()
        U[k, 11] = v
        with pytest.raises(B.EulerError) as e:
            s.set_state(U)
        assert e.value.status == B.EH_ERR_NOT_ADMISSIBLE
    s.set_state(w.U0)
    s.step()


def test_invalid_sizes_are_rejected():
    s = B.Solver()
    lib = s.lib
    import ctypes
    one = np.zeros(4)
    p = one.ctypes.data_as(ctypes.c_void_p)
    assert lib.eh_upload_mesh(s.ctx, 0, 1, p, p, p, p, p, 0, None, None, None, None) == B.EH_ERR_INVALID_ARG
    assert lib.eh_upload_mesh(s.ctx, 4, 1 << 31, p, p, p, p, p, 0, None, None, None, None) == B.EH_ERR_INVALID_ARG
    assert lib.eh_step(s.ctx, 0.0, None) == B.EH_ERR_STATE
