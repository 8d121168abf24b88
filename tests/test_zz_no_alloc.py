"""The allocation-free CFL step (eh_cfl_dt_noalloc) against the context-based
one (eh_cfl_dt) and against the oracle's CFL step (eq. dtCfl).

eh_cfl_dt_noalloc serves callers that may not allocate device memory (a host
framework that owns all device memory, a real-time loop); its only scratch is a
file-scope device array shared by all calls. This file is collected last so
that a failure here does not hide the other tests, and it passes alone or after
them. Needs a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DT_TOL = 1e-13  # the relative tolerance of the CFL step in the parity tests


def _device_mesh(torch, mesh):
    dev = torch.device("cuda", 0)
    isb = np.zeros(mesh.n, dtype=np.uint8)
    isb[mesh.bnd_node] = 1
    return dict(
        row_ptr=torch.as_tensor(np.ascontiguousarray(mesh.row_ptr, dtype=np.int64), device=dev),
        col=torch.as_tensor(np.ascontiguousarray(mesh.col, dtype=np.int32), device=dev),
        cij=torch.as_tensor(np.ascontiguousarray(mesh.cij), device=dev),
        mi=torch.as_tensor(np.ascontiguousarray(mesh.mi), device=dev),
        is_boundary=torch.as_tensor(isb, device=dev) if mesh.n_bnd else None)


@pytest.mark.parametrize("case", ["vortex", "cylinder", "box3d"])
def test_noalloc_cfl_step_matches_context_path_twice(case):
    torch = pytest.importorskip("torch")
    B.build()
    if case == "vortex":
        mesh = M.periodic_p1_square(48)
        states = [W.isentropic_vortex(mesh), W.isentropic_vortex(mesh, t=1.3)]
        bs = None
    elif case == "cylinder":
        mesh, _, bs = W.cylinder_problem(14)
        states = [W.perturbed_state(mesh, 1), W.perturbed_state(mesh, 2)]
    else:
        mesh = M.structured_q1_3d(7, 5, 4, kinds=(M.BC_SLIP,) * 6)
        base = dict(rho=1.0, vel=(0.4, 0.1, -0.2), p=1.0)
        states = [W.perturbed_state(mesh, s, base=base, amplitude=0.2) for s in (3, 4)]
        bs = None
    dm = _device_mesh(torch, mesh)
    solver = B.Solver(dim=mesh.dim, cfl=0.5)
    solver.upload_mesh(mesh, bs)
    orc = oracle.Oracle(mesh, cfl=0.5, bnd_state=bs)
    dt_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    for U in states:  # two calls in a row share the scratch array
        solver.set_state(U)
        expect = solver.cfl_dt()
        ref = orc.cfl_dt(U)
        Ud = torch.as_tensor(np.ascontiguousarray(U), device="cuda")
        B.cfl_dt_noalloc(mesh.dim, 1.4, 0.5, dm["row_ptr"], dm["col"], dm["cij"], dm["mi"], dm["is_boundary"], Ud,
                         dt_out)
        torch.cuda.synchronize()
        got = float(dt_out.item())
        assert abs(got - expect) <= DT_TOL * expect, (got, expect)
        assert abs(got - ref) <= DT_TOL * ref, (got, ref)


def test_noalloc_reports_a_non_admissible_row_as_nan():
    """A row whose internal energy is negative has no wave speed: the step is
    NaN, not the minimum over the other rows."""
    torch = pytest.importorskip("torch")
    B.build()
    mesh, _, _ = W.cylinder_problem(10)
    U = W.perturbed_state(mesh, 3)
    dm = _device_mesh(torch, mesh)
    dt_out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    Ud = torch.as_tensor(np.ascontiguousarray(U), device="cuda")
    B.cfl_dt_noalloc(2, 1.4, 0.5, dm["row_ptr"], dm["col"], dm["cij"], dm["mi"], dm["is_boundary"], Ud, dt_out)
    torch.cuda.synchronize()
    assert np.isfinite(float(dt_out.item()))
    bad = U.copy()
    bad[3, mesh.n // 2] = 0.25 * (bad[1, mesh.n // 2] ** 2 + bad[2, mesh.n // 2] ** 2) / bad[0, mesh.n // 2]
    Ud = torch.as_tensor(np.ascontiguousarray(bad), device="cuda")
    B.cfl_dt_noalloc(2, 1.4, 0.5, dm["row_ptr"], dm["col"], dm["cij"], dm["mi"], dm["is_boundary"], Ud, dt_out)
    torch.cuda.synchronize()
    assert np.isnan(float(dt_out.item()))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    B.build()
    lib = B.load()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.eh_cfl_dt_noalloc(2, 1.4, 0.5, B.CFL_NOALLOC_MAX_ROWS + 1, 10, dummy, dummy, dummy, dummy, None, dummy,
                               dummy, None)
    assert st == B.EH_ERR_INVALID_ARG
