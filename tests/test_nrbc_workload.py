"""The non-reflecting vortex workload (Sec. 6) and its diagnostics: the
initial state is a steady vortex in the frame moving with the free stream
(radial balance dp/dr = rho v_theta^2 / r), delta_1(0) = vbar and
delta_2(0) = 1. CPU only."""
import numpy as np
import pytest

import bench
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W


@pytest.mark.parametrize("case", sorted(W.NRBC_CASES))
def test_vortex_is_in_radial_balance(case):
    mach, vbar = W.NRBC_CASES[case]
    r = np.linspace(0.0, 0.6, 601)
    x = np.stack([r, np.zeros_like(r)], 1)  # along +x: v_theta = v_y
    U = W.nrbc_vortex_state(x, mach, vbar)
    rho = U[0]
    vth = U[2] / rho
    p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    dpdr = np.gradient(p, r)
    lhs, rhs = dpdr[5:-5], (rho * vth ** 2 / np.maximum(r, 1e-12))[5:-5]
    assert np.abs(lhs - rhs).max() <= 1e-3 * np.abs(rhs).max()
    assert np.isclose(np.abs(vth).max(), vbar, rtol=1e-4)  # the peak perturbation, at r = r0
    assert np.isclose(p[-1], (1.0 / mach) ** 2 / 1.4, rtol=1e-6)


def test_deltas_at_time_zero():
    mesh, U0, bs = W.nrbc_vortex_problem(40, "ii", M.BC_GODUNOV)
    assert set(np.unique(mesh.bnd_kind)) == {M.BC_GODUNOV}
    assert bs.shape == (4, mesh.bnd_node.size)
    v0 = U0[1:3] / U0[0]
    rows = mesh.row_of_entry()
    c0 = np.bincount(rows, weights=mesh.cij[0] * v0[1, mesh.col] - mesh.cij[1] * v0[0, mesh.col],
                     minlength=mesh.n) / mesh.mi
    d1, d2 = bench.nrbc_deltas(mesh, U0, float(np.abs(c0).max()))
    assert np.isclose(d1, W.NRBC_CASES["ii"][1], rtol=1e-3) and d2 == 1.0
