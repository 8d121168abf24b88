"""Pins of the seeded inputs: finite-element identities of Sec. 2.2 and the
initial data of the vortex workload. CPU only."""
import math

import numpy as np
import pytest

from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W


def _row_sums(mesh, vals):
    return np.bincount(mesh.row_of_entry(), weights=vals, minlength=mesh.n)


MESHES = {
    "p1": lambda: M.periodic_p1_square(16),
    "q1_periodic": lambda: M.structured_q1(12, 8, periodic_x=True, periodic_y=True),
    "q1_strip": lambda: W.riemann_strip(20),
    "q1_cylinder": lambda: M.cylinder_channel_q1(12),
}


@pytest.fixture(params=sorted(MESHES))
def mesh(request):
    return MESHES[request.param]()


def test_partition_of_unity_identities(mesh):
    """Sec. 2.2: m_i = sum_j m_ij and sum_j c_ij = 0."""
    assert np.allclose(_row_sums(mesh, mesh.mij), mesh.mi, rtol=1e-13, atol=1e-15)
    scale = np.abs(mesh.cij).max()
    for d in range(mesh.dim):
        assert np.abs(_row_sums(mesh, mesh.cij[d])).max() <= 1e-13 * scale


def test_column_sums_are_boundary_normals(mesh):
    """sum_i c_ij = int grad phi_j = int_bnd phi_j n = m^bnd_j n_j (eq. unit_normal_vector)."""
    cs = np.stack([np.bincount(mesh.col, weights=mesh.cij[d], minlength=mesh.n) for d in range(mesh.dim)])
    expect = np.zeros_like(cs)
    expect[:, mesh.bnd_node] = mesh.bnd_mass_full * mesh.bnd_normal_full
    assert np.abs(cs - expect).max() <= 1e-13 * max(1.0, np.abs(mesh.cij).max())


def test_pattern_symmetric_sorted_with_diagonal(mesh):
    rows = mesh.row_of_entry()
    key = set(zip(rows.tolist(), mesh.col.tolist()))
    assert all((j, i) in key for i, j in key)
    for i in range(mesh.n):
        seg = mesh.col[mesh.row_ptr[i]:mesh.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0) and i in seg


def test_cij_antisymmetric_for_interior_pairs(mesh):
    """c_ij + c_ji = int_bnd phi_i phi_j n, which vanishes unless both are boundary nodes."""
    rows = mesh.row_of_entry()
    pos = {(i, j): k for k, (i, j) in enumerate(zip(rows.tolist(), mesh.col.tolist()))}
    bnd = np.zeros(mesh.n, dtype=bool)
    bnd[mesh.bnd_node] = True
    scale = np.abs(mesh.cij).max()
    for (i, j), k in pos.items():
        if bnd[i] and bnd[j]:
            continue
        kt = pos[(j, i)]
        assert np.abs(mesh.cij[:, k] + mesh.cij[:, kt]).max() <= 1e-13 * scale


def test_mass_matrix_exactly_symmetric(mesh):
    rows = mesh.row_of_entry()
    pos = {(i, j): k for k, (i, j) in enumerate(zip(rows.tolist(), mesh.col.tolist()))}
    for (i, j), k in pos.items():
        assert mesh.mij[k] == mesh.mij[pos[(j, i)]]


def test_domain_measures():
    assert math.isclose(M.periodic_p1_square(16).mi.sum(), 100.0, rel_tol=1e-13)
    m = M.cylinder_channel_q1(12)
    # polygonal hole: area of the regular 48-gon? The vertices are on rays through the
    # square's boundary points, so compute the polygon area directly from the mesh.
    ring = m.coords[:48]
    x, y = ring[:, 0], ring[:, 1]
    hole = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    assert math.isclose(m.mi.sum(), 4.0 - hole, rel_tol=1e-12)
    assert 4.0 - hole > 4.0 - math.pi * 0.25 ** 2


def test_q1_quadrature_is_exact():
    """2x2 Gauss is exact for bilinear cells: 3x3 Gauss gives the same c_ij and m_ij."""
    rng = np.random.default_rng(3)
    base = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    xyz = base[None] + 0.2 * rng.uniform(-1, 1, (5, 4, 2))
    c2, m2, l2 = M._local_q1_2d(xyz)
    gx, gw = M._gauss(3)
    XI, ETA = np.meshgrid(gx, gx, indexing="ij")
    Wt = np.outer(gw, gw).ravel()
    phi, dphi = M._q1_2d_shape(XI.ravel(), ETA.ravel())
    J = np.einsum("car,qas->cqrs", xyz, dphi)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    grad = np.einsum("cqsr,qbs->cqbr", Jinv, dphi)
    c3 = np.einsum("q,qa,cqbr,cq->cabr", Wt, phi, grad, det)
    m3 = np.einsum("q,qa,qb,cq->cab", Wt, phi, phi, det)
    assert np.allclose(c2, c3, rtol=0, atol=1e-14)
    assert np.allclose(m2, m3, rtol=0, atol=1e-14)


def test_cylinder_boundary_kinds():
    m = M.cylinder_channel_q1(10)
    x, y = m.coords[m.bnd_node].T
    k = m.bnd_kind
    assert np.all(k[np.isclose(x, 0.0)] == M.BC_DIRICHLET)
    inner = np.isclose(x, 4.0) & (y > 0) & (y < 1)
    assert np.all(k[inner] == M.BC_DO_NOTHING)
    assert np.all(k[np.isclose(x, 4.0) & (np.isclose(y, 0) | np.isclose(y, 1))] == M.BC_SLIP)
    r = np.hypot(x - 0.6, y - 0.5)
    assert np.all(k[np.isclose(r, 0.25)] == M.BC_SLIP)
    # slip normals at the walls are (0, -1) / (0, 1); on the cylinder they point into the hole
    wall = (k == M.BC_SLIP) & np.isclose(y, 0.0)
    assert np.allclose(m.bnd_normal[:, wall].T, [0.0, -1.0])
    cyl = (k == M.BC_SLIP) & np.isclose(r, 0.25)
    radial = np.stack([x[cyl] - 0.6, y[cyl] - 0.5]) / 0.25
    assert np.all(np.einsum("dk,dk->k", m.bnd_normal[:, cyl], radial) < -0.99)


def test_vortex_initial_data_is_a_steady_isentropic_vortex():
    """Radial balance dp/dr = rho u_theta^2 / r and p / rho^gamma constant."""
    g = 1.4
    r = np.linspace(0.2, 4.0, 41)
    h = 1e-5
    def prim(rr):
        return W.isentropic_vortex_primitive(rr, 0.0 * rr, 0.0, u_inf=(0.0, 0.0))
    rho, u, v, p = prim(r)
    _, _, _, pp = prim(r + h)
    _, _, _, pm = prim(r - h)
    dpdr = (pp - pm) / (2 * h)
    # central differences: truncation ~1e-10, cancellation ~1e-11 absolute
    assert np.allclose(dpdr, rho * v ** 2 / r, rtol=1e-7, atol=1e-10)
    assert np.allclose(p / rho ** g, 1.0, rtol=1e-14)
    assert np.allclose(u, 0.0, atol=1e-15)


def test_extruded_mesh_equals_direct_3d_assembly():
    """The tensor-product extrusion equals 3x3x3-Gauss assembly of the same
    hexahedra (structured box, periodic in z): identical CSR, c_ij, m_ij, m_i."""
    base = M.structured_q1(4, 3, 0.0, 1.0, 0.0, 0.75)
    ext = M.extruded_q1(base, 5, z_len=1.25)
    ref = M.structured_q1_3d(4, 3, 5, box=((0.0, 1.0), (0.0, 0.75), (0.0, 1.25)),
                             periodic=(False, False, True))
    # both number nodes (x, y) major and z minor
    assert np.array_equal(ext.row_ptr, ref.row_ptr) and np.array_equal(ext.col, ref.col)
    assert np.allclose(ext.cij, ref.cij, rtol=0, atol=1e-15)
    assert np.allclose(ext.mij, ref.mij, rtol=0, atol=1e-16)
    assert np.allclose(ext.mi, ref.mi, rtol=1e-14)
    assert np.array_equal(np.sort(ext.bnd_node), np.sort(ref.bnd_node))


def test_extruded_cylinder_identities():
    m = M.extruded_q1(M.cylinder_channel_q1(8), 4)
    rows = m.row_of_entry()
    assert np.abs(np.stack([np.bincount(rows, weights=m.cij[d], minlength=m.n) for d in range(3)])).max() < 1e-15
    cs = np.stack([np.bincount(m.col, weights=m.cij[d], minlength=m.n) for d in range(3)])
    full = np.zeros((3, m.n))
    full[:, m.bnd_node] = m.bnd_mass_full * m.bnd_normal_full
    assert np.abs(cs - full).max() < 1e-14
    assert np.unique(np.diff(m.row_ptr)).max() == 27
