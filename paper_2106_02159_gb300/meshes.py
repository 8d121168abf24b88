"""Seeded synthetic meshes and their finite-element coefficients.

These are the INPUTS of the hyperbolic step (Sec. 2.2 of the paper): the CSR
stencil I(i), the matrices c_ij = int phi_i grad phi_j and m_ij = int phi_i
phi_j, the lumped masses m_i = int phi_i, and the boundary data of Sec. 3.3
(eq. unit_normal_vector) and Sec. 4.1 (eq. def_ns_nio). Nothing here computes
any part of the hyperbolic step itself; both the CUDA library and the oracle
receive these arrays.

Element types:
  * P1 triangles: c_ij = sum_K |K|/3 grad phi_j|_K, m_ij = |K|(1 + delta_ij)/12,
    m_i = sum_K |K|/3 (exact formulas).
  * Q1 quadrilaterals with a bilinear map: 2x2 Gauss, exact for c_ij and m_ij
    (the integrands are polynomials of degree <= 3 per reference variable).
  * Q1 hexahedra with a trilinear map: 3x3x3 Gauss (exact).
Boundary integrals int_{face} phi_i n ds: exact per straight edge / planar
face (2-point Gauss per direction on faces).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_SLIP = 1
BC_DIRICHLET = 2
BC_DO_NOTHING = 3
BC_CHARACTERISTIC = 4  # non-reflecting, by characteristic variables (Sec. 4.2.2)
BC_GODUNOV = 5         # non-reflecting, by the exact Riemann value (Sec. 4.2.1)


@dataclasses.dataclass
class Mesh:
    """A mesh with every array the hyperbolic step reads.

    Layouts: ``cij`` is ``[dim, nnz]`` (component-major), state vectors are
    ``[dim + 2, n]``. ``bnd_normal`` is the unit slip normal n^s_i for slip
    nodes and the unit normal of the non-slip part for the others.
    ``bnd_mass_full``/``bnd_normal_full`` are m^bnd_i and n_i of eq.
    unit_normal_vector (all boundary parts), used by conservation checks.
    """

    name: str
    dim: int
    coords: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    cij: np.ndarray
    mij: np.ndarray
    mi: np.ndarray
    bnd_node: np.ndarray
    bnd_kind: np.ndarray
    bnd_normal: np.ndarray
    bnd_mass_full: np.ndarray
    bnd_normal_full: np.ndarray
    # the cells (node ids) and their vertex coordinates, kept for the
    # parabolic (viscous) operators; None for meshes built by other means
    cells: np.ndarray | None = None
    cell_xyz: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.mi.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_bnd(self) -> int:
        return int(self.bnd_node.shape[0])

    def row_of_entry(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))


# --------------------------------------------------------------------------
# reference elements and quadrature
# --------------------------------------------------------------------------

def _gauss(npts: int):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def _q1_2d_shape(xi, eta):
    """Bilinear shape functions on [0,1]^2, vertices (0,0),(1,0),(1,1),(0,1)."""
    phi = np.stack([(1 - xi) * (1 - eta), xi * (1 - eta), xi * eta, (1 - xi) * eta], axis=-1)
    dxi = np.stack([-(1 - eta), (1 - eta), eta, -eta], axis=-1)
    deta = np.stack([-(1 - xi), -xi, xi, (1 - xi)], axis=-1)
    return phi, np.stack([dxi, deta], axis=-1)  # [..., 4], [..., 4, 2]


def _q1_3d_shape(xi, eta, zeta):
    """Trilinear shape functions on [0,1]^3; vertex a = (bx, by, bz) with
    index bx + 2 by + 4 bz is NOT used; the order is the bottom quad
    (0,0,0),(1,0,0),(1,1,0),(0,1,0) then the top quad at zeta = 1."""
    corners = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                        [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=float)
    phis, grads = [], []
    for c in corners:
        fx = xi if c[0] else 1 - xi
        fy = eta if c[1] else 1 - eta
        fz = zeta if c[2] else 1 - zeta
        gx = (1.0 if c[0] else -1.0)
        gy = (1.0 if c[1] else -1.0)
        gz = (1.0 if c[2] else -1.0)
        phis.append(fx * fy * fz)
        grads.append(np.stack([gx * fy * fz, fx * gy * fz, fx * fy * gz], axis=-1))
    return np.stack(phis, axis=-1), np.stack(grads, axis=-2)


def _local_p1(xyz):
    """xyz: [nc, 3, 2] -> c_loc [nc,3,3,2], m_loc [nc,3,3], ml [nc,3]."""
    x0, x1, x2 = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    e1, e2 = x1 - x0, x2 - x0
    det = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    if np.any(det <= 0):
        raise ValueError("P1 cell with non-positive orientation")
    area = 0.5 * det
    # gradients of barycentric coordinates
    g1 = np.stack([e2[:, 1], -e2[:, 0]], axis=-1) / det[:, None]
    g2 = np.stack([-e1[:, 1], e1[:, 0]], axis=-1) / det[:, None]
    g0 = -(g1 + g2)
    grads = np.stack([g0, g1, g2], axis=1)  # [nc, 3, 2]
    c_loc = (area / 3.0)[:, None, None, None] * np.broadcast_to(grads[:, None, :, :], (xyz.shape[0], 3, 3, 2))
    eye = np.eye(3)
    m_loc = area[:, None, None] * (1.0 + eye)[None] / 12.0
    ml = np.repeat((area / 3.0)[:, None], 3, axis=1)
    return np.ascontiguousarray(c_loc), m_loc, ml


def _local_q1_2d(xyz):
    """xyz: [nc, 4, 2]; 2x2 Gauss (exact for bilinear maps)."""
    gx, gw = _gauss(2)
    XI, ETA = np.meshgrid(gx, gx, indexing="ij")
    W = np.outer(gw, gw).ravel()
    phi, dphi = _q1_2d_shape(XI.ravel(), ETA.ravel())  # [q,4], [q,4,2]
    # Jacobian J[c,q] = sum_a x_a (x) dphi_a  -> [nc, q, 2, 2], J[.., r, s] = d x_r / d xi_s
    J = np.einsum("car,qas->cqrs", xyz, dphi)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    if np.any(det <= 0):
        raise ValueError("Q1 cell with non-positive Jacobian")
    # J^{-T} grad_ref, times det: adj(J)^T grad_ref
    adjT = np.empty_like(J)
    adjT[..., 0, 0] = J[..., 1, 1]
    adjT[..., 0, 1] = -J[..., 1, 0]
    adjT[..., 1, 0] = -J[..., 0, 1]
    adjT[..., 1, 1] = J[..., 0, 0]
    # grad phi_b * det = adj(J)^T dphi_b  -> [nc, q, 4, 2]
    gdet = np.einsum("cqrs,qbs->cqbr", adjT, dphi)
    c_loc = np.einsum("q,qa,cqbr->cabr", W, phi, gdet)
    m_loc = np.einsum("q,qa,qb,cq->cab", W, phi, phi, det)
    ml = np.einsum("q,qa,cq->ca", W, phi, det)
    return c_loc, m_loc, ml


def _local_q1_3d(xyz):
    """xyz: [nc, 8, 3]; 3x3x3 Gauss (exact for trilinear maps)."""
    gx, gw = _gauss(3)
    XI, ETA, ZETA = np.meshgrid(gx, gx, gx, indexing="ij")
    W = np.einsum("i,j,k->ijk", gw, gw, gw).ravel()
    phi, dphi = _q1_3d_shape(XI.ravel(), ETA.ravel(), ZETA.ravel())  # [q,8], [q,8,3]
    J = np.einsum("car,qas->cqrs", xyz, dphi)
    det = np.linalg.det(J)
    if np.any(det <= 0):
        raise ValueError("Q1 hex with non-positive Jacobian")
    # cofactor matrix: adj(J)^T = det * J^{-T}
    cof = np.empty_like(J)
    for r in range(3):
        for s in range(3):
            r1, r2 = [x for x in range(3) if x != r]
            s1, s2 = [x for x in range(3) if x != s]
            minor = J[..., r1, s1] * J[..., r2, s2] - J[..., r1, s2] * J[..., r2, s1]
            cof[..., r, s] = ((-1) ** (r + s)) * minor
    gdet = np.einsum("cqrs,qbs->cqbr", cof, dphi)
    c_loc = np.einsum("q,qa,cqbr->cabr", W, phi, gdet)
    m_loc = np.einsum("q,qa,qb,cq->cab", W, phi, phi, det)
    ml = np.einsum("q,qa,cq->ca", W, phi, det)
    return c_loc, m_loc, ml


# --------------------------------------------------------------------------
# global assembly
# --------------------------------------------------------------------------

def _assemble(n, dim, cells, local_fn, xyz, chunk=1 << 20):
    """Scatter local matrices into a CSR pattern with sorted columns."""
    nv = cells.shape[1]
    cc = cells.astype(np.int64)
    keys = (cc[:, :, None] * n + cc[:, None, :]).ravel()  # entry (a, b) of every cell, row-major
    ukeys, inverse = np.unique(keys, return_inverse=True)
    del keys
    rows = (ukeys // n).astype(np.int64)
    col = (ukeys % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    nnz = ukeys.size
    cij = np.zeros((dim, nnz))
    mij = np.zeros(nnz)
    mi = np.zeros(n)
    nc = cells.shape[0]
    for c0 in range(0, nc, chunk):
        c1 = min(nc, c0 + chunk)
        c_loc, m_loc, ml = local_fn(xyz[c0:c1])
        cc = cells[c0:c1].astype(np.int64)
        pos = inverse[c0 * nv * nv:c1 * nv * nv]
        for d in range(dim):
            cij[d] += np.bincount(pos, weights=c_loc[..., d].ravel(), minlength=nnz)
        mij += np.bincount(pos, weights=m_loc.ravel(), minlength=nnz)
        mi += np.bincount(cc.ravel(), weights=ml.ravel(), minlength=n)
    return row_ptr, col, cij, mij, mi


def _boundary(n, dim, faces, face_xyz, face_kind, cell_centroid):
    """Exact int_face phi_i n ds per boundary face; returns per-node data.

    faces: [nf, nvf] node ids, face_xyz: [nf, nvf, dim], face_kind: [nf],
    cell_centroid: [nf, dim] centroid of the cell owning the face (to orient
    the outward normal)."""
    nf = faces.shape[0]
    if nf == 0:
        e = np.zeros(0, dtype=np.int32)
        return e, e, np.zeros((dim, 0)), np.zeros(0), np.zeros((dim, 0))
    if dim == 2:
        t = face_xyz[:, 1] - face_xyz[:, 0]
        nrm = np.stack([t[:, 1], -t[:, 0]], axis=-1)  # length = |edge|
        mid = 0.5 * (face_xyz[:, 0] + face_xyz[:, 1])
        sgn = np.sign(np.einsum("fd,fd->f", mid - cell_centroid, nrm))
        nrm = nrm * sgn[:, None]
        contrib = np.repeat(0.5 * nrm[:, None, :], 2, axis=1)  # [nf, 2, dim]
    else:
        gx, gw = _gauss(2)
        XI, ETA = np.meshgrid(gx, gx, indexing="ij")
        W = np.outer(gw, gw).ravel()
        phi, dphi = _q1_2d_shape(XI.ravel(), ETA.ravel())
        dx = np.einsum("car,qas->cqrs", face_xyz, dphi)  # [nf, q, 3, 2]
        cr = np.cross(dx[..., 0], dx[..., 1])  # [nf, q, 3]
        mid = face_xyz.mean(axis=1)
        sgn = np.sign(np.einsum("fd,fd->f", mid - cell_centroid, cr.sum(axis=1)))
        cr = cr * sgn[:, None, None]
        contrib = np.einsum("q,qa,cqd->cad", W, phi, cr)
    nodes = faces.ravel()
    kinds = np.repeat(face_kind, faces.shape[1])
    vec = contrib.reshape(-1, dim)
    full = np.zeros((n, dim))
    slip = np.zeros((n, dim))
    nonslip = np.zeros((n, dim))
    touch = np.zeros((n, 6), dtype=bool)
    for d in range(dim):
        full[:, d] = np.bincount(nodes, weights=vec[:, d], minlength=n)
        slip[:, d] = np.bincount(nodes[kinds == BC_SLIP], weights=vec[kinds == BC_SLIP, d], minlength=n)
        nonslip[:, d] = np.bincount(nodes[kinds != BC_SLIP], weights=vec[kinds != BC_SLIP, d], minlength=n)
    for kd in (BC_SLIP, BC_DIRICHLET, BC_DO_NOTHING, BC_CHARACTERISTIC, BC_GODUNOV):
        touch[np.unique(nodes[kinds == kd]), kd] = True
    bnodes = np.unique(nodes)
    # kind priority: inflow (Dirichlet) > slip > non-reflecting > do-nothing
    kind = np.full(bnodes.size, BC_DO_NOTHING, dtype=np.int32)
    kind[touch[bnodes, BC_CHARACTERISTIC]] = BC_CHARACTERISTIC
    kind[touch[bnodes, BC_GODUNOV]] = BC_GODUNOV
    kind[touch[bnodes, BC_SLIP]] = BC_SLIP
    kind[touch[bnodes, BC_DIRICHLET]] = BC_DIRICHLET
    vs = slip[bnodes]
    vn = nonslip[bnodes]
    use = np.where((kind == BC_SLIP)[:, None], vs, vn)
    norm = np.linalg.norm(use, axis=1)
    normal = np.where(norm[:, None] > 0, use / np.where(norm > 0, norm, 1.0)[:, None], 0.0)
    vf = full[bnodes]
    mfull = np.linalg.norm(vf, axis=1)
    nfull = np.where(mfull[:, None] > 0, vf / np.where(mfull > 0, mfull, 1.0)[:, None], 0.0)
    return (bnodes.astype(np.int32), kind, np.ascontiguousarray(normal.T), mfull,
            np.ascontiguousarray(nfull.T))


def _finish(name, dim, coords, cells, xyz, local_fn, faces, face_xyz, face_kind, face_cell):
    n = coords.shape[0]
    row_ptr, col, cij, mij, mi = _assemble(n, dim, cells, local_fn, xyz)
    cent = xyz.mean(axis=1)
    if faces is None or len(faces) == 0:
        b = _boundary(n, dim, np.zeros((0, 2), dtype=np.int64), None, None, None)
    else:
        b = _boundary(n, dim, faces, face_xyz, face_kind, cent[face_cell])
    return Mesh(name=name, dim=dim, coords=coords, row_ptr=row_ptr, col=col, cij=cij, mij=mij, mi=mi,
                bnd_node=b[0], bnd_kind=b[1], bnd_normal=b[2], bnd_mass_full=b[3], bnd_normal_full=b[4],
                cells=np.ascontiguousarray(cells, dtype=np.int32), cell_xyz=np.ascontiguousarray(xyz))


def parabolic_data(mesh: Mesh) -> dict:
    """The finite-element data of the parabolic (viscous) sub-step of Sec. 5
    for a 2D P1 or Q1 mesh, with one quadrature rule for everything (P1: the
    centroid, exact; Q1: 2 x 2 Gauss):
      L[nnz]          L_ij = int grad phi_i . grad phi_j (Fourier term b)
      G[2][2][nnz]    G_ij[k][m] = int d_k phi_i d_m phi_j (viscous term a)
      qw[nc][nq]      quadrature weights times |det J|
      qphi[nc][nq][nv], qgrad[nc][nq][2][nv]  shape values and physical gradients
      cells[nc][nv]   node ids
    (the viscous energy source K_i of eq. def_Ki_nplusone is evaluated with
    the same quadrature)."""
    if mesh.dim != 2 or mesh.cells is None:
        raise ValueError("parabolic data: 2D P1/Q1 meshes built by this module")
    cells, xyz = mesh.cells, mesh.cell_xyz
    nc, nv = cells.shape
    if nv == 3:
        x0, x1, x2 = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        e1, e2 = x1 - x0, x2 - x0
        det = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
        g1 = np.stack([e2[:, 1], -e2[:, 0]], axis=-1) / det[:, None]
        g2 = np.stack([-e1[:, 1], e1[:, 0]], axis=-1) / det[:, None]
        grads = np.stack([-(g1 + g2), g1, g2], axis=1)  # [nc, 3, 2]
        qw = (0.5 * det)[:, None]
        qphi = np.full((nc, 1, 3), 1.0 / 3.0)
        qgrad = np.ascontiguousarray(grads.transpose(0, 2, 1)[:, None])  # [nc, 1, 2, 3]
    elif nv == 4:
        gx, gw = _gauss(2)
        XI, ETA = np.meshgrid(gx, gx, indexing="ij")
        W = np.outer(gw, gw).ravel()
        phi, dphi = _q1_2d_shape(XI.ravel(), ETA.ravel())
        J = np.einsum("car,qas->cqrs", xyz, dphi)
        det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
        adjT = np.empty_like(J)
        adjT[..., 0, 0] = J[..., 1, 1]
        adjT[..., 0, 1] = -J[..., 1, 0]
        adjT[..., 1, 0] = -J[..., 0, 1]
        adjT[..., 1, 1] = J[..., 0, 0]
        g = np.einsum("cqrs,qbs->cqrb", adjT, dphi) / det[..., None, None]  # [nc, q, 2, 4]
        qw = W[None, :] * det
        qphi = np.broadcast_to(phi[None], (nc, 4, 4)).copy()
        qgrad = np.ascontiguousarray(g)
    else:
        raise ValueError("parabolic data: P1 or Q1 cells only")
    Lloc = np.einsum("cq,cqka,cqkb->cab", qw, qgrad, qgrad)
    Gloc = np.einsum("cq,cqka,cqmb->ckmab", qw, qgrad, qgrad)
    key = mesh.row_of_entry().astype(np.int64) * mesh.n + mesh.col
    rows = np.repeat(cells, nv, axis=1).ravel().astype(np.int64)
    cols = np.tile(cells, (1, nv)).ravel().astype(np.int64)
    pos = np.searchsorted(key, rows * mesh.n + cols)
    if np.any(key[pos] != rows * mesh.n + cols):
        raise ValueError("parabolic data: cell pair missing from the CSR pattern")
    L = np.bincount(pos, weights=Lloc.reshape(nc, -1).ravel(), minlength=mesh.nnz)
    G = np.empty((2, 2, mesh.nnz))
    for k in range(2):
        for m in range(2):
            G[k, m] = np.bincount(pos, weights=Gloc[:, k, m].reshape(nc, -1).ravel(), minlength=mesh.nnz)
    return dict(L=L, G=G, qw=np.ascontiguousarray(qw), qphi=np.ascontiguousarray(qphi), qgrad=qgrad,
                cells=np.ascontiguousarray(cells, dtype=np.int32))


# --------------------------------------------------------------------------
# structured meshes
# --------------------------------------------------------------------------

def periodic_p1_square(nv: int = 64, lo: float = -5.0, hi: float = 5.0, shear: float = 0.0) -> Mesh:
    """nv x nv-vertex periodic P1 mesh of [lo,hi]^2; every square is split by
    its lower-left -> upper-right diagonal (7-point stencil). shear != 0 maps
    (x, y) to (x + shear y, y): the periodic parallelogram with lattice vectors
    (hi - lo)(1, 0) and (hi - lo)(shear, 1)."""
    h = (hi - lo) / nv
    a, b = np.meshgrid(np.arange(nv), np.arange(nv), indexing="ij")
    a, b = a.ravel(), b.ravel()
    vid = lambda x, y: (x % nv) * nv + (y % nv)  # noqa: E731
    coords = np.zeros((nv * nv, 2))
    coords[vid(a, b), 0] = lo + a * h
    coords[vid(a, b), 1] = lo + b * h
    x0, y0 = lo + a * h, lo + b * h
    t1 = np.stack([vid(a, b), vid(a + 1, b), vid(a + 1, b + 1)], axis=1)
    t2 = np.stack([vid(a, b), vid(a + 1, b + 1), vid(a, b + 1)], axis=1)
    p00 = np.stack([x0, y0], -1)
    p10 = np.stack([x0 + h, y0], -1)
    p11 = np.stack([x0 + h, y0 + h], -1)
    p01 = np.stack([x0, y0 + h], -1)
    cells = np.concatenate([t1, t2])
    xyz = np.concatenate([np.stack([p00, p10, p11], 1), np.stack([p00, p11, p01], 1)])
    if shear:
        coords[:, 0] += shear * coords[:, 1]
        xyz = xyz.copy()
        xyz[..., 0] += shear * xyz[..., 1]
    name = f"p1-periodic-{nv}x{nv}" + (f"-shear{shear:g}" if shear else "")
    return _finish(name, 2, coords, cells, xyz, _local_p1, None, None, None, None)


def structured_q1(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0, periodic_x=False, periodic_y=False,
                  kinds=(BC_DO_NOTHING, BC_DO_NOTHING, BC_SLIP, BC_SLIP), name=None) -> Mesh:
    """Cartesian Q1 mesh of [x0,x1]x[y0,y1] with nx x ny cells. ``kinds`` gives
    the boundary kind of the faces at x0, x1, y0, y1 (ignored if periodic)."""
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    nvx = nx if periodic_x else nx + 1
    nvy = ny if periodic_y else ny + 1
    vid = lambda i, j: (i % nvx) * nvy + (j % nvy)  # noqa: E731
    I, J = np.meshgrid(np.arange(nvx), np.arange(nvy), indexing="ij")
    coords = np.zeros((nvx * nvy, 2))
    coords[vid(I.ravel(), J.ravel())] = np.stack([x0 + I.ravel() * hx, y0 + J.ravel() * hy], -1)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    cells = np.stack([vid(ci, cj), vid(ci + 1, cj), vid(ci + 1, cj + 1), vid(ci, cj + 1)], axis=1)
    bx, by = x0 + ci * hx, y0 + cj * hy
    xyz = np.stack([np.stack([bx, by], -1), np.stack([bx + hx, by], -1),
                    np.stack([bx + hx, by + hy], -1), np.stack([bx, by + hy], -1)], axis=1)
    faces, fxyz, fk, fc = [], [], [], []
    cid = lambda i, j: i * ny + j  # noqa: E731
    if not periodic_x:
        for side, i in ((0, 0), (1, nx)):
            j = np.arange(ny)
            faces.append(np.stack([vid(np.full(ny, i), j), vid(np.full(ny, i), j + 1)], 1))
            fxyz.append(np.stack([np.stack([np.full(ny, x0 + i * hx), y0 + j * hy], -1),
                                  np.stack([np.full(ny, x0 + i * hx), y0 + (j + 1) * hy], -1)], 1))
            fk.append(np.full(ny, kinds[side]))
            fc.append(cid(np.full(ny, min(i, nx - 1)), j))
    if not periodic_y:
        for side, j in ((2, 0), (3, ny)):
            i = np.arange(nx)
            faces.append(np.stack([vid(i, np.full(nx, j)), vid(i + 1, np.full(nx, j))], 1))
            fxyz.append(np.stack([np.stack([x0 + i * hx, np.full(nx, y0 + j * hy)], -1),
                                  np.stack([x0 + (i + 1) * hx, np.full(nx, y0 + j * hy)], -1)], 1))
            fk.append(np.full(nx, kinds[side]))
            fc.append(cid(i, np.full(nx, min(j, ny - 1))))
    if faces:
        faces, fxyz, fk, fc = (np.concatenate(faces), np.concatenate(fxyz), np.concatenate(fk),
                               np.concatenate(fc))
    else:
        faces = None
    return _finish(name or f"q1-{nx}x{ny}", 2, coords, cells, xyz, _local_q1_2d, faces, fxyz, fk, fc)


def _radial_grading(m: int, length: float):
    """Geometric layer distribution t_0 = 0 < ... < t_nr = 1 along a ray of the
    given length, first layer ~ h/4 and last ~ h, h = 1/m."""
    h = 1.0 / m
    best = None
    for nr in range(1, 4 * m + 8):
        q = 4.0 ** (1.0 / (nr - 1)) if nr > 1 else 1.0
        first = length * (q - 1.0) / (q ** nr - 1.0) if nr > 1 else length
        err = abs(first - h / 4.0)
        if best is None or err < best[0]:
            best = (err, nr, q)
    _, nr, q = best
    if nr == 1:
        return np.array([0.0, 1.0])
    t = (q ** np.arange(nr + 1) - 1.0) / (q ** nr - 1.0)
    return t


def cylinder_channel_q1(m: int, name: str | None = None, element: str = "q1") -> Mesh:
    """Conforming block-structured Q1 mesh of the channel [0,4]x[0,1] minus the
    disc of radius 0.25 centred at (0.6, 0.5).

    Blocks: an O-grid between the circle and the square [0.1,1.1]x[0,1] (4m
    rays, geometrically graded layers, first layer ~h/4), and Cartesian blocks
    [0,0.1]x[0,1] and [1.1,4]x[0,1] with spacing h = 1/m. The cylinder is the
    polygon of its mesh vertices, so the mesh covers its own domain exactly.
    Boundary kinds: Dirichlet (supersonic inflow) at x = 0, do-nothing at
    x = 4, slip on y = 0, y = 1 and the cylinder.
    """
    cx, cy, r = 0.6, 0.5, 0.25
    nk = 4 * m
    s = np.arange(nk) / m
    side = np.minimum((s // 1).astype(int), 3)
    u = s - side
    sq = np.zeros((nk, 2))
    sq[side == 0] = np.stack([0.1 + u[side == 0], np.zeros((side == 0).sum())], -1)
    sq[side == 1] = np.stack([np.full((side == 1).sum(), 1.1), u[side == 1]], -1)
    sq[side == 2] = np.stack([1.1 - u[side == 2], np.ones((side == 2).sum())], -1)
    sq[side == 3] = np.stack([np.full((side == 3).sum(), 0.1), 1.0 - u[side == 3]], -1)
    ang = np.arctan2(sq[:, 1] - cy, sq[:, 0] - cx)
    circ = np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], -1)
    t = _radial_grading(m, 0.25)
    nr = t.size - 1
    ring = circ[None, :, :] + t[:, None, None] * (sq - circ)[None, :, :]  # [nr+1, nk, 2]
    ring_id = np.arange((nr + 1) * nk).reshape(nr + 1, nk)
    coords = [ring.reshape(-1, 2)]
    nxt = (nr + 1) * nk
    # left block [0, 0.1] x [0, 1]
    nlx = max(1, int(round(0.1 * m)))
    left_id = np.full((nlx + 1, m + 1), -1, dtype=np.int64)
    iy = np.arange(m + 1)
    left_id[nlx, :] = ring_id[nr, (nk - iy) % nk]
    cnt = nlx * (m + 1)
    left_id[:nlx, :] = nxt + np.arange(cnt).reshape(nlx, m + 1)
    gx, gy = np.meshgrid(np.arange(nlx) * (0.1 / nlx), iy / m, indexing="ij")
    coords.append(np.stack([gx.ravel(), gy.ravel()], -1))
    nxt += cnt
    # right block [1.1, 4] x [0, 1]
    nrx = max(1, int(round(2.9 * m)))
    right_id = np.full((nrx + 1, m + 1), -1, dtype=np.int64)
    right_id[0, :] = ring_id[nr, (m + iy) % nk]
    cnt = nrx * (m + 1)
    right_id[1:, :] = nxt + np.arange(cnt).reshape(nrx, m + 1)
    gx, gy = np.meshgrid(1.1 + np.arange(1, nrx + 1) * (2.9 / nrx), iy / m, indexing="ij")
    coords.append(np.stack([gx.ravel(), gy.ravel()], -1))
    coords = np.concatenate(coords)
    # cells
    l, k = np.meshgrid(np.arange(nr), np.arange(nk), indexing="ij")
    l, k = l.ravel(), k.ravel()
    k1 = (k + 1) % nk
    ring_cells = np.stack([ring_id[l, k], ring_id[l + 1, k], ring_id[l + 1, k1], ring_id[l, k1]], 1)

    def cart_cells(ids, nx_):
        i, j = np.meshgrid(np.arange(nx_), np.arange(m), indexing="ij")
        i, j = i.ravel(), j.ravel()
        return np.stack([ids[i, j], ids[i + 1, j], ids[i + 1, j + 1], ids[i, j + 1]], 1)

    lc = cart_cells(left_id, nlx)
    rc = cart_cells(right_id, nrx)
    cells = np.concatenate([ring_cells, lc, rc])
    xyz = coords[cells]
    # boundary faces
    faces, fk, fc = [], [], []
    nring = ring_cells.shape[0]
    # cylinder: ring layer 0 edges, cell index = l*nk + k with l = 0
    kk = np.arange(nk)
    faces.append(np.stack([ring_id[0, kk], ring_id[0, (kk + 1) % nk]], 1))
    fk.append(np.full(nk, BC_SLIP))
    fc.append(kk)
    # square bottom (k in [0, m)) and top (k in [2m, 3m)) on the walls, layer nr-1 cells
    for k0 in (0, 2 * m):
        kk = np.arange(k0, k0 + m)
        faces.append(np.stack([ring_id[nr, kk], ring_id[nr, (kk + 1) % nk]], 1))
        fk.append(np.full(m, BC_SLIP))
        fc.append((nr - 1) * nk + kk)
    off = nring
    for ids, nx_, cells_off, xkind in ((left_id, nlx, off, "left"), (right_id, nrx, off + lc.shape[0], "right")):
        i = np.arange(nx_)
        faces.append(np.stack([ids[i, 0], ids[i + 1, 0]], 1))
        fk.append(np.full(nx_, BC_SLIP))
        fc.append(cells_off + i * m + 0)
        faces.append(np.stack([ids[i, m], ids[i + 1, m]], 1))
        fk.append(np.full(nx_, BC_SLIP))
        fc.append(cells_off + i * m + (m - 1))
        j = np.arange(m)
        if xkind == "left":
            faces.append(np.stack([ids[0, j], ids[0, j + 1]], 1))
            fk.append(np.full(m, BC_DIRICHLET))
            fc.append(cells_off + 0 * m + j)
        else:
            faces.append(np.stack([ids[nx_, j], ids[nx_, j + 1]], 1))
            fk.append(np.full(m, BC_DO_NOTHING))
            fc.append(cells_off + (nx_ - 1) * m + j)
    faces = np.concatenate(faces)
    fk = np.concatenate(fk)
    fc = np.concatenate(fc)
    if element == "p1":
        # every (convex) quad [a, b, c, d] split into [a, b, c] and [a, c, d];
        # a boundary edge keeps the interior side of its quad
        tri = np.empty((2 * cells.shape[0], 3), dtype=cells.dtype)
        tri[0::2] = cells[:, [0, 1, 2]]
        tri[1::2] = cells[:, [0, 2, 3]]
        return _finish(name or f"p1-cylinder-m{m}", 2, coords, tri, coords[tri], _local_p1, faces, coords[faces],
                       fk, 2 * fc)
    return _finish(name or f"q1-cylinder-m{m}", 2, coords, cells, xyz, _local_q1_2d, faces, coords[faces], fk, fc)


def cylinder_channel_p1(m: int, name: str | None = None) -> Mesh:
    """The cylinder channel mesh with every quadrilateral split into two P1
    triangles (same vertices, boundary and kinds)."""
    return cylinder_channel_q1(m, name, element="p1")


def cylinder_channel_vertices(m: int) -> int:
    """Vertex count of ``cylinder_channel_q1(m)`` without building it."""
    nr = _radial_grading(m, 0.25).size - 1
    nlx = max(1, int(round(0.1 * m)))
    nrx = max(1, int(round(2.9 * m)))
    return (nr + 1) * 4 * m + (nlx + nrx) * (m + 1)


def cylinder_m_for_vertices(target: int) -> int:
    lo, hi = 2, 4096
    while lo < hi:
        mid = (lo + hi) // 2
        if cylinder_channel_vertices(mid) < target:
            lo = mid + 1
        else:
            hi = mid
    return lo


def structured_q1_3d(nx: int, ny: int, nz: int, box=((0.0, 1.0), (0.0, 1.0), (0.0, 1.0)),
                     periodic=(False, False, False), kinds=(BC_SLIP,) * 6, name=None) -> Mesh:
    """Cartesian Q1 hex mesh (27-point stencil) of a box; ``kinds`` gives the
    boundary kind of the faces x-, x+, y-, y+, z-, z+ (ignored if periodic)."""
    ncell = (nx, ny, nz)
    h = [(box[d][1] - box[d][0]) / ncell[d] for d in range(3)]
    nv = [ncell[d] if periodic[d] else ncell[d] + 1 for d in range(3)]

    def vid(i, j, k):
        return ((i % nv[0]) * nv[1] + (j % nv[1])) * nv[2] + (k % nv[2])

    I, J, K = np.meshgrid(*[np.arange(v) for v in nv], indexing="ij")
    coords = np.zeros((nv[0] * nv[1] * nv[2], 3))
    coords[vid(I.ravel(), J.ravel(), K.ravel())] = np.stack(
        [box[0][0] + I.ravel() * h[0], box[1][0] + J.ravel() * h[1], box[2][0] + K.ravel() * h[2]], -1)
    ci, cj, ck = [a.ravel() for a in np.meshgrid(*[np.arange(c) for c in ncell], indexing="ij")]
    corner = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
    cells = np.stack([vid(ci + a, cj + b, ck + c) for a, b, c in corner], axis=1)
    base = np.stack([box[0][0] + ci * h[0], box[1][0] + cj * h[1], box[2][0] + ck * h[2]], -1)
    xyz = base[:, None, :] + corner[None, :, :] * np.array(h)[None, None, :]
    faces, fk, fc = [], [], []
    cid = (ci * ncell[1] + cj) * ncell[2] + ck
    quad = {0: [(0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)], 1: [(0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0)],
            2: [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)]}
    idx = (ci, cj, ck)
    for d in range(3):
        if periodic[d]:
            continue
        for side in (0, 1):
            sel = idx[d] == (0 if side == 0 else ncell[d] - 1)
            off = np.zeros(3, dtype=int)
            off[d] = side
            fverts = []
            for q in quad[d]:
                o = np.array(q) + off
                fverts.append(vid(ci[sel] + o[0], cj[sel] + o[1], ck[sel] + o[2]))
            faces.append(np.stack(fverts, 1))
            fk.append(np.full(sel.sum(), kinds[2 * d + side]))
            fc.append(cid[sel])
    if faces:
        faces, fk, fc = np.concatenate(faces), np.concatenate(fk), np.concatenate(fc)
        fxyz = np.empty((faces.shape[0], 4, 3))
        # face geometry from the unwrapped cell corners
        for q in range(4):
            fxyz[:, q] = coords[faces[:, q]]
        return _finish(name or f"q1-3d-{nx}x{ny}x{nz}", 3, coords, cells, xyz, _local_q1_3d, faces, fxyz, fk, fc)
    return _finish(name or f"q1-3d-{nx}x{ny}x{nz}", 3, coords, cells, xyz, _local_q1_3d, None, None, None, None)


def concatenate(meshes, bnd_states=None):
    """Block-diagonal union of independent meshes of one dimension (a batch).

    Returns (mesh, row_offset[k+1], bnd_state or None): instance k owns rows
    [row_offset[k], row_offset[k+1]); bnd_states (one per mesh, or None) are
    concatenated along the boundary nodes."""
    dim = meshes[0].dim
    assert all(m.dim == dim for m in meshes)
    noff = np.cumsum([0] + [m.n for m in meshes])
    eoff = np.cumsum([0] + [m.nnz for m in meshes])
    row_ptr = np.concatenate([m.row_ptr[:-1] + eoff[k] for k, m in enumerate(meshes)] + [[eoff[-1]]])
    col = np.concatenate([m.col.astype(np.int64) + noff[k] for k, m in enumerate(meshes)]).astype(np.int32)
    cat = lambda f, axis=-1: np.ascontiguousarray(np.concatenate([f(m) for m in meshes], axis=axis))  # noqa: E731
    mesh = Mesh(name=f"batch-{len(meshes)}", dim=dim, coords=cat(lambda m: m.coords, 0), row_ptr=row_ptr.astype(np.int64),
                col=col, cij=cat(lambda m: m.cij), mij=cat(lambda m: m.mij), mi=cat(lambda m: m.mi),
                bnd_node=np.concatenate([m.bnd_node.astype(np.int64) + noff[k]
                                         for k, m in enumerate(meshes)]).astype(np.int32),
                bnd_kind=cat(lambda m: m.bnd_kind), bnd_normal=cat(lambda m: m.bnd_normal),
                bnd_mass_full=cat(lambda m: m.bnd_mass_full), bnd_normal_full=cat(lambda m: m.bnd_normal_full))
    bs = None
    if bnd_states is not None:
        S = dim + 2
        bs = np.ascontiguousarray(np.concatenate(
            [b if b is not None else np.zeros((S, m.n_bnd)) for m, b in zip(meshes, bnd_states)], axis=1))
    return mesh, noff.astype(np.int64), bs


def extruded_q1(base: Mesh, nz: int, z_len: float = 2.0, name: str | None = None) -> Mesh:
    """Q1 hexahedra: the 2D Q1 mesh ``base`` extruded over z in [0, z_len)
    with nz periodic layers (27-point rows for 9-point 2D rows).

    With phi_(a,k)(x, y, z) = phi_a(x, y) psi_k(z) (psi: periodic 1D hat
    functions, spacing hz) every coefficient is an exact tensor product:
      c_(a,k),(b,l) = (c2_ab,x m1_kl, c2_ab,y m1_kl, m2_ab c1_kl),
      m_(a,k),(b,l) = m2_ab m1_kl,  m_(a,k) = m2_a hz,
    with m1 = hz (1/6, 2/3, 1/6) and c1 = (-1/2, 0, 1/2) on (k-1, k, k+1).
    Node index a nz + k; boundary faces are the 2D boundary edges times the
    layers, so n_i = (n2_a, 0) and m^bnd_i = m2^bnd_a hz."""
    if base.dim != 2:
        raise ValueError("extrude a 2D mesh")
    if nz < 3:
        raise ValueError("need at least 3 periodic layers")
    hz = z_len / nz
    n2, nnz2 = base.n, base.nnz
    k = np.arange(nz, dtype=np.int64)
    lz = np.stack([(k - 1) % nz, k, (k + 1) % nz], axis=1)   # neighbour layers
    m1 = np.array([hz / 6.0, 2.0 * hz / 3.0, hz / 6.0])
    c1 = np.array([-0.5, 0.0, 0.5])
    order = np.argsort(lz, axis=1, kind="stable")              # sorted column order per layer
    lz_s = np.take_along_axis(lz, order, axis=1)               # [nz, 3]
    m1_s = m1[order]
    c1_s = c1[order]
    rows2 = base.row_of_entry()
    cnt2 = np.diff(base.row_ptr)                               # 2D row lengths
    n = n2 * nz
    nnz = nnz2 * 3 * nz
    row_len = np.repeat(cnt2 * 3, nz)                          # row (a, k) has 3 cnt2[a] entries
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(row_len)
    # entries of row (a, k): for every 2D entry e of row a, the 3 layers l of k
    # (columns b nz + l increase with b, then with l: sorted)
    col = np.empty(nnz, dtype=np.int32)
    cij = np.empty((3, nnz))
    mij = np.empty(nnz)
    # vectorised over (a, k): block of row a has cnt2[a] * 3 entries per layer
    e_start = base.row_ptr[:-1]
    for a0 in range(0, n2, 4096):
        a1 = min(n2, a0 + 4096)
        for a in range(a0, a1):
            e0, e1 = int(base.row_ptr[a]), int(base.row_ptr[a + 1])
            b = base.col[e0:e1].astype(np.int64)               # [c]
            c = e1 - e0
            base_pos = row_ptr[a * nz]
            # [nz, c, 3]
            colv = b[None, :, None] * nz + lz_s[:, None, :]
            pos = base_pos + np.arange(nz * c * 3)
            col[pos] = colv.reshape(-1)
            cx = base.cij[0, e0:e1][None, :, None] * m1_s[:, None, :]
            cy = base.cij[1, e0:e1][None, :, None] * m1_s[:, None, :]
            cz = base.mij[e0:e1][None, :, None] * c1_s[:, None, :]
            cij[0, pos] = cx.reshape(-1)
            cij[1, pos] = cy.reshape(-1)
            cij[2, pos] = cz.reshape(-1)
            mij[pos] = (base.mij[e0:e1][None, :, None] * m1_s[:, None, :]).reshape(-1)
    del e_start, rows2
    mi = np.repeat(base.mi, nz) * hz
    coords = np.empty((n, 3))
    coords[:, :2] = np.repeat(base.coords, nz, axis=0)
    coords[:, 2] = np.tile(k * hz, n2)
    bn = (base.bnd_node.astype(np.int64)[:, None] * nz + k[None, :]).reshape(-1).astype(np.int32)
    rep = lambda x: np.repeat(x, nz)  # noqa: E731
    normal = np.zeros((3, bn.size))
    normal[:2] = np.repeat(base.bnd_normal, nz, axis=1)
    nfull = np.zeros((3, bn.size))
    nfull[:2] = np.repeat(base.bnd_normal_full, nz, axis=1)
    return Mesh(name=name or f"{base.name}-extruded{nz}", dim=3, coords=coords, row_ptr=row_ptr, col=col,
                cij=cij, mij=mij, mi=mi, bnd_node=bn, bnd_kind=rep(base.bnd_kind), bnd_normal=normal,
                bnd_mass_full=rep(base.bnd_mass_full) * hz, bnd_normal_full=nfull)
