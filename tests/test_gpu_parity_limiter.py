"""Parity of the convex limiter (Sec. 3.3) and of the batched and served
paths with the FP64 oracle, through the C ABI. Needs a GPU.

What these tests separate: "a limiter decision flipped" from "the arithmetic
is wrong".
 - The first pass's limiter directions P_ij (eq. LambdaArrangement) are
   compared entry by entry; the symmetrised limiter l_ij entry by entry: equal
   where both searches ended at the same exit (0 or 1), within L_CONT_TOL where
   both ended inside (0, 1); every other entry is a flip. A flip is accepted
   only where it is a roundoff decision: the oracle's own constraints (density
   bounds and the entropy function psi of the search, Sec. 3.3), evaluated on
   the oracle's data, are met with equality to within FLIP_TIGHT (relative) at
   one of the two disputed values of l. Flips are counted and reported.
 - Stage-resynchronised runs feed the oracle, at every stage of 100 SSPRK(3,3)
   steps, the GPU's own input of that stage: each stage's result is held to
   1e-12 (relative L1) at every node outside the reach of a limiter difference
   (the nodes of an entry whose l_ij differs by more than L_SAME_TOL and, for
   the first pass, their neighbours, whose second search starts from the
   changed state); every flip whose inputs agree must be a roundoff decision
   as above. The excluded share is reported.
 - Batched instances (one launch for many independent meshes) and served
   requests (the eh_batch_* stream) are compared with the oracle run on each
   instance alone.
 - A 3D box of 216,000 rows (27-entry rows), large enough that the grid-stride
   row loops of the limiter kernels wrap several times.
 - The integer mesh data on the device (CSR and transpose index) bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu

# two symmetrised limiters agree "continuously" when both are strictly inside
# (0, 1) (the search iterated or clipped at the density bound) and differ by
# less than this; a larger difference is a flip of the iteration's path
L_CONT_TOL = 1e-9
# a flip is a roundoff decision when a constraint of the search, relative to
# its own magnitude, is met to within this at one of the two disputed l
FLIP_TIGHT = 1e-11
# limiters closer than this count as the same (their effect on the state,
# l P_ij, is far below the per-stage tolerance)
L_SAME_TOL = 1e-13
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    oracle.set_threads(0)


def solver_for(mesh, bnd_state=None, **kw):
    s = B.Solver(dim=mesh.dim, **kw)
    s.upload_mesh(mesh, bnd_state)
    return s


def limiter_flips(l_gpu, l_orc):
    """Entries where the two limiters took different discrete decisions (one at
    0 or 1 and the other not, or both inside (0, 1) but more than L_CONT_TOL
    apart)."""
    ends_g = (l_gpu == 0.0) | (l_gpu == 1.0)
    ends_o = (l_orc == 0.0) | (l_orc == 1.0)
    disagree_end = (ends_g | ends_o) & (l_gpu != l_orc)
    both_inside = ~ends_g & ~ends_o
    return disagree_end | (both_inside & (np.abs(l_gpu - l_orc) > L_CONT_TOL))


def _constraint_margin(ub, P, bounds, l):
    """Relative margin of the line search's constraints (Sec. 3.3) at the
    states ub[:, r] + l P[:, k]: min over rho - rho_min, rho_max - rho and
    psi = eps - Phi_min rho^gamma, each over its own magnitude (negative:
    violated)."""
    u = ub + l * P
    rho = u[0]
    dim = u.shape[0] - 2
    eps = u[dim + 1] - 0.5 * (u[1:dim + 1] ** 2).sum(0) / rho
    rmin, rmax, phimin = bounds
    with np.errstate(invalid="ignore", divide="ignore"):
        prg = phimin * np.abs(rho) ** GAMMA
        g = np.minimum((rho - rmin) / np.abs(rmin), (rmax - rho) / np.abs(rmax))
        g = np.minimum(g, (eps - prg) / (np.abs(eps) + prg))
    return g


def illegitimate_flips(mesh, flips, l_gpu, l_orc, ub, P, bounds):
    """Flipped entries that are NOT roundoff decisions: for neither search
    direction of the entry (row i with P_ij, row j with P_ji) is a constraint
    met to within FLIP_TIGHT at min(l_gpu, l_orc) or at max(l_gpu, l_orc).
    ub [S][n] start states, P [S][nnz] directions, bounds [3][n] -- the
    oracle's, of the pass in question."""
    ks = np.nonzero(flips)[0]
    if ks.size == 0:
        return ks
    rows = mesh.row_of_entry()
    T = H.transpose_index(mesh)
    lo = np.minimum(l_gpu[ks], l_orc[ks])
    hi = np.maximum(l_gpu[ks], l_orc[ks])
    tight = np.zeros(ks.size, dtype=bool)
    for kk, r in ((ks, rows[ks]), (T[ks], mesh.col[ks])):
        m_lo = _constraint_margin(ub[:, r], P[:, kk], bounds[:, r], lo)
        m_hi = _constraint_margin(ub[:, r], P[:, kk], bounds[:, r], hi)
        m = np.minimum(m_lo, m_hi)
        tight |= np.abs(m) <= FLIP_TIGHT
    return ks[~tight]


CASES = {
    "vortex32": lambda: (W.vortex_workload(32).mesh, W.vortex_workload(32).U0, None),
    "cylinder": lambda: (lambda m, U0, bs: (m, W.perturbed_state(m, 7), bs))(*W.cylinder_problem(12)),
    "strip_strong_shock": lambda: (lambda m: (m, W.riemann_initial(m, "strong_shock"), None))(W.riemann_strip(90)),
}


@pytest.mark.parametrize("relax", [False, True])
@pytest.mark.parametrize("case", sorted(CASES))
def test_first_pass_limiter_matches_oracle(case, relax):
    """P_ij at 1e-12 of its largest entry per component; l_ij exact at the
    exits and within L_CONT_TOL inside (0, 1), flips counted (Algorithm 1,
    steps 4-5)."""
    mesh, U0, bs = CASES[case]()
    orc = oracle.Oracle(mesh, bnd_state=bs, bound_relaxation=relax)
    U0 = orc.apply_bc(U0)
    _, tau, tr = orc.forward_euler(U0, trace=True)
    s = solver_for(mesh, bs, bound_relaxation=relax)
    s.set_state(U0)
    s.stage(tau)
    P = s.trace(B.EH_TRACE_P_PASS1)
    # per component, relative to its largest entry; a component that is only
    # roundoff everywhere (the transverse momentum of a 1D problem) against
    # 1e-3 of the largest component instead
    pmax = np.abs(tr["P"]).max(axis=1, keepdims=True)
    scale = np.maximum(pmax, 1e-3 * pmax.max()) + 1e-300
    perr = (np.abs(P - tr["P"]) / scale).max()
    H.record(f"P_pass1[{case},relax={relax}]", perr, None, 1e-12)
    assert perr <= 1e-12, perr
    l1_g, l1_o = s.trace(B.EH_TRACE_L_PASS1), tr["lij"][0]
    assert np.all((l1_g >= 0.0) & (l1_g <= 1.0))
    assert np.array_equal(l1_g, l1_g[H.transpose_index(mesh)])  # symmetrised
    flips = limiter_flips(l1_g, l1_o)
    inside = (l1_g > 0.0) & (l1_g < 1.0) & (l1_o > 0.0) & (l1_o < 1.0) & ~flips
    cont = float(np.abs(l1_g - l1_o)[inside].max()) if inside.any() else 0.0
    bad = illegitimate_flips(mesh, flips, l1_g, l1_o, tr["UL"], tr["P"], tr["bounds"])
    H.record(f"l_pass1[{case},relax={relax}]", cont, None, L_CONT_TOL, flips=int(flips.sum()),
             entries=int(mesh.nnz), inside=int(inside.sum()), illegitimate=int(bad.size))
    print(case, relax, "flips", int(flips.sum()), "of", mesh.nnz, "inside", int(inside.sum()), "max diff inside", cont)
    assert bad.size == 0, (bad[:10], l1_g[bad[:10]], l1_o[bad[:10]])


def _stage_resync(mesh, U0, bs, steps, relax=False):
    """Runs ``steps`` SSPRK(3,3) steps stage by stage on the GPU (eh_stage: one
    forward-Euler stage plus the post-processing of Sec. 4; the SSP
    combinations of eq. SPPRK33 on the host) and, at every stage, the oracle on
    the GPU's input of that stage. Returns per-stage records."""
    orc = oracle.Oracle(mesh, bnd_state=bs, bound_relaxation=relax)
    s = solver_for(mesh, bs, bound_relaxation=relax)
    U = orc.apply_bc(U0)
    rows = mesh.row_of_entry()
    recs = []

    def spread_nodes(mask_nodes):
        """The nodes of mask_nodes and their neighbours."""
        out = mask_nodes.copy()
        out[mesh.col[mask_nodes[rows]]] = True
        return out

    def stage(Uin, tau):
        s.set_state(Uin)
        used = s.stage(tau)
        got = s.get_state()
        l1, ll = s.trace(B.EH_TRACE_L_PASS1), s.trace(B.EH_TRACE_L_LAST)
        ref, _, tr = orc.forward_euler(Uin, used, trace=True)
        ref = orc.apply_bc(ref)
        f1 = limiter_flips(l1, tr["lij"][0])
        f2 = limiter_flips(ll, tr["lij"][-1])
        # every first-pass difference (a flip, or a continuous difference of
        # the iterated search) changes the second pass's direction (1 - l) P_ij
        # and start states U^(1) of both nodes, hence every second search in
        # their rows
        d1 = np.abs(l1 - tr["lij"][0]) > L_SAME_TOL
        n1 = np.zeros(mesh.n, dtype=bool)
        n1[rows[d1]] = True
        n1[mesh.col[d1]] = True
        n1 = spread_nodes(n1)
        # first-pass flips, and second-pass flips whose inputs agree, must be
        # roundoff decisions on the oracle's own data of that pass
        f2_own = f2 & ~n1[rows] & ~n1[mesh.col]
        P2 = tr["P"] * (1.0 - tr["lij"][0])
        bad = illegitimate_flips(mesh, f1, l1, tr["lij"][0], tr["UL"], tr["P"], tr["bounds"]).size
        bad += illegitimate_flips(mesh, f2_own, ll, tr["lij"][-1], tr["Upass"][0], P2, tr["bounds"]).size
        # the state is compared away from every node whose limiters differ
        d2 = np.abs(ll - tr["lij"][-1]) > L_SAME_TOL
        touched = n1.copy()
        touched[rows[d2]] = True
        touched[mesh.col[d2]] = True
        keep = ~touched
        err = H.rel_l1(got[:, keep], ref[:, keep]).max() if keep.any() else 0.0
        recs.append(dict(err=float(err), flips=int(f1.sum() + f2.sum()), illegitimate=int(bad),
                         nodes_excluded=int(touched.sum())))
        return got, used

    for _ in range(steps):
        w1, tau = stage(U, 0.0)
        v, _ = stage(w1, tau)
        w2 = U + 0.25 * (v - U)
        v, _ = stage(w2, tau)
        U = U + (2.0 / 3.0) * (v - U)
    return recs


@pytest.mark.parametrize("case", ["vortex64_strict", "cylinder16_strict", "vortex64_relaxed", "cylinder16_relaxed"])
def test_stage_resynchronised_100_steps(case):
    """100 steps, every stage's GPU result within 1e-12 of the oracle fed the
    same input, away from flipped limiter decisions; every flip a roundoff
    decision. (With strict bounds the isentropic vortex meets its entropy
    bound to roundoff almost everywhere -- Phi is constant -- so most of its
    entries are roundoff decisions there; the relaxed runs are the
    well-conditioned counterpart.)"""
    relax = case.endswith("relaxed")
    if case.startswith("vortex"):
        w = W.vortex_workload(64)
        mesh, U0, bs = w.mesh, w.U0, None
    else:
        mesh, U0, bs = W.cylinder_problem(16)
    recs = _stage_resync(mesh, U0, bs, 100, relax=relax)
    errs = np.array([r["err"] for r in recs])
    flips = np.array([r["flips"] for r in recs])
    bad = np.array([r["illegitimate"] for r in recs])
    excl = np.array([r["nodes_excluded"] for r in recs])
    H.record(f"stage_resync_100[{case}]", errs.max(), None, H.STEP_TOL, stages=len(recs),
             stages_with_flips=int((flips > 0).sum()), flips_total=int(flips.sum()),
             illegitimate=int(bad.sum()), mean_nodes_excluded=float(excl.mean()),
             max_nodes_excluded=int(excl.max()), nodes=int(mesh.n), median_err=float(np.median(errs)))
    print(case, "max err", errs.max(), "stages with flips", int((flips > 0).sum()), "of", len(recs),
          "flips", int(flips.sum()), "illegitimate", int(bad.sum()), "mean excluded nodes", excl.mean(), "of", mesh.n)
    assert errs.max() <= H.STEP_TOL, errs.max()
    assert bad.sum() == 0


C4_KIND = [(6, 1.7), (9, 3.9), (11, 2.6)]


@pytest.mark.parametrize("relax", [True, False])
def test_batched_instances_match_oracle(relax):
    """Three C4-kind instances (Q1 cylinders, m = 6, 9, 11 cells across, Mach
    1.7, 3.9, 2.6) in one batched context, 60 steps, each with its own CFL step;
    each compared with the oracle run on that instance alone."""
    steps = 60
    inst = [W.cylinder_instance(m, mach) for m, mach in C4_KIND]
    mesh, off, bs = M.concatenate([x[0] for x in inst], [x[2] for x in inst])
    s = solver_for(mesh, bs, bound_relaxation=relax)
    s.set_instances(off)
    s.set_state(np.concatenate([x[1] for x in inst], axis=1))
    s.apply_boundary_conditions()
    s.run(steps)
    U = s.get_state()
    for k, (m_k, U0_k, bs_k) in enumerate(inst):
        orc = oracle.Oracle(m_k, bnd_state=bs_k, bound_relaxation=relax)
        U0b = orc.apply_bc(U0_k)
        ref, _ = orc.run(U0b, steps)
        err = H.rel_l1(U[:, off[k]:off[k + 1]], ref).max()
        if relax:
            tol, spread = H.RUN_TOL, None
        else:
            orf = oracle.Oracle(m_k, bnd_state=bs_k, lib=oracle.load_fma())
            spread = H.oracle_spread(lambda V: orc.run(V, steps)[0], U0b, fn_fma=lambda V: orf.run(V, steps)[0])
            tol = H.tolerance(H.RUN_TOL, spread)
        H.record(f"batched_instance[{k},relax={relax}]", err, spread, tol)
        assert err <= tol, (k, err, spread)


def test_served_requests_match_oracle():
    """Two requests through the served stream (eh_batch_admit / advance /
    poll), a P1 and a Q1 cylinder at different Mach numbers, each to its own
    t_final; each result against the oracle's solve alone to the same time."""
    reqs = []
    for m, p1, mach, tf in ((7, True, 2.2, 0.04), (9, False, 3.4, 0.03)):
        mesh = M.cylinder_channel_p1(m) if p1 else M.cylinder_channel_q1(m)
        U0 = W.uniform_state(mesh, 1.4, (mach, 0.0), 1.0)
        reqs.append((mesh, U0, np.ascontiguousarray(U0[:, mesh.bnd_node]), tf))
    b = B.Batch(1 << 30, dim=2)
    try:
        tickets = [b.admit(mesh, U0, tf, bs) for mesh, U0, bs, tf in reqs]
        assert all(t is not None for t in tickets)
        results = {}
        while len(results) < len(tickets):
            b.advance(4)
            for t in tickets:
                if t not in results:
                    out = b.poll(t)
                    if out is not None:
                        results[t] = out
    finally:
        b.close()
    for t, (mesh, U0, bs, tf) in zip(tickets, reqs):
        U, t_reached, steps = results[t]
        orc = oracle.Oracle(mesh, bnd_state=bs)
        U0b = orc.apply_bc(U0)
        ref, t_ref, steps_ref = orc.run_to(U0b, tf)
        assert steps >= steps_ref and abs(t_reached - t_ref) <= 1e-13 * tf  # steps: launched, frozen ones too
        orf = oracle.Oracle(mesh, bnd_state=bs, lib=oracle.load_fma())
        spread = H.oracle_spread(lambda V: orc.run_to(V, tf)[0], U0b, fn_fma=lambda V: orf.run_to(V, tf)[0])
        err = H.rel_l1(U, ref).max()
        tol = H.tolerance(H.RUN_TOL, spread)
        H.record(f"served_request[{mesh.name}]", err, spread, tol, steps=steps_ref)
        assert err <= tol, (err, spread)


def test_three_dimensional_large_box_matches_oracle():
    """60^3 periodic Q1 hexes: 216,000 rows of 27 entries (well past one
    wave of 64-256-row blocks on every SM); 2 steps, relaxed bounds at 1e-12
    per step, strict bounds against the oracle's spread. The limiter kernels
    capped at 256 rows in flight per SM (152 x 256 rows per sweep, so their
    grid-stride loops wrap five times) give the same bits."""
    mesh = M.structured_q1_3d(60, 60, 60, periodic=(True, True, True))
    U0 = W.perturbed_state(mesh, 11, base=dict(rho=1.0, vel=(0.5, -0.2, 0.1), p=1.0), amplitude=0.2)
    steps = 2
    for relax in (True, False):
        orc = oracle.Oracle(mesh, bound_relaxation=relax)
        ref, _ = orc.run(U0, steps)
        s = solver_for(mesh, bound_relaxation=relax)
        s.set_state(U0)
        s.run(steps)
        U = s.get_state()
        err = H.rel_l1(U, ref).max()
        s.close()
        q = solver_for(mesh, bound_relaxation=relax)
        for k in ("lim1", "pass", "final"):
            q.set_launch_shape(k, 64, 256)
        q.set_state(U0)
        q.run(steps)
        assert np.array_equal(q.get_state(), U), relax
        q.close()
        orf = oracle.Oracle(mesh, bound_relaxation=relax, lib=oracle.load_fma())
        spread = H.oracle_spread(lambda V: orc.run(V, steps)[0], U0, samples=1,
                                 fn_fma=lambda V: orf.run(V, steps)[0])
        tol = H.tolerance(steps * H.STEP_TOL, spread)
        H.record(f"box3d_216k[relax={relax}]", err, spread, tol)
        assert err <= tol, (relax, err, spread)


@pytest.mark.parametrize("mesh_fn", [lambda: W.cylinder_problem(20)[::2], lambda: (M.periodic_p1_square(40), None),
                                     lambda: (M.structured_q1_3d(9, 7, 6, periodic=(True, False, True)), None)])
def test_mesh_integers_bit_exact(mesh_fn):
    """The CSR arrays held on the device equal the uploaded ones, and the
    transpose index built by the library equals one built here independently
    (sorted keys and a binary search), bit for bit."""
    mesh, bs = mesh_fn()
    s = solver_for(mesh, bs)
    row_ptr, col, tr = s.mesh_index()
    assert np.array_equal(row_ptr, mesh.row_ptr.astype(np.int64))
    assert np.array_equal(col, mesh.col.astype(np.int32))
    assert np.array_equal(tr.astype(np.int64), H.transpose_index(mesh))
    rows = mesh.row_of_entry()
    assert np.array_equal(mesh.col[tr], rows) and np.array_equal(rows[tr], mesh.col)
