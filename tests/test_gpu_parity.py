"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Element-by-element on the same seeded inputs: one forward-Euler stage with its
intermediates, one SSPRK(3,3) step and 100 steps on the isentropic-vortex
workload, the cylinder channel with every boundary kind, and a strong-shock
strip; determinism, graph replay and error paths. Needs a GPU.

Tolerances (relative L1 per component). With relaxed bounds the method is
well conditioned and the targets are 1e-12 per step and 1e-9 after 100 steps.
With the paper's strict bounds the line search decides l_ij = 0 or 1 from the
last bits wherever the bounds are as tight as roundoff (near-uniform flow,
isentropic regions, shock fronts), so the oracle itself moves by up to ~1e-10
per step and ~1e-7 over 100 steps when its input is perturbed by one ulp or
when the same source is compiled with fused multiply-adds (the GPU compiler's
default rounding). A flip is a discrete event, so the difference between two
valid roundings is heavy-tailed: every run with shocks or strict bounds is
held to max(target, F x the largest of those measured spreads of the oracle),
F = helpers.SPREAD_FACTOR; the smooth relaxed-bound runs are held to the target
itself. Every comparison is logged with helpers.record. The arithmetic itself
is held to 1e-12 per stage, flips excluded and counted, by the
stage-resynchronised runs of test_gpu_parity_limiter.py."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import binding as B
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from . import helpers as H

pytestmark = pytest.mark.gpu

STEP_TOL = H.STEP_TOL
RUN_TOL = H.RUN_TOL
rel_l1 = H.rel_l1
oracle_spread = H.oracle_spread
tolerance = H.tolerance


def fma_twin(orc, mesh, bs, **kw):
    """The same oracle configuration on the contracted build."""
    return oracle.Oracle(mesh, bnd_state=bs, lib=oracle.load_fma(), **kw)


def solver_for(mesh, bnd_state=None, **kw):
    s = B.Solver(dim=mesh.dim, **kw)
    s.upload_mesh(mesh, bnd_state)
    return s


CASES = {
    "vortex32": lambda: (W.vortex_workload(32).mesh, W.vortex_workload(32).U0, None),
    "cylinder": lambda: (lambda m, U0, bs: (m, W.perturbed_state(m, 7), bs))(*W.cylinder_problem(12)),
    "strip_strong_shock": lambda: (lambda m: (m, W.riemann_initial(m, "strong_shock"), None))(W.riemann_strip(90)),
}


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    oracle.set_threads(0)


@pytest.mark.parametrize("case", sorted(CASES))
def test_stage_intermediates_match_oracle(case):
    mesh, U0, bs = CASES[case]()
    orc = oracle.Oracle(mesh, bnd_state=bs)
    U0 = orc.apply_bc(U0)
    ref, tau_ref, tr = orc.forward_euler(U0, trace=True)
    ref = orc.apply_bc(ref)
    s = solver_for(mesh, bs)
    s.set_state(U0)
    tau = s.stage()
    assert abs(tau - tau_ref) <= 1e-13 * tau_ref
    assert s.trace(B.EH_TRACE_TAU_BOUND) == pytest.approx(tr["tau_bound"], rel=1e-13)
    d = s.trace(B.EH_TRACE_D_IJ)
    assert np.abs(d - tr["dij"]).max() <= 1e-13 * np.abs(tr["dij"]).max()
    # alpha is |N|/D; compare where the row's states differ (D well above roundoff)
    alpha = s.trace(B.EH_TRACE_ALPHA)
    rows = mesh.row_of_entry()
    var = np.zeros(mesh.n)
    np.maximum.at(var, rows, np.abs(U0[0, mesh.col] - U0[0, rows]) / U0[0, rows])
    sel = var > 1e-6
    if sel.any():
        assert np.abs(alpha - tr["alpha"])[sel].max() <= 1e-9
    assert np.all((alpha >= 0) & (alpha <= 1))
    for what, key in ((B.EH_TRACE_U_LOW, "UL"), (B.EH_TRACE_F_HIGH, "FH")):
        got = s.trace(what)
        # relative to the array's largest entry: F^H sums terms that cancel,
        # so a component's own maximum can sit near its roundoff
        scale = np.abs(tr[key]).max() + 1e-300
        assert (np.abs(got - tr[key]) / scale).max() <= 1e-12, key
    bounds = s.trace(B.EH_TRACE_BOUNDS)
    assert np.allclose(bounds, tr["bounds"], rtol=1e-13, atol=0)
    orf = fma_twin(orc, mesh, bs)
    spread = oracle_spread(lambda U: orc.forward_euler(U, tau_ref)[0], U0,
                           fn_fma=lambda U: orf.forward_euler(U, tau_ref)[0])
    tol = tolerance(STEP_TOL, spread)
    up1 = s.trace(B.EH_TRACE_U_PASS1)
    H.record(f"stage_upass1[{case}]", rel_l1(up1, tr["Upass"][0]).max(), spread, tol)
    assert rel_l1(up1, tr["Upass"][0]).max() <= tol
    l1 = s.trace(B.EH_TRACE_L_PASS1)
    T = H.transpose_index(mesh)
    assert np.array_equal(l1, l1[T])
    assert np.all((l1 >= 0) & (l1 <= 1))
    U1 = s.get_state()
    H.record(f"stage[{case}]", rel_l1(U1, ref).max(), spread, tol)
    assert rel_l1(U1, ref).max() <= tol, (rel_l1(U1, ref), spread)


@pytest.mark.parametrize("relax", [False, True])
@pytest.mark.parametrize("case", sorted(CASES))
def test_ssprk3_step_matches_oracle(case, relax):
    mesh, U0, bs = CASES[case]()
    orc = oracle.Oracle(mesh, bnd_state=bs, bound_relaxation=relax)
    U0 = orc.apply_bc(U0)
    ref, dt_ref, bounds_ref = orc.ssprk3_step(U0)
    s = solver_for(mesh, bs, bound_relaxation=relax)
    s.set_state(U0)
    dt = s.step()
    assert abs(dt - dt_ref) <= 1e-13 * dt_ref
    err = rel_l1(s.get_state(), ref).max()
    orf = fma_twin(orc, mesh, bs, bound_relaxation=relax)
    spread = oracle_spread(lambda U: orc.ssprk3_step(U, dt_ref)[0], U0,
                           fn_fma=lambda U: orf.ssprk3_step(U, dt_ref)[0])
    H.record(f"ssprk3_step[{case},relax={relax}]", err, spread, tolerance(STEP_TOL, spread))
    assert err <= tolerance(STEP_TOL, spread), (err, spread)
    if relax and case.startswith("vortex"):
        assert err <= STEP_TOL
    diag = s.diagnostics()
    assert np.allclose(diag["last_stage_bound"], bounds_ref, rtol=1e-12)


@pytest.mark.parametrize("relax", [False, True])
def test_vortex_100_steps_matches_oracle(relax):
    """The 64x64 P1 isentropic-vortex workload, CFL 0.5, 100 steps, FP64."""
    w = W.vortex_workload(64)
    orc = oracle.Oracle(w.mesh, cfl=0.5, bound_relaxation=relax)
    ref, t_ref = orc.run(w.U0, 100)
    s = solver_for(w.mesh, bound_relaxation=relax)
    s.set_state(w.U0)
    s.run(100)
    err = rel_l1(s.get_state(), ref).max()
    if relax:
        H.record("vortex_100_steps[relax]", err, None, RUN_TOL)
        assert err <= RUN_TOL, err
    else:
        orf = fma_twin(orc, w.mesh, None, cfl=0.5)
        spread = oracle_spread(lambda U: orc.run(U, 100)[0], w.U0, fn_fma=lambda U: orf.run(U, 100)[0])
        H.record("vortex_100_steps[strict]", err, spread, tolerance(RUN_TOL, spread))
        assert err <= tolerance(RUN_TOL, spread), (err, spread)
    assert s.diagnostics()["not_admissible"] == 0


@pytest.mark.parametrize("relax", [False, True])
def test_cylinder_100_steps_matches_oracle(relax):
    mesh, U0, bs = W.cylinder_problem(16)
    orc = oracle.Oracle(mesh, bnd_state=bs, bound_relaxation=relax)
    U0 = orc.apply_bc(U0)
    ref, _ = orc.run(U0, 100)
    s = solver_for(mesh, bs, bound_relaxation=relax)
    s.set_state(U0)
    s.run(100)
    err = rel_l1(s.get_state(), ref).max()
    orf = fma_twin(orc, mesh, bs, bound_relaxation=relax)
    spread = oracle_spread(lambda U: orc.run(U, 100)[0], U0, fn_fma=lambda U: orf.run(U, 100)[0])
    H.record(f"cylinder_100_steps[relax={relax}]", err, spread, tolerance(RUN_TOL, spread))
    assert err <= tolerance(RUN_TOL, spread), (err, spread)


@pytest.mark.parametrize("relax,passes", [(True, 2), (True, 3), (False, 1), (False, 3)])
def test_options_match_oracle(relax, passes):
    mesh, U0, bs = W.cylinder_problem(10)
    U0 = W.perturbed_state(mesh, 3)
    orc = oracle.Oracle(mesh, bnd_state=bs, bound_relaxation=relax, limiter_passes=passes)
    U0 = orc.apply_bc(U0)
    ref, _ = orc.run(U0, 5)
    s = solver_for(mesh, bs, bound_relaxation=relax, limiter_passes=passes)
    s.set_state(U0)
    for _ in range(5):
        s.step(sync=False)
    err = rel_l1(s.get_state(), ref).max()
    orf = fma_twin(orc, mesh, bs, bound_relaxation=relax, limiter_passes=passes)
    spread = oracle_spread(lambda U: orc.run(U, 5)[0], U0, fn_fma=lambda U: orf.run(U, 5)[0])
    H.record(f"options[relax={relax},passes={passes}]", err, spread, tolerance(5 * STEP_TOL, spread))
    assert err <= tolerance(5 * STEP_TOL, spread), (err, spread)


def test_generic_gamma_path_matches_oracle():
    """gamma != 7/5 takes the pow() path of every root and power."""
    w = W.vortex_workload(24)
    U0 = W.conserved(*[np.asarray(a) for a in (w.U0[0],)], [w.U0[1] / w.U0[0], w.U0[2] / w.U0[0]],
                     0.4 * (w.U0[3] - 0.5 * (w.U0[1] ** 2 + w.U0[2] ** 2) / w.U0[0]), gamma=1.3)
    orc = oracle.Oracle(w.mesh, gamma=1.3, bound_relaxation=True)
    ref, _ = orc.run(U0, 10)
    s = solver_for(w.mesh, gamma=1.3, bound_relaxation=True)
    s.set_state(U0)
    s.run(10)
    assert rel_l1(s.get_state(), ref).max() <= 10 * STEP_TOL


def test_three_dimensional_q1_matches_oracle():
    """3D trilinear hexes, 27-point rows, periodic box."""
    mesh = M.structured_q1_3d(6, 5, 4, periodic=(True, True, True))
    U0 = W.perturbed_state(mesh, 11, base=dict(rho=1.0, vel=(0.5, -0.2, 0.1), p=1.0), amplitude=0.2)
    orc = oracle.Oracle(mesh)
    ref, _ = orc.run(U0, 3)
    s = solver_for(mesh)
    s.set_state(U0)
    s.run(3)
    err = rel_l1(s.get_state(), ref).max()
    orf = fma_twin(orc, mesh, None)
    spread = oracle_spread(lambda U: orc.run(U, 3)[0], U0, fn_fma=lambda U: orf.run(U, 3)[0])
    H.record("box3d_3_steps[strict]", err, spread, tolerance(3 * STEP_TOL, spread))
    assert err <= tolerance(3 * STEP_TOL, spread), (err, spread)
    # relaxed bounds: well conditioned, held to the target itself
    orc = oracle.Oracle(mesh, bound_relaxation=True)
    ref, _ = orc.run(U0, 3)
    s = solver_for(mesh, bound_relaxation=True)
    s.set_state(U0)
    s.run(3)
    assert rel_l1(s.get_state(), ref).max() <= 3 * STEP_TOL


def test_bitwise_determinism_and_graph_replay():
    mesh, U0, bs = W.cylinder_problem(12)
    U0 = W.perturbed_state(mesh, 5)
    outs = []
    for mode in ("step", "step", "run"):
        s = solver_for(mesh, bs)
        s.set_state(U0)
        s.apply_boundary_conditions()
        if mode == "step":
            for _ in range(7):
                s.step(sync=False)
        else:
            s.run(7)
        outs.append(s.get_state())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


def test_uniform_state_fixed_point_on_gpu():
    cyl = M.cylinder_channel_q1(8)
    U = W.uniform_state(cyl, 1.0, (0.0, 0.0), 1.0)
    s = solver_for(cyl, U[:, cyl.bnd_node].copy())
    s.set_state(U)
    s.run(20)
    assert np.array_equal(s.get_state(), U)


def test_error_paths():
    w = W.vortex_workload(16)
    s = solver_for(w.mesh)
    bad = w.U0.copy()
    bad[0, 5] = -1.0
    with pytest.raises(B.EulerError) as e:
        s.set_state(bad)
    assert e.value.status == B.EH_ERR_NOT_ADMISSIBLE
    with pytest.raises(B.EulerError) as e:
        s.step()
    assert e.value.status == B.EH_ERR_STATE
    s.set_state(w.U0)
    dt = s.cfl_dt()
    with pytest.raises(B.EulerError) as e:
        s.step(dt * 2.5)  # above the c_cfl = 1 limit (cfl = 0.5)
    assert e.value.status == B.EH_ERR_CFL
    # the error is sticky until the next eh_set_state; the state is unchanged
    out = np.empty_like(w.U0)
    with pytest.raises(B.EulerError) as e:
        s.get_state(out)
    assert e.value.status == B.EH_ERR_CFL
    assert np.array_equal(out, w.U0)
    s.set_state(w.U0)
    s.step()
    # empty / oversize / non-symmetric meshes
    m = w.mesh
    with pytest.raises(B.EulerError) as e:
        import dataclasses
        s2 = B.Solver()
        bad_col = m.col.copy()
        bad_col[1], bad_col[2] = bad_col[2], bad_col[1]  # unsorted row
        s2.upload_mesh(dataclasses.replace(m, col=bad_col))
    assert e.value.status == B.EH_ERR_BAD_MESH


def test_full_size_sampled_parity():
    """The benchmark workload at full size (~4.0M-vertex Q1 cylinder channel):
    the CFL step on the whole mesh, then one SSPRK(3,3) step on the GPU, checked
    node by node on sampled vertices (interior and every boundary kind) against
    the oracle run on the sampled vertices' dependency closure (one step reaches
    ~18 rings; the closure keeps 24)."""
    m = M.cylinder_m_for_vertices(4_000_000)
    mesh, _, bs = W.cylinder_problem(m)
    U0 = W.perturbed_state(mesh, 2106)
    dt = oracle.Oracle(mesh, bnd_state=bs).cfl_dt(U0)
    s = solver_for(mesh, bs)
    s.set_state(U0)
    assert abs(s.cfl_dt() - dt) <= 1e-13 * dt
    s.step(dt)
    U1 = s.get_state()
    assert s.diagnostics()["not_admissible"] == 0
    rng = np.random.default_rng(4)
    seeds = list(rng.choice(mesh.n, 48, replace=False))
    for kind in (M.BC_SLIP, M.BC_DIRICHLET, M.BC_DO_NOTHING):
        nodes = mesh.bnd_node[mesh.bnd_kind == kind]
        seeds += list(rng.choice(nodes, 6, replace=False))
    seeds = np.unique(seeds)  # submesh() returns the seeds' new ids in sorted order
    sub, old, seed_new, sub_bs = H.submesh(mesh, seeds, 24, bs)
    orc = oracle.Oracle(sub, bnd_state=sub_bs)
    ref, _, _ = orc.ssprk3_step(U0[:, old], dt)
    orf = oracle.Oracle(sub, bnd_state=sub_bs, lib=oracle.load_fma())
    twins = [orf.ssprk3_step(U0[:, old], dt)[0]]
    rng_noise = np.random.default_rng(0)
    for _ in range(H.SPREAD_SAMPLES):  # the same spread samples as H.oracle_spread, in this test's metric
        Up = U0[:, old] * (1.0 + 2.2e-16 * rng_noise.choice([-1.0, 0.0, 1.0], (U0.shape[0], old.size)))
        twins.append(orc.ssprk3_step(Up, dt)[0])
    got = U1[:, np.asarray(seeds)]
    want = ref[:, seed_new]
    scale = np.abs(want).max(0)
    err = np.abs(got - want).max(0) / scale
    spread = np.max([np.abs(t[:, seed_new] - want).max(0) / scale for t in twins], axis=0)
    H.record("full_size_sampled[cylinder 4.0M]", err.max(), spread.max(), tolerance(1e-12, spread.max()),
             median=float(np.median(err)), p90=float(np.percentile(err, 90)))
    # three stages over ~18 rings: a seed within reach of a limiter decision
    # taken on roundoff moves by more than the alternative roundings happened
    # to move it; that part of the check is test_full_size_stage_parity's,
    # which excludes exactly those seeds and checks every flip. Here: most
    # seeds at roundoff, none far off.
    assert np.median(err) <= 1e-13 and np.percentile(err, 90) <= 1e-12, (np.median(err), np.percentile(err, 90))
    assert err.max() <= 1e-9, err.max()


def test_full_size_stage_parity():
    """The same workload (4.0M vertices), one forward-Euler stage (eh_stage,
    with the traced limiters) from the perturbed state: every sampled vertex
    outside the reach of a limiter difference agrees with the oracle (run on
    its dependency closure: one stage reaches ~6 rings, the closure keeps 12)
    to 1e-12 of its largest component, and every limiter flip near the
    samples whose inputs agree is a roundoff decision."""
    from . import test_gpu_parity_limiter as TL
    m = M.cylinder_m_for_vertices(4_000_000)
    mesh, _, bs = W.cylinder_problem(m)
    U0 = W.perturbed_state(mesh, 2106)
    s = solver_for(mesh, bs)
    s.set_state(U0)
    s.apply_boundary_conditions()
    U0 = s.get_state()
    tau = s.stage(0.0)
    U1 = s.get_state()
    l1_full, ll_full = s.trace(B.EH_TRACE_L_PASS1), s.trace(B.EH_TRACE_L_LAST)
    s.close()
    rng = np.random.default_rng(5)
    seeds = list(rng.choice(mesh.n, 96, replace=False))
    for kind in (M.BC_SLIP, M.BC_DIRICHLET, M.BC_DO_NOTHING):
        seeds += list(rng.choice(mesh.bnd_node[mesh.bnd_kind == kind], 8, replace=False))
    seeds = np.unique(seeds)
    sub, old, seed_new, sub_bs = H.submesh(mesh, seeds, 12, bs)
    orc = oracle.Oracle(sub, bnd_state=sub_bs)
    ref, _, tr = orc.forward_euler(U0[:, old], tau, trace=True)
    ref = orc.apply_bc(ref)
    # the closure's entries in the full mesh (CSR keys are sorted)
    srows = sub.row_of_entry()
    full_key = mesh.row_of_entry().astype(np.int64) * mesh.n + mesh.col
    kmap = np.searchsorted(full_key, old[srows].astype(np.int64) * mesh.n + old[sub.col])
    l1, ll = l1_full[kmap], ll_full[kmap]
    # rows within 4 rings of the seeds: their limiters are exact in the closure
    near = np.zeros(sub.n, dtype=bool)
    near[seed_new] = True
    for _ in range(4):
        near[sub.col[near[srows]]] = True
    on = near[srows]
    f1 = TL.limiter_flips(l1, tr["lij"][0]) & on
    d1 = (np.abs(l1 - tr["lij"][0]) > TL.L_SAME_TOL) & on
    d2 = (np.abs(ll - tr["lij"][-1]) > TL.L_SAME_TOL) & on
    reach = np.zeros(sub.n, dtype=bool)
    reach[srows[d1]] = True
    reach[sub.col[d1]] = True
    reach[sub.col[reach[srows]]] = True
    reach[srows[d2]] = True
    reach[sub.col[d2]] = True
    bad = TL.illegitimate_flips(sub, f1, l1, tr["lij"][0], tr["UL"], tr["P"], tr["bounds"])
    keep = ~reach[seed_new]
    got, want = U1[:, seeds[keep]], ref[:, seed_new[keep]]
    err = (np.abs(got - want).max(0) / np.abs(want).max(0)) if keep.any() else np.zeros(1)
    H.record("full_size_stage[cylinder 4.0M]", err.max(), None, 1e-12, seeds=int(seeds.size),
             seeds_in_reach_of_flips=int((~keep).sum()), flips_near=int(f1.sum()), illegitimate=int(bad.size))
    assert keep.sum() >= seeds.size // 2
    assert err.max() <= 1e-12, err.max()
    assert bad.size == 0
