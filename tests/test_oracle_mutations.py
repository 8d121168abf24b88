"""Planted mistakes: each test compiles a copy of the oracle with one plausible
error (a wrong sign, a dropped factor, a transposed operand, a skipped step)
and checks that at least one pin rejects it. The mistakes are planted in a
temporary copy on the CPU; the oracle itself is never modified. CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M
from paper_2106_02159_gb300 import workloads as W

from . import helpers as H
from . import riemann_exact as RE

SRC = os.path.join(os.path.dirname(oracle.__file__), "euler_oracle.c")


def _mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))
    return oracle.load(oracle.build(force=True, src=str(path), out=str(tmp_path / "libmutant.so")))


# --- detectors: each returns True when the pin holds ------------------------

def _safe(fn):
    def wrapped(lib):
        try:
            return fn(lib)
        except oracle.OracleError:
            return False  # the oracle itself refused (e.g. a non-admissible state)
    wrapped.__name__ = fn.__name__
    return wrapped


def _graded(lib):
    mesh, U0, bs = W.cylinder_problem(8)
    orc = oracle.Oracle(mesh, bnd_state=bs, lib=lib)
    U, _ = orc.run(orc.apply_bc(U0), 6)
    return mesh, orc, U


@_safe
def pin_low_order_flux_form(lib):
    mesh, orc, U = _graded(lib)
    _, tau, tr = orc.forward_euler(U, trace=True)
    rows = mesh.row_of_entry()
    from .test_oracle_pins import _flux_matrix
    f = _flux_matrix(U)
    fc = np.einsum("sdk,dk->sk", f[:, :, mesh.col], mesh.cij)
    FL = -fc + tr["dij"] * (U[:, mesh.col] - U[:, rows])
    rhs = np.stack([np.bincount(rows, weights=FL[s], minlength=mesh.n) for s in range(4)])
    return bool(np.abs(U + tau * rhs / mesh.mi - tr["UL"]).max() <= 1e-12 * np.abs(U).max())


@_safe
def pin_compact_high_order_form(lib):
    mesh, orc, U = _graded(lib)
    _, tau, tr = orc.forward_euler(U, trace=True)
    rows = mesh.row_of_entry()
    FH = tr["FH"]
    BF = FH + np.stack([np.bincount(rows, weights=-(mesh.mij / mesh.mi[mesh.col]) * FH[s, mesh.col],
                                     minlength=mesh.n) for s in range(4)])
    UH = U + tau * (FH + BF) / mesh.mi
    lam = 1.0 / (np.diff(mesh.row_ptr) - 1)
    sumP = np.stack([np.bincount(rows, weights=lam[rows] * tr["P"][s], minlength=mesh.n) for s in range(4)])
    return bool(np.abs(tr["UL"] + sumP - UH).max() <= 1e-12 * np.abs(U).max())


@_safe
def pin_lambda_bound(lib):
    rng = np.random.default_rng(1)
    m = 20000
    rho = np.exp(rng.uniform(-3, 3, (2, m)))
    p = np.exp(rng.uniform(-3, 3, (2, m)))
    u = rng.uniform(-3, 3, (2, m))
    ul = W.conserved(rho[0], [u[0], 0 * u[0]], p[0]).T.copy()
    ur = W.conserved(rho[1], [u[1], 0 * u[1]], p[1]).T.copy()
    n = np.tile([1.0, 0.0], (m, 1))
    lam = oracle.lambda_max_batch(ul, ur, n, lib=lib)
    ex, _ = RE.max_wave_speed(rho[0], u[0], p[0], rho[1], u[1], p[1])
    return bool(np.all(lam >= ex * (1 - 1e-10)))


@_safe
def pin_periodic_conservation(lib):
    w = W.vortex_workload(24)
    orc = oracle.Oracle(w.mesh, lib=lib)
    U, _ = orc.run(w.U0, 2)
    d = np.abs((w.mesh.mi * U).sum(1) - (w.mesh.mi * w.U0).sum(1))
    return bool(np.all(d <= 1e-13 * (w.mesh.mi * np.abs(w.U0)).sum(1)))


@_safe
def pin_cfl_closed_form(lib):
    mesh = M.periodic_p1_square(8)
    U = W.uniform_state(mesh, 1.0, (0.0, 0.0), 1.0)
    rows = mesh.row_of_entry()
    T = H.transpose_index(mesh)
    norms = np.linalg.norm(mesh.cij, axis=0)
    upper = np.where(mesh.col > rows, norms, norms[T])
    off = rows != mesh.col
    dii = math.sqrt(1.4) * np.bincount(rows[off], weights=upper[off], minlength=mesh.n)
    expect = 0.5 * np.min(mesh.mi / (2.0 * dii))
    return math.isclose(oracle.Oracle(mesh, cfl=0.5, lib=lib).cfl_dt(U), expect, rel_tol=1e-13)


@_safe
def pin_sod_error(lib):
    mesh = W.riemann_strip(100)
    orc = oracle.Oracle(mesh, lib=lib)
    data = W.RIEMANN_CASES["sod"]
    try:
        U, t, _ = orc.run_to(W.riemann_initial(mesh, "sod"), data[-1])
    except oracle.OracleError:
        return False
    rho, _, _ = RE.sample(mesh.coords[:, 0], t, *data[:6])
    e = (mesh.mi * np.abs(U[0] - rho)).sum() / (mesh.mi * rho).sum()
    return bool(np.isfinite(e) and e < 0.025)


@_safe
def pin_indicator_small_in_smooth_flow(lib):
    mesh = M.periodic_p1_square(64)
    _, _, tr = oracle.Oracle(mesh, lib=lib).forward_euler(W.isentropic_vortex(mesh), trace=True)
    core = np.hypot(*mesh.coords.T) < 3.0
    return bool(tr["alpha"][core].max() < 0.5 and tr["alpha"][core].mean() < 0.05)


@_safe
def pin_slip_conservation(lib):
    mesh = H.all_slip(M.cylinder_channel_q1(8))
    x, y = mesh.coords.T
    bump = np.exp(-40 * ((x - 2.0) ** 2 + (y - 0.5) ** 2))
    U = W.conserved(1.0 + 0.5 * bump, [0.2 + 0 * x, 0.1 + 0 * x], 1.0 + 2.0 * bump)
    orc = oracle.Oracle(mesh, lib=lib)
    U = orc.apply_bc(U)
    m0 = (mesh.mi * U).sum(1)
    for _ in range(3):
        U, _, _ = orc.ssprk3_step(U)
    m = (mesh.mi * U).sum(1)
    return bool(abs(m[0] - m0[0]) <= 1e-13 * abs(m0[0]) and abs(m[3] - m0[3]) <= 1e-13 * abs(m0[3]))


@_safe
def pin_stage_symmetries(lib):
    w = W.vortex_workload(16)
    orc = oracle.Oracle(w.mesh, lib=lib)
    _, _, tr = orc.forward_euler(w.U0, trace=True)
    T = H.transpose_index(w.mesh)
    off = w.mesh.row_of_entry() != w.mesh.col
    return bool(np.array_equal(tr["dij"][off], tr["dij"][T][off]))


@_safe
def pin_vortex_second_order(lib):
    errs = []
    for nv in (32, 64):
        mesh = M.periodic_p1_square(nv)
        orc = oracle.Oracle(mesh, bound_relaxation=True, lib=lib)
        U, t, _ = orc.run_to(W.isentropic_vortex(mesh), 1.0)
        ex = W.isentropic_vortex(mesh, t=t)
        errs.append((mesh.mi * np.abs(U[0] - ex[0])).sum() / (mesh.mi * ex[0]).sum())
    return math.log2(errs[0] / errs[1]) >= 1.8


@_safe
def pin_characteristic_invariants(lib):
    from .test_oracle_bc import _invariants, _random_pair
    rng = np.random.default_rng(31)
    for inflow in (True, False):
        for _ in range(100):
            n, u, ud = _random_pair(rng, 2, (-0.95, -0.01) if inflow else (0.0, 0.95))
            up = oracle.bc_characteristic(u, n, ud, lib=lib)
            iu, idd, ip = _invariants(u, n), _invariants(ud, n), _invariants(up, n)
            src = idd if inflow else iu
            if not (np.isclose(ip["C1"], idd["C1"], rtol=1e-12, atol=1e-12)
                    and np.isclose(ip["C3"], iu["C3"], rtol=1e-12, atol=1e-12)
                    and np.isclose(ip["S"], src["S"], rtol=1e-11)
                    and np.allclose(ip["vt"], src["vt"], rtol=1e-12, atol=1e-12)):
                return False
    return True


@_safe
def pin_godunov_exact(lib):
    from .test_oracle_bc import G, _cons, _prim, _random_pair
    rng = np.random.default_rng(51)
    for _ in range(400):
        n, u, ud = _random_pair(rng, 2, (-2.5, 2.5), data_condition=False)
        rl, _, pl, al, ul, tl = _prim(u, n)
        rr, _, pr, ar, ur, tr = _prim(ud, n)
        if 2 * (al + ar) / (G - 1) <= ur - ul:
            continue
        rho, un, p = RE.sample(np.array([0.5]), 1.0, rl, ul, pl, rr, ur, pr, gamma=G, x0=0.5)
        _, us = RE.star_pressure(rl, ul, pl, rr, ur, pr, gamma=G)
        ref = _cons(rho[0], un[0] * n + (tl if float(us) >= 0 else tr), p[0])
        if not np.allclose(oracle.bc_godunov(u, n, ud, lib=lib), ref, rtol=1e-9, atol=1e-10):
            return False
    return True


@_safe
def pin_adaptive_cfl_accepts_admissible_low_order(lib):
    mesh = W.riemann_strip(120)
    U0 = W.riemann_initial(mesh, "strong_shock")
    U, dt, c, r = oracle.Oracle(mesh, cfl=0.5, lib=lib).ssprk3_step_adaptive(U0, 16.0)
    if not (r >= 1 and c == 16.0 / 2 ** r):
        return False
    _, _, stages = H.ssprk3_with_traces(oracle.Oracle(mesh, cfl=c, lib=lib), U0)
    for _, _, tr in stages:
        ul = tr["UL"]
        if not ((ul[0] > 0).all() and (ul[-1] - 0.5 * (ul[1:-1] ** 2).sum(0) / ul[0] > 0).all()):
            return False
    return True


@_safe
def pin_parabolic_plane_wave(lib):
    import math as _m
    from .test_oracle_parabolic import SHEAR, _box, _plane_wave, _state
    mu, lam, T = 0.01, 0.02, 0.2
    k = (1.0, 1.0 - SHEAR)
    errs = []
    for n in (16, 32):
        mesh = _box(n, "p1sheared")
        v0 = _plane_wave(mesh.coords, 0.0, mu, lam, k)
        U = _state(mesh, v0[0], v0[1], np.full(mesh.n, 10.0))
        o = oracle.Oracle(mesh, cfl=0.5, lib=lib)
        o.set_viscosity(M.parabolic_data(mesh), mu, lam, 0.0)
        for _ in range(n // 4):
            U, _ = o.parabolic_step(U, T / (n // 4))
        ex = _plane_wave(mesh.coords, T, mu, lam, k)
        errs.append(np.sqrt((mesh.mi * ((U[1:3] / U[0] - ex) ** 2).sum(0)).sum()))
    return _m.log2(errs[0] / errs[1]) >= 1.8


@_safe
def pin_parabolic_energy_conservation(lib):
    from .test_oracle_parabolic import _box, _random_smooth
    mesh = _box(20, "q1")
    U = _random_smooth(mesh, 1)
    o = oracle.Oracle(mesh, cfl=0.5, lib=lib)
    o.set_viscosity(M.parabolic_data(mesh), 0.05, 0.03, 0.04)
    U1, _ = o.parabolic_step(U, 0.01)
    E0, E1 = (mesh.mi * U[3]).sum(), (mesh.mi * U1[3]).sum()
    return abs(E1 - E0) <= 1e-11 * E0


@_safe
def pin_parabolic_energy_conservation_traction_free(lib):
    from .test_oracle_parabolic import _state
    mesh = M.structured_q1(14, 10, 0.0, 1.0, 0.0, 0.8)
    x = mesh.coords
    U = _state(mesh, np.sin(2.0 * x[:, 0]) * np.cos(1.5 * x[:, 1]), np.cos(2.5 * x[:, 0] * x[:, 1]),
               3.0 + x[:, 0] * x[:, 1], 1.0 + 0.2 * x[:, 0])
    o = oracle.Oracle(mesh, cfl=0.5, lib=lib)
    o.set_viscosity(M.parabolic_data(mesh), 0.05, 0.03, 0.04)
    U1, _ = o.parabolic_step(U, 0.02)
    E0, E1 = (mesh.mi * U[3]).sum(), (mesh.mi * U1[3]).sum()
    return abs(E1 - E0) <= 1e-11 * E0


@_safe
def pin_parabolic_fct(lib):
    from .test_oracle_parabolic import _box, _state
    mesh = _box(32, "q1")
    x = mesh.coords
    e = np.where(np.abs(x[:, 0] - 0.5) < 0.1, 50.0, 1e-3)
    U = _state(mesh, np.zeros(mesh.n), np.zeros(mesh.n), e)
    o = oracle.Oracle(mesh, cfl=0.5, lib=lib)
    o.set_viscosity(M.parabolic_data(mesh), 0.0, 0.0, 5.0)
    U1, info = o.parabolic_step(U, 0.05)
    e1 = U1[3] / U1[0]
    return bool(info["limited"] == 1 and e1.min() >= e.min() * (1 - 1e-12)
                and abs((mesh.mi * U1[3]).sum() - (mesh.mi * U[3]).sum()) <= 1e-11 * (mesh.mi * U[3]).sum())


MUTATIONS = {
    "bar_state_sign": ("ubar[s] = dL > 0.0 ? 0.5 * (ui[s] + uj[s]) - dfc[s] / (2.0 * dL) : ui[s];",
                       "ubar[s] = dL > 0.0 ? 0.5 * (ui[s] + uj[s]) + dfc[s] / (2.0 * dL) : ui[s];",
                       pin_low_order_flux_form),
    "lambda_shock_factor": ("double k = (gamma + 1.0) / (2.0 * gamma);", "double k = (gamma - 1.0) / (2.0 * gamma);",
                            pin_lambda_bound),
    "lambda_right_velocity_not_divided": ("  un_r /= rho_r;\n", "\n", pin_lambda_bound),
    "b_ij_b_ji_transposed": ("double val = bij * c->FH[s * n + j] - bji * c->FH[s * n + i]",
                             "double val = bji * c->FH[s * n + j] - bij * c->FH[s * n + i]",
                             pin_compact_high_order_form),
    "limiter_not_symmetrised": ("c->lij[k] = fmin(c->lraw[k], c->lraw[c->transpose[k]]);",
                                "c->lij[k] = c->lraw[k];", pin_periodic_conservation),
    "cfl_missing_factor_two": ("double t = -p->cfl * p->mi[i] / (2.0 * c->dij[kdiag]);",
                               "double t = -p->cfl * p->mi[i] / (c->dij[kdiag]);", pin_cfl_closed_form),
    "indicator_commutator_sign": ("N += a - b;", "N += a + b;", pin_indicator_small_in_smooth_flow),
    "slip_projection_sign": ("U[(1 + d) * n + i] -= mn * p->bnd_normal[(int64_t)d * p->n_bnd + b];",
                             "U[(1 + d) * n + i] += mn * p->bnd_normal[(int64_t)d * p->n_bnd + b];",
                             pin_slip_conservation),
    "transpose_fill_skipped": ("if (j < i) c->dij[k] = c->dij[c->transpose[k]];",
                               "if (j < i) c->dij[k] = 1.0;", pin_stage_symmetries),
    "ssp_stage_weight": ("w[q] = u0[q] + 0.25 * (v[q] - u0[q]);", "w[q] = u0[q] + 0.5 * (v[q] - u0[q]);",
                         pin_vortex_second_order),
    "characteristic_c1_sign": ("double c1d = wd.vn - 2.0 * wd.a / (gamma - 1.0);",
                               "double c1d = wd.vn + 2.0 * wd.a / (gamma - 1.0);", pin_characteristic_invariants),
    "characteristic_entropy_source": ("const nprim *src = w.vn < 0.0 ? &wd : &w;",
                                      "const nprim *src = w.vn < 0.0 ? &w : &wd;", pin_characteristic_invariants),
    "godunov_shock_density": ("out->rho = l->rho * (p / l->p + g6) / (g6 * p / l->p + 1.0);",
                              "out->rho = l->rho * (p / l->p - g6) / (g6 * p / l->p + 1.0);", pin_godunov_exact),
    "adaptive_cfl_ignores_low_order_states": ("(st == ORACLE_OK && (c->low_not_admissible > 0 ||",
                                              "(st == ORACLE_OK && (0 ||", pin_adaptive_cfl_accepts_admissible_low_order),
    "parabolic_bulk_coefficient": ("const double lm = pp->lambda - 2.0 * pp->mu / 3.0;\n  for (int i = 0; i < n; ++i) {\n    if (wall[i])",
                                   "const double lm = pp->lambda + 2.0 * pp->mu / 3.0;\n  for (int i = 0; i < n; ++i) {\n    if (wall[i])",
                                   pin_parabolic_plane_wave),
    # in the continuum both orders give grad div v (so the waves converge either way); the
    # discrete dissipation then differs from int sigma:eps, and total energy drifts
    "parabolic_stress_transpose": ("pp->mu * pp->G[(m * 2 + a) * nnz + k]", "pp->mu * pp->G[(a * 2 + m) * nnz + k]",
                                   pin_parabolic_energy_conservation_traction_free),
    "parabolic_crank_nicolson_extrapolation": ("eH[i] = 2.0 * eh[i] - en[i];", "eH[i] = eh[i];",
                                               pin_parabolic_energy_conservation),
    "parabolic_viscous_heating_factor": ("const double se = 2.0 * pp->mu * ee + lm * div * div;",
                                         "const double se = pp->mu * ee + lm * div * div;",
                                         pin_parabolic_energy_conservation),
    "parabolic_fct_limiter_sides": ("const double l = A > 0.0 ? fmin(Rp[i], Rm[j]) : fmin(Rm[i], Rp[j]);",
                                    "const double l = A > 0.0 ? fmin(Rp[i], Rp[j]) : fmin(Rm[i], Rm[j]);",
                                    pin_parabolic_fct),
    "godunov_tangential_side": ("  for (int d = 0; d < dim; ++d) out->vt[d] = r->vt[d];\n  if (p > r->p) {",
                                "  for (int d = 0; d < dim; ++d) out->vt[d] = l->vt[d];\n  if (p > r->p) {",
                                pin_godunov_exact),
}


@pytest.fixture(scope="module")
def real_lib():
    return oracle.load()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_rejects_planted_mistake(name, tmp_path, real_lib):
    old, new, pin = MUTATIONS[name]
    assert pin(real_lib), f"pin {pin.__name__} must hold for the oracle itself"
    mlib = _mutant(tmp_path, old, new)
    assert not pin(mlib), f"planted mistake {name!r} was not caught by {pin.__name__}"
