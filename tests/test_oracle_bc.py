"""Pins of the oracle's non-reflecting boundary post-processing (Sec. 4.2):
the characteristic variables (Sec. 4.2.2) and the Godunov value (Sec. 4.2.1).
The checks are the defining relations, not the closed forms: invariants of
the output against the prescribed ones, the exact Riemann solution of
tests/riemann_exact.py (pinned there by jump conditions), admissibility
(Lemma 4.3), fixed points and rotation invariance. CPU only."""
import numpy as np
import pytest

import oracle

from . import riemann_exact as RE

G = 1.4


def _cons(rho, v, p):
    v = np.asarray(v, dtype=float)
    return np.concatenate([[rho], rho * v, [p / (G - 1.0) + 0.5 * rho * v @ v]])


def _prim(u, n):
    rho = u[0]
    v = u[1:-1] / rho
    p = (G - 1.0) * (u[-1] - 0.5 * rho * v @ v)
    a = np.sqrt(G * p / rho)
    vn = v @ n
    return rho, v, p, a, vn, v - vn * n


def _invariants(u, n):
    rho, v, p, a, vn, vt = _prim(u, n)
    return dict(C1=vn - 2 * a / (G - 1), C3=vn + 2 * a / (G - 1), S=p * rho ** -G, vt=vt)


def _random_pair(rng, dim, vn_range, data_condition=True):
    """Admissible U and U^D along a random unit normal n."""
    n = rng.normal(size=dim)
    n /= np.linalg.norm(n)
    out = []
    for _ in range(2):
        rho = np.exp(rng.uniform(-1, 1))
        p = np.exp(rng.uniform(-1, 1))
        a = np.sqrt(G * p / rho)
        t = rng.normal(size=dim)
        t -= (t @ n) * n
        vn = rng.uniform(*vn_range) * a
        out.append((rho, vn * n + 0.5 * t, p))
    if data_condition:  # (gamma - 1)/2 v_n^D <= a^D
        rho, v, p = out[1]
        a = np.sqrt(G * p / rho)
        vn = v @ n
        if 0.5 * (G - 1) * vn > a:
            v = v - (vn - a) * n
        out[1] = (rho, v, p)
    return n, _cons(*out[0]), _cons(*out[1])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("bc", ["characteristic", "godunov"])
def test_nonreflecting_fixed_point(dim, bc):
    """U^D = U: every characteristic already matches, so U^P = U (all regimes)."""
    rng = np.random.default_rng(10 + dim)
    f = oracle.bc_characteristic if bc == "characteristic" else oracle.bc_godunov
    for vr in ((-3, -1.2), (-0.9, -0.05), (0.05, 0.9), (1.2, 3)):
        for _ in range(50):
            n, u, _ = _random_pair(rng, dim, vr)
            up = f(u, n, u)
            assert np.allclose(up, u, rtol=1e-12, atol=1e-12), (vr, u, up)


@pytest.mark.parametrize("dim", [2, 3])
def test_characteristic_supersonic_cases(dim):
    rng = np.random.default_rng(20 + dim)
    for _ in range(200):
        n, u, ud = _random_pair(rng, dim, (-4, -1.01))  # supersonic inflow: U^P = U^D
        assert np.array_equal(oracle.bc_characteristic(u, n, ud), ud)
        n, u, ud = _random_pair(rng, dim, (1.0, 4))  # supersonic outflow: U^P = U
        assert np.array_equal(oracle.bc_characteristic(u, n, ud), u)


@pytest.mark.parametrize("dim", [2, 3])
def test_characteristic_invariants_match_their_sources(dim):
    """Subsonic inflow: C1, S, v^perp from U^D and C3 from U. Subsonic outflow:
    C1 from U^D and C3, S, v^perp from U."""
    rng = np.random.default_rng(30 + dim)
    for inflow in (True, False):
        for _ in range(300):
            n, u, ud = _random_pair(rng, dim, (-0.95, -0.01) if inflow else (0.0, 0.95))
            up = oracle.bc_characteristic(u, n, ud)
            iu, idd, ip = _invariants(u, n), _invariants(ud, n), _invariants(up, n)
            assert np.isclose(ip["C1"], idd["C1"], rtol=1e-12, atol=1e-12)
            assert np.isclose(ip["C3"], iu["C3"], rtol=1e-12, atol=1e-12)
            src = idd if inflow else iu
            assert np.isclose(ip["S"], src["S"], rtol=1e-11)
            assert np.allclose(ip["vt"], src["vt"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("bc", ["characteristic", "godunov"])
def test_nonreflecting_output_is_admissible(bc):
    """Lemma 4.3: admissible U and Dirichlet data with (gamma-1)/2 v_n^D <= a^D
    give an admissible post-processed state."""
    rng = np.random.default_rng(40)
    f = oracle.bc_characteristic if bc == "characteristic" else oracle.bc_godunov
    for _ in range(2000):
        n, u, ud = _random_pair(rng, 2, (-3, 3))
        up = f(u, n, ud)
        rho, v, p, *_ = _prim(up, n)
        assert rho > 0 and p > 0, (u, ud, up)


def test_godunov_is_the_exact_riemann_value_at_the_interface():
    """The Godunov value is the exact solution at x/t = 0 of the Riemann
    problem along n (left: U, right: U^D); the tangential velocity is carried
    by the contact (upwind side)."""
    rng = np.random.default_rng(50)
    checked = 0
    for _ in range(3000):
        n, u, ud = _random_pair(rng, 2, (-2.5, 2.5), data_condition=False)
        rl, vl, pl, al, ul, tl = _prim(u, n)
        rr, vr, pr, ar, ur, tr = _prim(ud, n)
        if 2 * (al + ar) / (G - 1) <= ur - ul:
            continue  # vacuum between the rarefactions
        rho, un, p = RE.sample(np.array([0.5]), 1.0, rl, ul, pl, rr, ur, pr, gamma=G, x0=0.5)
        _, us = RE.star_pressure(rl, ul, pl, rr, ur, pr, gamma=G)
        vt = tl if float(us) >= 0 else tr
        ref = _cons(rho[0], un[0] * n + vt, p[0])
        up = oracle.bc_godunov(u, n, ud)
        assert np.allclose(up, ref, rtol=1e-9, atol=1e-10), (u, ud, up, ref)
        checked += 1
    assert checked > 2500


@pytest.mark.parametrize("bc", ["characteristic", "godunov"])
def test_nonreflecting_rotation_invariance(bc):
    rng = np.random.default_rng(60)
    f = oracle.bc_characteristic if bc == "characteristic" else oracle.bc_godunov
    for _ in range(300):
        n, u, ud = _random_pair(rng, 2, (-2, 2))
        th = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])

        def rot(w):
            return np.concatenate([[w[0]], R @ w[1:3], [w[3]]])
        up = f(u, n, ud)
        upr = f(rot(u), R @ n, rot(ud))
        assert np.allclose(upr, rot(up), rtol=1e-11, atol=1e-12)
