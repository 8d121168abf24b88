"""Exact solution of the 1D Riemann problem of the ideal-gas Euler equations.

Test-only helper used to pin the oracle: the star pressure p* solves
  f_L(p) + f_R(p) + (u_R - u_L) = 0,
  f_K(p) = (p - p_K) sqrt(A_K / (p + B_K))           if p > p_K (shock),
  f_K(p) = 2 a_K/(gamma-1) ((p/p_K)^z - 1)           if p <= p_K (rarefaction),
with A_K = 2/((gamma+1) rho_K), B_K = (gamma-1)/(gamma+1) p_K and
z = (gamma-1)/(2 gamma) (Toro, Riemann Solvers and Numerical Methods, ch. 4),
found by safeguarded Newton iterations. Vectorised over numpy arrays.
"""
from __future__ import annotations

import numpy as np


def _f_and_df(p, rho, pk, a, gamma):
    A = 2.0 / ((gamma + 1.0) * rho)
    B = (gamma - 1.0) / (gamma + 1.0) * pk
    z = (gamma - 1.0) / (2.0 * gamma)
    shock = p > pk
    ps = np.where(shock, p, pk)
    sq = np.sqrt(A / (ps + B))
    f_s = (ps - pk) * sq
    df_s = sq * (1.0 - 0.5 * (ps - pk) / (ps + B))
    pr = np.where(shock, pk, np.maximum(p, 1e-300))
    f_r = 2.0 * a / (gamma - 1.0) * ((pr / pk) ** z - 1.0)
    df_r = (pr / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * a)
    return np.where(shock, f_s, f_r), np.where(shock, df_s, df_r)


def star_pressure(rl, ul, pl, rr, ur, pr, gamma=1.4, iters=100):
    """p* and u* of the exact solution; p* = 0 when a vacuum forms."""
    rl, ul, pl, rr, ur, pr = (np.asarray(v, dtype=np.float64) for v in (rl, ul, pl, rr, ur, pr))
    al = np.sqrt(gamma * pl / rl)
    ar = np.sqrt(gamma * pr / rr)
    du = ur - ul
    vacuum = 2.0 * (al + ar) / (gamma - 1.0) <= du
    # bracket: F(p) = f_L + f_R + du is increasing in p
    lo = np.zeros_like(pl)
    hi = np.maximum(pl, pr)
    for _ in range(200):
        fl, _ = _f_and_df(hi, rl, pl, al, gamma)
        fr, _ = _f_and_df(hi, rr, pr, ar, gamma)
        need = (fl + fr + du) < 0
        if not need.any():
            break
        hi = np.where(need, hi * 2.0, hi)
    p = 0.5 * (lo + hi)
    for _ in range(iters):
        fl, dfl = _f_and_df(p, rl, pl, al, gamma)
        fr, dfr = _f_and_df(p, rr, pr, ar, gamma)
        F = fl + fr + du
        lo = np.where(F < 0, p, lo)
        hi = np.where(F >= 0, p, hi)
        pn = p - F / (dfl + dfr)
        bad = ~((pn > lo) & (pn < hi))
        p = np.where(bad, 0.5 * (lo + hi), pn)
    p = np.where(vacuum, 0.0, p)
    fl, _ = _f_and_df(np.maximum(p, 1e-300), rl, pl, al, gamma)
    fr, _ = _f_and_df(np.maximum(p, 1e-300), rr, pr, ar, gamma)
    us = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, us


def max_wave_speed(rl, ul, pl, rr, ur, pr, gamma=1.4):
    """max(|lambda_1^-|, |lambda_3^+|) of the exact solution (outermost waves)."""
    p, _ = star_pressure(rl, ul, pl, rr, ur, pr, gamma)
    al = np.sqrt(gamma * pl / rl)
    ar = np.sqrt(gamma * pr / rr)
    k = (gamma + 1.0) / (2.0 * gamma)
    sl = np.where(p > pl, ul - al * np.sqrt(1.0 + k * (p - pl) / pl), ul - al)
    sr = np.where(p > pr, ur + ar * np.sqrt(1.0 + k * (p - pr) / pr), ur + ar)
    return np.maximum(np.maximum(-sl, 0.0), np.maximum(sr, 0.0)), p


def sample(x, t, rl, ul, pl, rr, ur, pr, gamma=1.4, x0=0.5):
    """Exact (rho, u, p) at positions x and time t > 0 (scalar data)."""
    ps, us = star_pressure(rl, ul, pl, rr, ur, pr, gamma)
    ps, us = float(ps), float(us)
    g = gamma
    al, ar = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    s = (np.asarray(x, dtype=np.float64) - x0) / t
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    # left of contact
    left = s <= us
    if ps > pl:  # left shock
        sl = ul - al * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
        rls = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
        m0 = left & (s < sl)
        m1 = left & (s >= sl)
        rho[m0], u[m0], p[m0] = rl, ul, pl
        rho[m1], u[m1], p[m1] = rls, us, ps
    else:  # left rarefaction
        rls = rl * (ps / pl) ** (1.0 / g) if ps > 0 else 0.0
        als = al * (ps / pl) ** ((g - 1) / (2 * g)) if ps > 0 else 0.0
        shl = ul - al
        stl = us - als if ps > 0 else ul + 2 * al / (g - 1)
        m0 = left & (s < shl)
        m1 = left & (s >= shl) & (s < stl)
        m2 = left & (s >= stl)
        rho[m0], u[m0], p[m0] = rl, ul, pl
        uf = 2.0 / (g + 1) * (al + (g - 1) / 2 * ul + s[m1])
        rho[m1] = rl * (2.0 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s[m1])) ** (2.0 / (g - 1))
        u[m1] = uf
        p[m1] = pl * (2.0 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s[m1])) ** (2.0 * g / (g - 1))
        rho[m2], u[m2], p[m2] = rls, us, ps
    right = ~left
    if ps > pr:
        sr = ur + ar * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        rrs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
        m0 = right & (s > sr)
        m1 = right & (s <= sr)
        rho[m0], u[m0], p[m0] = rr, ur, pr
        rho[m1], u[m1], p[m1] = rrs, us, ps
    else:
        rrs = rr * (ps / pr) ** (1.0 / g) if ps > 0 else 0.0
        ars = ar * (ps / pr) ** ((g - 1) / (2 * g)) if ps > 0 else 0.0
        shr = ur + ar
        str_ = us + ars if ps > 0 else ur - 2 * ar / (g - 1)
        m0 = right & (s > shr)
        m1 = right & (s <= shr) & (s > str_)
        m2 = right & (s <= str_)
        rho[m0], u[m0], p[m0] = rr, ur, pr
        u[m1] = 2.0 / (g + 1) * (-ar + (g - 1) / 2 * ur + s[m1])
        rho[m1] = rr * (2.0 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s[m1])) ** (2.0 / (g - 1))
        p[m1] = pr * (2.0 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s[m1])) ** (2.0 * g / (g - 1))
        rho[m2], u[m2], p[m2] = rrs, us, ps
    return rho, u, p
