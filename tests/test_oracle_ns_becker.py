"""Pin of the oracle's Navier-Stokes step (Strang splitting of the hyperbolic
and parabolic sub-steps, Sec. 5) against an exact solution of the
compressible Navier-Stokes equations: the steady viscous shock of Becker,
which Sec. 6.1 uses to verify the full algorithm (second-order convergence,
Table tab:becker-validation). The paper takes its parameters from a cited
work; here: gamma = 1.4, upstream rho = 1, p = 1/gamma (a = 1), Mach 2,
mu = 0.02, lambda = 0, Prandtl number 3/4 (kappa/c_v = 4 mu gamma / 3), the
shock at rest, Dirichlet data at x = -1/2 and x = 1/2, periodic in y.

The profile follows from the steady 1D equations in the shock frame. Mass:
rho v = m. With Pr = 3/4 the energy equation reads m H - (4/3) mu H' = const
for the total enthalpy H = gamma e + v^2/2, so H = H0 throughout. Momentum,
m v + p - (4/3) mu v' = m v_L + p_L with p = (m/v) (gamma-1)/gamma (H0 - v^2/2),
becomes
    (4/3) (mu/m) v v' = (gamma+1)/(2 gamma) (v - v_L)(v - v_R),
v_L, v_R the two roots (the Rankine-Hugoniot states), whose integral is
    x(v) = K/(v_L - v_R) [v_L ln((v_L - v)/(v_L - v0)) - v_R ln((v - v_R)/(v0 - v_R))],
K = 8 gamma mu / (3 m (gamma+1)), centred where v = v0 = (v_L + v_R)/2. The test
inverts it by bisection, so it shares nothing with the oracle. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2106_02159_gb300 import meshes as M

GAMMA = 1.4


def becker_state(x, mach=2.0, mu=0.02):
    g = GAMMA
    rho_l, v_l, p_l = 1.0, mach, 1.0 / g
    m = rho_l * v_l
    H0 = g * p_l / ((g - 1.0) * rho_l) + 0.5 * v_l ** 2
    c = v_l + p_l / m
    a2, a0 = (g + 1.0) / (2.0 * g), (g - 1.0) / g * H0
    disc = np.sqrt(c * c - 4.0 * a2 * a0)
    assert abs((c + disc) / (2.0 * a2) - v_l) < 1e-12 * v_l  # the upstream state is a root
    v_r = (c - disc) / (2.0 * a2)
    K = 8.0 * g * mu / (3.0 * m * (g + 1.0))
    v0 = 0.5 * (v_l + v_r)

    def x_of_v(v):
        return K / (v_l - v_r) * (v_l * np.log((v_l - v) / (v_l - v0)) - v_r * np.log((v - v_r) / (v0 - v_r)))

    lo, hi = np.full_like(x, v_r * (1.0 + 1e-15)), np.full_like(x, v_l * (1.0 - 1e-15))
    for _ in range(200):  # x(v) decreases in v
        mid = 0.5 * (lo + hi)
        right = x_of_v(mid) < x
        hi, lo = np.where(right, mid, hi), np.where(right, lo, mid)
    v = 0.5 * (lo + hi)
    rho = m / v
    e = (H0 - 0.5 * v * v) / g
    return np.stack([rho, rho * v, np.zeros_like(v), rho * (e + 0.5 * v * v)])


def run(nx, mu=0.02, kappa_factor=1.0, mu_factor=1.0, t_end=0.3):
    """Density L1 error (relative) after t_end of Navier-Stokes steps started
    from the exact profile (the solver's viscosity and heat conduction scaled
    by mu_factor and kappa_factor)."""
    mesh = M.structured_q1(nx, 2, -0.5, 0.5, 0.0, 2.0 / nx, periodic_y=True,
                           kinds=(M.BC_DIRICHLET, M.BC_DIRICHLET, M.BC_SLIP, M.BC_SLIP))
    U0 = becker_state(mesh.coords[:, 0], mu=mu)
    o = oracle.Oracle(mesh, bnd_state=np.ascontiguousarray(U0[:, mesh.bnd_node]), cfl=0.5)
    o.set_viscosity(M.parabolic_data(mesh), mu_factor * mu, 0.0, kappa_factor * 4.0 * mu * GAMMA / 3.0)
    U, t = o.apply_bc(U0), 0.0
    while t < t_end - 1e-14:
        U, tau, info = o.ns_step(U)
        t += 2.0 * tau
    assert (U[0] > 0).all()
    return np.abs(U[0] - U0[0]).sum() / np.abs(U0[0]).sum()


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(0)


def test_becker_shock_is_kept_at_second_order():
    e100, e200 = run(100), run(200)
    # measured: 6.8e-4 and 1.3e-4 (rate 2.4; 2.1e-5 at 400 cells, rate 2.6)
    assert e200 < 3e-4, e200
    assert e100 / e200 > 3.0, (e100, e200)


def test_becker_pin_rejects_wrong_transport_coefficients():
    # a Prandtl number other than 3/4 (heat conduction doubled) or a wrong
    # viscosity breaks the constant total enthalpy the exact profile rests on
    ok = run(200)
    assert run(200, kappa_factor=2.0) > 20.0 * ok   # measured 7.5e-3
    assert run(200, mu_factor=1.25) > 20.0 * ok     # measured 4.7e-3
